"""Serving source-subproblem solves: a seeded Poisson request stream of
mixed grid sizes, run through the continuous-batching server (ssx_server_*)
or one request at a time, with per-request latencies.

The request mix follows the serving workload of this library's measurement
set: grids drawn uniformly from {401 x 201 (h = 10 m), 1001 x 401 (h = 8 m),
2001 x 801 (h = 5 m)}, 1000-5000 steps, dt at CFL 0.25 of the 3 km/s
maximum, random shot positions on seeded lens or gradient models; the
extended-source line sits at 80 % of the depth through the shot, or higher
when the record is short: no deeper than 0.6 km per second of record, so
that the wave (at >= 1.2 km/s, the slowest speed of the models) reaches the
surface receivers within the first half of the record; the data come from a
Ricker point source at the shot on the line. `scale` shrinks the grids and
step counts for quick runs.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch

from . import ssx, workloads as W

SIZES = [(401, 201, 0.010), (1001, 401, 0.008), (2001, 801, 0.005)]


def request_specs(n: int, rate_hz: float, seed: int = 0, scale: float = 1.0, maxit: int = 30,
                  rtol: float = 1e-3, order: int = 8, nt_range=(1000, 5000)):
    """[(arrival time s, Spec)] of a seeded Poisson stream of n requests."""
    rng = np.random.default_rng(W.SEED + 1000 + seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        nx, nz, h = SIZES[rng.integers(len(SIZES))]
        nx, nz = max(33, int(round(nx * scale))) | 1, max(25, int(round(nz * scale))) | 1
        nt = max(60, int(round(rng.integers(nt_range[0], nt_range[1] + 1) * scale)))
        dt = 0.25 * h / 3.0
        model = "gradient_lens" if rng.random() < 0.5 else "gradient"
        zmax = (nz - 1) * h
        dz = max(0.1, 4 * h)
        z_lo = dz + 4 * h    # the W~_m slab's datum dz above the line stays inside the model
        k_s = round(min(0.8 * zmax, max(z_lo, 0.6 * nt * dt)) / h)
        if k_s * h < z_lo - 1e-12:
            k_s += 1
        z_s = k_s * h
        ixs = int(rng.integers(nx // 5, 4 * nx // 5))
        xs = ixs * h
        spec = W.Spec(name=f"req{i}_{nx}x{nz}_nt{nt}", nx=nx, nz=nz, h=h, dt=dt, nt=nt,
                      order=order, n_sponge=20 if scale < 1 else 40, rho=1.0, z_s=z_s,
                      ix_line0=0, n_line=nx, z_r=0.0, ix_rec0=0, n_rec=nx, x_s=xs, x_d=xs,
                      z_d=z_s, f_peak=15.0,
                      alpha=(1e-3, 1e-2, 1e-1)[int(rng.integers(3))], maxit=maxit, rtol=rtol,
                      dz_datum=dz, model=model)
        out.append((t, spec))
    return out


def make_inputs(specs, device="cuda"):
    """Model and data gather (device) of every request, computed before any
    timing: the data of request i come from its own point source."""
    inputs = []
    for _, sp in specs:
        vel = torch.as_tensor(W.velocity(sp), dtype=torch.float32, device=device).contiguous()
        ctx = ssx.Context.from_spec(sp)
        ctx.set_velocity_model(vel, sp.rho)
        ctx.set_geometry(sp.z_s, sp.ix_line0, sp.n_line, sp.z_r, sp.ix_rec0, sp.n_rec, sp.x_s,
                         sp.dz_datum)
        d = ctx.point_source_data(sp.x_d, sp.z_d, torch.as_tensor(W.ricker(sp), device=device))
        torch.cuda.synchronize()
        ctx.close()
        inputs.append((vel, d))
    return inputs


def serve(specs, inputs, hbm_budget_bytes=80 * 10 ** 9, order=8, realtime=True, stats=None,
          cache_budget=None):
    """Continuous batching: requests are submitted at their arrival times
    (host clock from the start) and served by one ssx_server. Returns
    (outputs, per-request records, wall seconds); `stats` (a dict, optional)
    receives the server's counters with its shared launches event-timed."""
    srv = ssx.Server(order, hbm_budget_bytes)
    if cache_budget is not None:
        srv.set_cache_budget(cache_budget)
    if stats is not None:
        srv.set_timing(True)
    outs = [torch.empty(sp.nt, sp.n_line, dtype=torch.float64, device="cuda") for _, sp in specs]
    ids = [None] * len(specs)
    t0 = time.perf_counter()
    nxt = 0
    done = set()
    records = [None] * len(specs)
    while len(done) < len(specs):
        now = time.perf_counter() - t0
        while nxt < len(specs) and (not realtime or specs[nxt][0] <= now):
            sp = specs[nxt][1]
            ids[nxt] = srv.submit(sp, inputs[nxt][0], inputs[nxt][1], outs[nxt])
            nxt += 1
        a, q = srv.step()
        for i, rid in enumerate(ids):
            if rid is None or i in done:
                continue
            r = srv.poll(rid)
            if r["done"]:
                done.add(i)
                records[i] = r
        if a == 0 and q == 0 and nxt < len(specs):   # idle until the next arrival
            time.sleep(max(0.0, min(0.01, specs[nxt][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    if stats is not None:
        stats.update(srv.stats())
    srv.close()
    return outs, records, wall


def serve_one_at_a_time(specs, inputs, realtime=True, stats=None):
    """The plain one-shot-at-a-time solve: requests in arrival order, each
    solved alone; latency = completion - arrival. `stats` (optional) receives
    the summed event-timed sweep time and point updates of the solves."""
    outs, records = [], []
    tot = {"sweep_ms": 0.0, "timed_point_updates": 0.0, "kernel_launches": 0}
    t0 = time.perf_counter()
    for (arr, sp), (vel, d) in zip(specs, inputs):
        if realtime:
            wait = arr - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        start = time.perf_counter() - t0
        ctx = ssx.Context.from_spec(sp)
        ctx.set_velocity_model(vel, sp.rho)
        ctx.set_geometry(sp.z_s, sp.ix_line0, sp.n_line, sp.z_r, sp.ix_rec0, sp.n_rec, sp.x_s,
                         sp.dz_datum)
        if stats is not None:
            ctx.set_timing(True)
        h, hist, iters, status = ctx.solve(d, sp.alpha, sp.maxit, sp.rtol, allow_breakdown=True)
        torch.cuda.synchronize()
        if stats is not None:
            st = ctx.stats()
            for k in tot:
                tot[k] += st[k]
        ctx.close()
        end = time.perf_counter() - t0
        outs.append(h)
        records.append({"done": True, "status": status, "iters": iters,
                        "latency_ms": 1000.0 * (end - (arr if realtime else 0.0)),
                        "queue_ms": 1000.0 * (start - (arr if realtime else 0.0))})
    if stats is not None:
        stats.update(tot)
    return outs, records, time.perf_counter() - t0


def percentiles(records):
    lat = np.array([r["latency_ms"] for r in records])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
