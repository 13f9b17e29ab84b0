"""Continuous batching (NEXT-2): requests that arrive while others run join
the shared launches at the next round, are admitted by a device-memory
budget, and each result is the same alone and in the mix."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2203_16573_gb300 import build, serve, ssx
    build.build()
    specs = serve.request_specs(5, 50.0, seed=3, scale=0.12, maxit=5, rtol=1e-6)
    inputs = serve.make_inputs(specs)
    solo = []
    for (_, sp), (vel, d) in zip(specs, inputs):
        c = ssx.Context.from_spec(sp)
        c.set_velocity_model(vel, sp.rho)
        c.set_geometry(sp.z_s, sp.ix_line0, sp.n_line, sp.z_r, sp.ix_rec0, sp.n_rec, sp.x_s,
                       sp.dz_datum)
        h, hist, it, st = c.solve(d, sp.alpha, sp.maxit, sp.rtol)
        solo.append((h.clone(), it, st))
        c.close()
    return ssx, specs, inputs, solo


def test_requests_joining_mid_flight_match_solo_solves(env):
    ssx, specs, inputs, solo = env
    srv = ssx.Server(8, 80 * 10 ** 9)
    outs = [torch.full((sp.nt, sp.n_line), float("nan"), dtype=torch.float64, device="cuda")
            for _, sp in specs]
    ids = [srv.submit(specs[i][1], *inputs[i], outs[i]) for i in range(2)]
    for _ in range(3):                     # the first two are mid-solve ...
        srv.step()
    ids += [srv.submit(specs[i][1], *inputs[i], outs[i]) for i in range(2, 5)]   # ... when these arrive
    for _ in range(100):
        a, q = srv.step()
        if a == 0 and q == 0:
            break
    for i, rid in enumerate(ids):
        r = srv.poll(rid)
        assert r["done"] and r["status"] == solo[i][2] and r["iters"] == solo[i][1]
        assert torch.equal(outs[i], solo[i][0])
    srv.close()


def test_memory_budget_admits_one_at_a_time_and_results_hold(env):
    ssx, specs, inputs, solo = env
    srv = ssx.Server(8, 1)                  # no room for two: strictly one admitted at a time
    outs = [torch.empty(sp.nt, sp.n_line, dtype=torch.float64, device="cuda") for _, sp in specs]
    ids = [srv.submit(specs[i][1], *inputs[i], outs[i]) for i in range(3)]
    seen_queue = False
    for _ in range(200):
        a, q = srv.step()
        assert a <= 1
        seen_queue = seen_queue or q > 0
        if a == 0 and q == 0:
            break
    assert seen_queue
    for i, rid in enumerate(ids):
        r = srv.poll(rid)
        assert r["done"] and torch.equal(outs[i], solo[i][0])
    assert srv.poll(ids[2])["queue_ms"] > 0
    srv.close()


def test_requests_served_in_a_mix_match_the_oracle(oracle):
    """Three requests of different grids served together (the third joins
    while the first two are mid-solve), each compared with the FP64 oracle's
    Algorithm 1 on the same inputs: the same iteration count and h within
    1e-4 relative L2 (element by element). The data gathers are the
    oracle's own point-source data."""
    from paper_2203_16573_gb300 import build, serve, ssx, workloads as W
    build.build()
    specs = serve.request_specs(3, 50.0, seed=5, scale=0.12, maxit=5, rtol=0.0)
    probs, ins = [], []
    for _, sp in specs:
        vel = W.velocity(sp)
        P = oracle.Problem(sp, vel)
        d = P.point_source_data(W.ricker(sp), sp.x_d, sp.z_d)
        probs.append((P, d))
        ins.append((torch.as_tensor(vel, dtype=torch.float32, device="cuda").contiguous(),
                    torch.as_tensor(d, dtype=torch.float64, device="cuda")))
    srv = ssx.Server(8, 80 * 10 ** 9)
    outs = [torch.full((sp.nt, sp.n_line), float("nan"), dtype=torch.float64, device="cuda")
            for _, sp in specs]
    ids = [srv.submit(specs[i][1], *ins[i], outs[i]) for i in range(2)]
    srv.step()
    srv.step()
    ids.append(srv.submit(specs[2][1], *ins[2], outs[2]))
    for _ in range(100):
        a, q = srv.step()
        if a == 0 and q == 0:
            break
    for (_, sp), (P, d), rid, h in zip(specs, probs, ids, outs):
        r = srv.poll(rid)
        assert r["done"] and r["iters"] == sp.maxit
        h_or, hist_or = oracle.pcg(P, d, sp.alpha, sp.maxit, sp.rtol)
        err = float(np.linalg.norm(h.cpu().numpy() - h_or) / np.linalg.norm(h_or))
        assert err <= 1e-4, (sp.name, err)
    srv.close()
