"""Host logic of the serving workload (CPU): the seeded Poisson request
stream that the continuous-batching server and the one-at-a-time baseline
are both fed. Checks the stream's statistics and every request's recipe
(grid sizes, step counts, CFL time step, line and shot geometry)."""
import math

import numpy as np

from paper_2203_16573_gb300 import serve


def test_stream_is_seeded():
    a = serve.request_specs(20, 4.0, seed=5)
    b = serve.request_specs(20, 4.0, seed=5)
    c = serve.request_specs(20, 4.0, seed=6)
    assert [(t, s) for t, s in a] == [(t, s) for t, s in b]
    assert [t for t, _ in a] != [t for t, _ in c]


def test_arrivals_are_poisson_at_the_requested_rate():
    rate, n = 4.0, 4000
    t = np.array([t for t, _ in serve.request_specs(n, rate, seed=1)])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate (standard error 1/(rate sqrt n) = 1.6 %),
    # coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.06


def test_every_request_follows_the_recipe():
    specs = serve.request_specs(300, 4.0, seed=2)
    seen = set()
    for _, s in specs:
        assert (s.nx, s.nz, s.h) in serve.SIZES
        seen.add((s.nx, s.nz, s.h))
        assert 1000 <= s.nt <= 5000
        assert math.isclose(3.0 * s.dt / s.h, 0.25)           # CFL 0.25 at 3 km/s
        assert s.order == 8 and s.n_sponge == 40
        k_s = s.z_s / s.h                                      # line on a grid row at 80 % depth,
        assert abs(k_s - round(k_s)) < 1e-9                    # or 0.6 km per second of record
        zmax, T = (s.nz - 1) * s.h, s.nt * s.dt
        assert abs(s.z_s - min(0.8 * zmax, max(0.6 * T, s.dz_datum + 4 * s.h))) <= s.h + 1e-12
        assert s.z_s - s.dz_datum >= 4 * s.h - 1e-12
        i_s = s.x_s / s.h                                      # shot on a column, inside the middle 3/5
        assert abs(i_s - round(i_s)) < 1e-9 and s.nx // 5 <= round(i_s) < 4 * s.nx // 5
        assert (s.x_d, s.z_d) == (s.x_s, s.z_s)
        assert s.ix_line0 == 0 and s.n_line == s.nx and s.ix_rec0 == 0 and s.n_rec == s.nx
        assert s.z_r == 0.0 and s.alpha in (1e-3, 1e-2, 1e-1)
        assert s.model in ("gradient", "gradient_lens")
    assert seen == set(serve.SIZES)


def test_scaled_stream_keeps_odd_grids_and_minimum_sizes():
    for scale in (0.05, 0.12):
        for _, s in serve.request_specs(50, 4.0, seed=3, scale=scale):
            assert s.nx % 2 == 1 and s.nz % 2 == 1
            assert s.nx >= 33 and s.nz >= 25 and s.nt >= 60
            assert s.n_sponge == 20
            assert s.z_s - s.dz_datum >= 4 * s.h - 1e-12 and s.z_s <= (s.nz - 1) * s.h


def test_latency_percentiles():
    recs = [{"latency_ms": float(v)} for v in range(1, 101)]
    p = serve.percentiles(recs)
    assert p["p50_ms"] == 50.5 and p["mean_ms"] == 50.5
    assert 99.0 < p["p99_ms"] < 100.0
