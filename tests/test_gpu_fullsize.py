"""The batched survey workload at its full size (2001 x 801 model at h = 5 m,
order 8, 5000 steps): one shot's S h against the FP64 oracle, and two shots
solved in shared launches against their solo solves, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2203_16573_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def ssx():
    from paper_2203_16573_gb300 import build, ssx as mod
    build.build()
    return mod


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_survey_shot_forward_matches_oracle_at_full_size(ssx, oracle):
    sp = W.c3_shots(64)[21]
    vel = W.velocity(sp)
    ctx = ssx.Context.for_problem(sp, vel)
    h = W.smooth_random_gather(sp.nt, sp.n_line, 41)
    d = ctx.forward(dev(h)).cpu().numpy()
    ref = oracle.Problem(sp, vel).S(h)
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(d - ref) / np.linalg.norm(ref) <= TOL


def test_survey_shots_batched_equal_solo_at_full_size(ssx):
    specs = [W.c3_shots(64)[k] for k in (10, 40)]
    vel = torch.as_tensor(W.velocity(specs[0]), dtype=torch.float32, device="cuda")
    ctxs, ds = [], []
    for sp in specs:
        c = ssx.Context.from_spec(sp)
        c.set_velocity_model(vel, sp.rho)
        c.set_geometry(sp.z_s, sp.ix_line0, sp.n_line, sp.z_r, sp.ix_rec0, sp.n_rec, sp.x_s,
                       sp.dz_datum)
        ds.append(c.point_source_data(sp.x_d, sp.z_d, torch.as_tensor(W.ricker(sp), device="cuda")))
        ctxs.append(c)
    hb, hists, iters, status = ssx.solve_batch(ctxs, ds, [sp.alpha for sp in specs], 1, 0.0,
                                               ssx.MODE_PCG)
    for c, d, sp, h, hh in zip(ctxs, ds, specs, hb, hists):
        h1, hh1, it1, _ = c.solve(d, sp.alpha, 1, 0.0, ssx.MODE_PCG)
        assert it1 == 1 and float(h1.abs().max()) > 0
        assert torch.equal(h, h1)
        np.testing.assert_array_equal(hh, hh1)
