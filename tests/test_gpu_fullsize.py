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


def test_lens_solve_operators_commute_with_the_mirror_at_full_size(ssx):
    """The single-shot lens workload (601 x 301, order 8, 3000 steps) has
    x_s, the source line and the receivers on or centred on the middle
    column. With its model made exactly symmetric about that column,
    reflecting the gathers about x_s commutes with S, S^T, the three
    thin-slab weights and M^{-1} (the staggered grid, the sponge ramps and
    |x - x_s| map onto themselves), and the solve of reflected data returns
    the reflected source: a property of the full-size launches that needs
    no oracle run."""
    from paper_2203_16573_gb300 import ssx as S
    spec = W.c2()
    v = W.velocity(spec)
    ctx = ssx.Context.for_problem(spec, 0.5 * (v + v[:, ::-1]))
    h = dev(W.smooth_random_gather(spec.nt, spec.n_line, 61))
    d = dev(W.smooth_random_gather(spec.nt, spec.n_rec, 62))
    flip = lambda a: torch.flip(a, dims=[1])
    ops = ((ctx.forward, h), (ctx.adjoint, d), (lambda x: ctx.weight_apply(S.W_D, x), d),
           (lambda x: ctx.weight_apply(S.W_M, x), h), (lambda x: ctx.weight_apply(S.W_M_INV, x), h),
           (lambda x: ctx.precond_apply(spec.alpha, x), h))
    for k, (op, x) in enumerate(ops):
        y = op(x).clone()
        ym = op(flip(x).contiguous())
        assert float(y.norm()) > 0, k
        if k < 5:
            # every term of every update is negated or kept exactly under the
            # reflection, and each sum keeps its order: bit for bit
            assert torch.equal(flip(y), ym), k
        else:
            # M^-1's scaling D = (1 + alpha |x - x_s|^2)^(-1/2) rounds |x - x_s|
            # differently on the two sides
            assert float((flip(y) - ym).norm() / y.norm()) <= 1e-12, k
    d0 = ctx.point_source_data(spec.x_d, spec.z_d, torch.as_tensor(W.ricker(spec), device="cuda"))
    d1 = d0 + 0.05 * float(d0.abs().max()) * d     # not symmetric by itself
    h1, hist1, _, _ = ctx.solve(d1, spec.alpha, 3, 0.0)
    h1 = h1.clone()
    h2, hist2, _, _ = ctx.solve(flip(d1).contiguous(), spec.alpha, 3, 0.0)
    assert float((flip(h1) - h2).norm() / h1.norm()) <= 1e-5
    np.testing.assert_allclose(hist2, hist1, rtol=1e-5)
