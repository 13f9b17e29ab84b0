"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (the solver's stated bar): traces, gathers and recovered sources
within 1e-4 relative L2; PCG residual histories within 1e-3 relative per
iteration. GPU fields are FP32, Krylov vectors and scalars FP64.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from paper_2203_16573_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4
HIST_TOL = 1e-3


def rel(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ssx():
    from paper_2203_16573_gb300 import build, ssx as S
    build.build()
    assert torch.cuda.is_available()
    return S


def make(ssx, oracle, spec):
    vel = W.velocity(spec)
    return ssx.Context.for_problem(spec, vel), oracle.Problem(spec, vel)


def frac_spec(order, nt=300, **kw):
    """small c2-like case with both lines between grid rows (interpolation)"""
    return dataclasses.replace(W.small(order=order, nt=nt), z_s=0.5537, z_r=0.0471, **kw)


# ------------------------------------------------------------- S and S^T --
@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("fractional", [False, True])
def test_forward_and_adjoint_parity(ssx, oracle, order, fractional):
    spec = frac_spec(order) if fractional else W.small(order=order, nt=300)
    ctx, P = make(ssx, oracle, spec)
    h = W.smooth_random_gather(spec.nt, spec.n_line, 1)
    d = W.smooth_random_gather(spec.nt, spec.n_rec, 2)
    assert rel(ctx.forward(dev(h)), P.S(h)) <= TOL
    assert rel(ctx.adjoint(dev(d)), P.ST(d)) <= TOL


@pytest.mark.parametrize("order", [4, 8])
def test_gpu_dot_product_test(ssx, order):
    """<S h, d> = <h, S^T d> for the FP32 sweeps (exact transpose up to FP32
    rounding of the fields)."""
    spec = frac_spec(order, nt=500)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    h = dev(W.random_gather(spec.nt, spec.n_line, 3))
    d = dev(W.random_gather(spec.nt, spec.n_rec, 4))
    a = float((ctx.forward(h) * d).sum())
    b = float((h * ctx.adjoint(d)).sum())
    assert abs(a - b) <= 1e-5 * abs(a)


def test_point_source_data_parity(ssx, oracle):
    spec = W.small(order=8, nt=400)
    ctx, P = make(ssx, oracle, spec)
    w = W.ricker(spec)
    d_gpu = ctx.point_source_data(spec.x_d, spec.z_d, dev(w))
    assert rel(d_gpu, P.point_source_data(w, spec.x_d, spec.z_d)) <= TOL


# ---------------------------------------------------------------- weights --
@pytest.mark.parametrize("which", ["Wd", "Wm", "Wminv"])
@pytest.mark.parametrize("fractional", [False, True])
def test_weight_parity(ssx, oracle, which, fractional):
    spec = frac_spec(8) if fractional else W.small(order=8, nt=300)
    ctx, P = make(ssx, oracle, spec)
    code = {"Wd": ssx.W_D, "Wm": ssx.W_M, "Wminv": ssx.W_M_INV}[which]
    n = spec.n_rec if which == "Wd" else spec.n_line
    x = W.smooth_random_gather(spec.nt, n, 5)
    assert rel(ctx.weight_apply(code, dev(x)), getattr(P, which)(x)) <= TOL


@pytest.mark.parametrize("mode", ["pcg", "cg"])
def test_normal_operator_and_preconditioner_parity(ssx, oracle, mode):
    spec = W.small(order=8, nt=300)
    ctx, P = make(ssx, oracle, spec)
    m = ssx.MODE_PCG if mode == "pcg" else ssx.MODE_CG
    x = W.smooth_random_gather(spec.nt, spec.n_line, 6)
    assert rel(ctx.normal_apply(m, 0.3, dev(x)), P.N(x, 0.3, mode)) <= TOL
    assert rel(ctx.normal_apply(m, 0.0, dev(x)), P.N(x, 0.0, mode)) <= TOL
    if mode == "pcg":
        assert rel(ctx.precond_apply(0.3, dev(x)), P.Minv(x, 0.3)) <= TOL


def test_mirrored_geometry_weights_positive_and_match(ssx, oracle):
    """Receivers below the source line: datum side and prefactor sign follow."""
    spec = dataclasses.replace(W.small(order=4, nt=300), z_s=0.08, z_r=0.6)
    ctx, P = make(ssx, oracle, spec)
    x = W.smooth_random_gather(spec.nt, spec.n_line, 7)
    y = ctx.weight_apply(ssx.W_M_INV, dev(x))
    assert rel(y, P.Wminv(x)) <= TOL
    assert float((y * dev(x)).sum()) > 0


# -------------------------------------------------------------------- PCG --
def _check_solve(ctx, P, spec, d, mode, maxit, rtol):
    from paper_2203_16573_gb300 import ssx as S
    m = S.MODE_PCG if mode == "pcg" else S.MODE_CG
    h_or, hist_or = oracle_pcg(P, d, spec.alpha, maxit, rtol, mode)
    h_gpu, hist_gpu, iters, status = ctx.solve(dev(d), spec.alpha, maxit, rtol, m)
    assert iters == len(hist_or) - 1, (iters, len(hist_or))
    herr = np.abs(hist_gpu - hist_or) / hist_or
    print(f"\nsolve parity: h rel L2 {rel(h_gpu, h_or):.3e}, history max rel {herr.max():.3e}")
    np.testing.assert_array_less(herr, HIST_TOL)
    assert rel(h_gpu, h_or) <= TOL
    return h_gpu, hist_gpu, status


def oracle_pcg(P, d, alpha, maxit, rtol, mode):
    from oracle import ssx_oracle
    return ssx_oracle.pcg(P, d, alpha, maxit, rtol, mode)


@pytest.mark.parametrize("mode", ["pcg", "cg"])
def test_pcg_parity_small(ssx, oracle, mode):
    spec = W.small(order=8, nt=500)
    ctx, P = make(ssx, oracle, spec)
    d = P.point_source_data(W.ricker(spec), spec.x_d, spec.z_d)
    _check_solve(ctx, P, spec, d, mode, 12, 0.0)


def test_config1_solve_parity(ssx, oracle):
    """Homogeneous 201 x 101, order 4, 1000 steps, 10 Hz Ricker point source
    on the line, 20 preconditioned CG iterations (rtol 1e-3)."""
    spec = W.c1()
    ctx, P = make(ssx, oracle, spec)
    w = W.ricker(spec)
    d = P.point_source_data(w, spec.x_d, spec.z_d)
    assert rel(ctx.point_source_data(spec.x_d, spec.z_d, dev(w)), d) <= TOL
    _check_solve(ctx, P, spec, d, "pcg", spec.maxit, spec.rtol)


def test_config2_full_solve_parity(ssx, oracle):
    """The bench's workload, solved as the bench solves it: full 601 x 301,
    order 8, 3000-step lens model, 30 preconditioned CG iterations with the
    tile configurations the autotuner picks per phase. Against the oracle:
    the data gather, r_0 = S^T W~_d d as a gather (element by element), the
    whole residual history (1e-3 per entry) and the recovered source h
    (1e-4 relative L2); then the FP32 dot-product test at this size."""
    spec = W.c2()
    ctx, P = make(ssx, oracle, spec)
    w = W.ricker(spec)
    d = P.point_source_data(w, spec.x_d, spec.z_d)
    assert rel(ctx.point_source_data(spec.x_d, spec.z_d, dev(w)), d) <= TOL
    r0 = P.rhs(d)
    assert rel(ctx.adjoint(ctx.weight_apply(ssx.W_D, dev(d))), r0) <= TOL
    h_gpu, hist_gpu, status = _check_solve(ctx, P, spec, d, "pcg", spec.maxit, spec.rtol)
    print(f"\nc2 solve: {len(hist_gpu) - 1} iterations, status {status}, "
          f"final relative residual {hist_gpu[-1] / hist_gpu[0]:.4e}")
    h = dev(W.random_gather(spec.nt, spec.n_line, 8))
    y = dev(W.random_gather(spec.nt, spec.n_rec, 9))
    a, b = float((ctx.forward(h) * y).sum()), float((h * ctx.adjoint(y)).sum())
    assert abs(a - b) <= 1e-5 * abs(a)


def test_second_context_reuses_the_phase_tuning(ssx):
    """Phase tile choices are kept per shape for the process: a second
    context of the single-shot workload's shapes runs its solve on the first
    context's choices (including the TMA-staged kernel, whose grid cap the
    second context looks up itself) and gets the same bits."""
    spec = W.c2()
    vel = W.velocity(spec)
    a = ssx.Context.for_problem(spec, vel)
    d = a.point_source_data(spec.x_d, spec.z_d, dev(W.ricker(spec)))
    ha, hista, ita, _ = a.solve(d, spec.alpha, 3, 0.0)
    ha = ha.clone()
    a.close()
    b = ssx.Context.for_problem(spec, vel)
    hb, histb, itb, _ = b.solve(d, spec.alpha, 3, 0.0)
    assert ita == itb == 3 and torch.equal(ha, hb)
    np.testing.assert_array_equal(hista, histb)


# ------------------------------------------------------------- edge cases --
@pytest.mark.parametrize("nt", [1, 2, 7])
def test_few_steps_and_single_point_lines(ssx, oracle, nt):
    """nt = 1 and 2 (the lines 2 rows apart so one step couples them) and
    one-point lines."""
    spec = dataclasses.replace(W.small(order=4, nt=nt), z_r=0.53, ix_line0=40, n_line=1,
                               ix_rec0=38, n_rec=5)
    ctx, P = make(ssx, oracle, spec)
    h = W.random_gather(spec.nt, 1, 10)
    d = W.random_gather(spec.nt, spec.n_rec, 11)
    for got, ref in ((ctx.forward(dev(h)), P.S(h)), (ctx.adjoint(dev(d)), P.ST(d))):
        if nt == 1:   # one step cannot carry the source two rows up
            assert np.abs(ref).max() == 0 and float(got.abs().max()) == 0.0
        else:
            assert np.abs(ref).max() > 0 and rel(got, ref) <= TOL


def test_no_sponge_tiny_grid_parity(ssx, oracle):
    spec = dataclasses.replace(W.tiny(order=8), n_sponge=0, nx=9, nz=12, ix_line0=0, n_line=9,
                               ix_rec0=0, n_rec=9, z_s=0.08, z_r=0.03, dz_datum=0.02)
    ctx, P = make(ssx, oracle, spec)
    h = W.random_gather(spec.nt, spec.n_line, 12)
    assert rel(ctx.forward(dev(h)), P.S(h)) <= TOL
    x = W.random_gather(spec.nt, spec.n_line, 13)
    assert rel(ctx.weight_apply(ssx.W_M_INV, dev(x)), P.Wminv(x)) <= TOL


def test_zero_data_gives_zero_source(ssx):
    spec = W.small(order=4, nt=100)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    h, hist, iters, status = ctx.solve(torch.zeros(spec.nt, spec.n_rec, dtype=torch.float64,
                                                   device="cuda"), 0.1, 5, 1e-3)
    assert iters == 0 and status == "SSX_OK" and float(h.abs().max()) == 0.0 and hist[0] == 0.0


def test_errors_are_reported_not_raised_from_cuda(ssx):
    spec = W.small(order=4, nt=50)
    ctx = ssx.Context.from_spec(spec)
    # operators before the model and geometry are set: SSX_ERR_ARG, no device work
    assert ctx._lib.ssx_forward(ctx._c, None, None) == 1
    assert b"not called" in ctx._lib.ssx_last_error(ctx._c)
    with pytest.raises(ssx.SSXError) as e:
        ctx.set_geometry(spec.z_s, 0, spec.nx + 1, spec.z_r, 0, 10, spec.x_s)
    assert e.value.code == 1
    with pytest.raises(ssx.SSXError) as e:
        ctx.set_geometry(spec.z_s, 0, 10, spec.z_s, 0, 10, spec.x_s)
    assert e.value.code == 1
    fast = torch.full((spec.nz, spec.nx), 100.0, dtype=torch.float32, device="cuda")
    with pytest.raises(ssx.SSXError) as e:
        ctx.set_velocity_model(fast, 1.0)
    assert e.value.code == 3                      # SSX_ERR_CFL
    ctx.set_velocity_model(torch.as_tensor(W.velocity(spec), dtype=torch.float32, device="cuda"), 1.0)
    ctx.set_geometry(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec, spec.x_s)
    with pytest.raises(TypeError):
        ctx.forward(torch.zeros(spec.nt, spec.n_line, dtype=torch.float32, device="cuda"))


def test_deterministic(ssx):
    spec = frac_spec(8)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    x = dev(W.random_gather(spec.nt, spec.n_line, 14))
    a = ctx.normal_apply(ssx.MODE_PCG, 0.2, x).clone()
    b = ctx.normal_apply(ssx.MODE_PCG, 0.2, x).clone()
    assert torch.equal(a, b)


def test_stream_ordering_with_torch_stream(ssx, oracle):
    """Work queued by torch on a side stream before the call is seen by it."""
    spec = W.small(order=4, nt=200)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = ssx.Context.for_problem(spec, W.velocity(spec))
        h = dev(W.smooth_random_gather(spec.nt, spec.n_line, 15))
        h2 = h * 2.0               # queued on s
        d = ctx.forward(h2)        # must run after the multiply
        d2 = d * 0.5
    s.synchronize()
    P = oracle.Problem(spec, W.velocity(spec))
    assert rel(d2, P.S(h.cpu().numpy())) <= TOL


# ------------------------------------------------------------ sweep forms --
@pytest.mark.parametrize("spec_name", ["small", "c2"])
def test_persistent_and_per_step_sweeps_agree(ssx, spec_name):
    """The cooperative whole-sweep launch and the per-step graph replay run the
    same per-tile arithmetic: identical results."""
    spec = frac_spec(8) if spec_name == "small" else W.c2()
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    x = dev(W.smooth_random_gather(spec.nt, spec.n_line, 16))
    y = dev(W.smooth_random_gather(spec.nt, spec.n_rec, 17))
    out = {}
    for mode in (ssx.SWEEP_PERSISTENT, ssx.SWEEP_STEP):
        ctx.set_sweep_mode(mode)
        out[mode] = (ctx.forward(x).clone(), ctx.adjoint(y).clone(),
                     ctx.weight_apply(ssx.W_M_INV, x).clone())
    for a, b in zip(out[ssx.SWEEP_PERSISTENT], out[ssx.SWEEP_STEP]):
        assert torch.equal(a, b)


def test_persistent_wait_timeout_is_reported_and_context_survives(ssx, oracle):
    """A neighbour wait that nothing satisfies runs out (0.2 s), the call
    returns SSX_ERR_CUDA, and the next call on the same context is correct."""
    spec = W.small(order=4, nt=200)
    ctx, P = make(ssx, oracle, spec)
    ctx.set_sweep_mode(ssx.SWEEP_PERSISTENT)
    h = W.smooth_random_gather(spec.nt, spec.n_line, 18)
    ctx.set_sweep_mode(ssx.SWEEP_TEST_STALL)
    with pytest.raises(ssx.SSXError) as e:
        ctx.forward(dev(h))
    assert e.value.code == 2 and "timed out" in e.value.msg
    assert rel(ctx.forward(dev(h)), P.S(h)) <= TOL


@pytest.mark.parametrize("cfg_offset", [0, 2])
def test_march_kernel_parity_and_copy_wait_timeout(ssx, oracle, cfg_offset):
    """The marching phase kernel on its own: S, S^T, W~_d and one preconditioned
    solve against the oracle on a grid of several tall tiles with ragged edges;
    then a tile whose copies are withheld (test hook) makes its CTA's bounded
    wait run out (0.2 s), the call returns SSX_ERR_CUDA, and the next call on
    the same context gives the same bits as before."""
    spec = frac_spec(8, nt=160)
    ctx, P = make(ssx, oracle, spec)
    ctx.set_tile_config(2 * ssx.N_TILE_CONFIGS + cfg_offset)
    h = W.smooth_random_gather(spec.nt, spec.n_line, 23)
    d = W.smooth_random_gather(spec.nt, spec.n_rec, 24)
    assert rel(ctx.forward(dev(h)), P.S(h)) <= TOL
    assert rel(ctx.adjoint(dev(d)), P.ST(d)) <= TOL
    assert rel(ctx.weight_apply(ssx.W_D, dev(d)), P.Wd(d)) <= TOL
    _check_solve(ctx, P, spec, d, "pcg", 4, 0.0)
    ref = ctx.forward(dev(h)).clone()
    ctx.set_sweep_mode(ssx.SWEEP_TEST_STALL)
    with pytest.raises(ssx.SSXError) as e:
        ctx.forward(dev(h))
    assert e.value.code == 2 and "timed out" in e.value.msg
    assert torch.equal(ctx.forward(dev(h)), ref)
    ctx.set_tile_config(-1)


@pytest.mark.parametrize("m,nt", [(0, 160), (1, 161), (2, 160)])
def test_two_step_kernel_parity(ssx, oracle, m, nt):
    """The two-step (temporally blocked) phase kernel forced on every phase of
    one sweep: S, S^T, W~_d and a preconditioned solve (whose M^-1 slab
    phases are single sweeps) against the oracle, with both lines between grid
    rows; an odd step count ends with a launch of one step."""
    spec = frac_spec(8, nt=nt)
    ctx, P = make(ssx, oracle, spec)
    ctx.set_tile_config(2 * ssx.N_TILE_CONFIGS + ssx.N_MARCH_CONFIGS + m)
    h = W.smooth_random_gather(spec.nt, spec.n_line, 25)
    d = W.smooth_random_gather(spec.nt, spec.n_rec, 26)
    assert rel(ctx.forward(dev(h)), P.S(h)) <= TOL
    assert rel(ctx.adjoint(dev(d)), P.ST(d)) <= TOL
    assert rel(ctx.weight_apply(ssx.W_D, dev(d)), P.Wd(d)) <= TOL
    _check_solve(ctx, P, spec, d, "pcg", 4, 0.0)
    ctx.set_tile_config(-1)


def test_tma_copy_wait_timeout_is_reported_and_context_survives(ssx):
    """The TMA-staged phase kernel: a tile whose copies are withheld (test
    hook) makes its CTA's bounded mbarrier wait run out (0.2 s); the call
    returns SSX_ERR_CUDA, no copy is left in flight, and the next call on the
    same context gives the same bits as before."""
    spec = frac_spec(8, nt=80)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    ctx.set_tile_config(ssx.N_TILE_CONFIGS)   # TMA-staged kernel, shape 0
    x = dev(W.smooth_random_gather(spec.nt, spec.n_line, 21))
    ref = ctx.forward(x).clone()
    ctx.set_sweep_mode(ssx.SWEEP_TEST_STALL)
    with pytest.raises(ssx.SSXError) as e:
        ctx.forward(x)
    assert e.value.code == 2 and "timed out" in e.value.msg
    assert torch.equal(ctx.forward(x), ref)
    ctx.set_tile_config(-1)


@pytest.mark.parametrize("order,nt", [(4, 120), (8, 120), (8, 121)])
def test_every_tile_configuration_gives_identical_results(ssx, order, nt):
    """All tile shapes / CTA sizes, both launch forms, the TMA-staged phase
    kernel (ids N..2N-1), the marching kernel (ids 2N..; order 8) and the
    two-step kernel (two time steps per launch; order 8; an odd step count
    ends with a launch of one step) run the same per-point arithmetic:
    bitwise-identical sweeps (ragged tiles on both grid edges, lines between
    rows)."""
    spec = frac_spec(order, nt=nt)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    x = dev(W.smooth_random_gather(spec.nt, spec.n_line, 19))
    y = dev(W.smooth_random_gather(spec.nt, spec.n_rec, 20))
    ref = None
    for mode in (ssx.SWEEP_STEP, ssx.SWEEP_PERSISTENT):
        ctx.set_sweep_mode(mode)
        N = ssx.N_TILE_CONFIGS
        n_all = 2 * N + ssx.N_MARCH_CONFIGS + ssx.N_TWO_CONFIGS
        for cfg in range(n_all if mode == ssx.SWEEP_STEP else N):
            ctx.set_tile_config(cfg)
            got = (ctx.forward(x).clone(), ctx.adjoint(y).clone(),
                   ctx.weight_apply(ssx.W_D, y).clone())
            if ref is None:
                ref = got
            for a, b in zip(got, ref):
                assert torch.equal(a, b), (mode, cfg)
    ctx.set_tile_config(-1)
    ctx.set_sweep_mode(ssx.SWEEP_AUTO)
    st = ctx.stats()
    assert len(st["tile_cfg"]) == 6


def test_phase_breakdown_accounts_for_the_timed_sweeps(ssx):
    """ssx_get_phase_stats: a timed PCG solve has rows for its four phases,
    each with its launches (time steps) and device time; together with the
    operator sweeps outside phases they make up the timed sweeps."""
    spec = W.small(order=8, nt=200)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    d = dev(W.smooth_random_gather(spec.nt, spec.n_rec, 31))
    ctx.solve(d, 0.1, 2, 0.0)
    ctx.reset_stats()
    assert ctx.phase_stats() == []
    ctx.set_timing(True)
    ctx.solve(d, 0.1, 2, 0.0)
    ctx.set_timing(False)
    rows = ctx.phase_stats()
    st = ctx.stats()
    names = {r["phase"] for r in rows}
    assert {"e1", "e2", "e3", "e4"} <= names, rows
    for r in rows:
        assert r["ms"] > 0 and r["steps"] >= spec.nt and r["sweeps"] >= 1 and r["tiles"] >= 1
        assert 0 <= r["tile_config"] < 2 * ssx.N_TILE_CONFIGS + ssx.N_MARCH_CONFIGS + ssx.N_TWO_CONFIGS
        assert r["chain"] in (0, 8, 16, 32)
    assert sum(r["ms"] for r in rows) <= st["sweep_ms"] * (1 + 1e-6)
    assert sum(r["steps"] for r in rows) <= st["timed_steps"]


def test_model_change_refreshes_captured_sweeps(ssx, oracle):
    """Captured sweeps hold the grid coefficients: a new model (and density)
    on the same context must give the new operator."""
    spec = W.small(order=4, nt=150)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    h = W.smooth_random_gather(spec.nt, spec.n_line, 21)
    ctx.forward(dev(h))
    spec2 = dataclasses.replace(spec, rho=2.5, model="homogeneous", v0=1.8)
    ctx.set_velocity_model(torch.as_tensor(W.velocity(spec2), dtype=torch.float32, device="cuda"),
                           spec2.rho)
    P2 = oracle.Problem(spec2, W.velocity(spec2))
    assert rel(ctx.forward(dev(h)), P2.S(h)) <= TOL
    assert rel(ctx.normal_apply(ssx.MODE_PCG, 0.1, dev(h)), P2.N(h, 0.1)) <= TOL


# -------------------------------------------------- diagnostics (NEXT-4) --
@pytest.mark.parametrize("transpose", [False, True])
def test_lambda_tilde_parity(ssx, oracle, transpose):
    spec = frac_spec(8)
    ctx, P = make(ssx, oracle, spec)
    x = W.smooth_random_gather(spec.nt, spec.n_line, 22)
    assert rel(ctx.lambda_apply(dev(x), transpose), P.lambda_tilde(x, transpose)) <= TOL


def test_time_reversal_inverse_parity(ssx, oracle):
    spec = W.small(order=8, nt=400)
    ctx, P = make(ssx, oracle, spec)
    d = P.point_source_data(W.ricker(spec), spec.x_d, spec.z_d)
    assert rel(ctx.time_reversal_inverse(dev(d)), P.time_reversal_inverse(d)) <= TOL


# ------------------------------------------------------ batching (NEXT-1) --
def _shot(base, k, **kw):
    """shot k of a small survey: its own source position, line window, alpha"""
    xs = base.h * (20 + 30 * k)
    return dataclasses.replace(base, x_s=xs, x_d=xs, ix_line0=5 + 10 * k, n_line=90,
                               alpha=(1e-3, 1e-2, 1e-1)[k % 3], **kw)


@pytest.mark.parametrize("mode", ["pcg", "cg"])
def test_batched_solves_equal_solo_solves(ssx, oracle, mode):
    """Three shots in shared launches give bit-for-bit the solo results, and
    one of them matches the oracle."""
    base = W.small(order=8, nt=300)
    specs = [_shot(base, k) for k in range(3)]
    m = ssx.MODE_PCG if mode == "pcg" else ssx.MODE_CG
    ctxs, ds, Ps = [], [], []
    for sp in specs:
        c, P = make(ssx, oracle, sp)
        ctxs.append(c)
        Ps.append(P)
        ds.append(dev(P.point_source_data(W.ricker(sp), sp.x_d, sp.z_d)))
    hb, hists, iters, status = ssx.solve_batch(ctxs, ds, [sp.alpha for sp in specs], 6, 0.0, m)
    for c, d, sp, h, hh, it in zip(ctxs, ds, specs, hb, hists, iters):
        h1, hh1, it1, st1 = c.solve(d, sp.alpha, 6, 0.0, m)
        assert it == it1 == 6
        assert torch.equal(h, h1)
        np.testing.assert_array_equal(hh, hh1)
    h_or, hist_or = oracle_pcg(Ps[1], ds[1].cpu().numpy(), specs[1].alpha, 6, 0.0, mode)
    assert rel(hb[1], h_or) <= TOL
    np.testing.assert_array_less(np.abs(hists[1] - hist_or) / hist_or, HIST_TOL)


def test_batched_uneven_grids_and_stopping(ssx, oracle):
    """Shots of different grid sizes, lengths and orders of stopping share the
    launches; each keeps its solo result (one stops early on its rtol)."""
    a = W.small(order=4, nt=260)
    b = dataclasses.replace(W.small(order=4, nt=180), nx=97, nz=61, n_line=90, n_rec=97,
                            z_s=0.45, x_s=0.5, x_d=0.5, ix_line0=2)
    ctxs, ds = [], []
    for sp in (a, b):
        c, P = make(ssx, oracle, sp)
        ctxs.append(c)
        ds.append(dev(P.point_source_data(W.ricker(sp), sp.x_d, sp.z_d)))
    rtol = 0.05
    hb, hists, iters, status = ssx.solve_batch(ctxs, ds, [a.alpha, b.alpha], 10, rtol)
    for c, d, sp, h, hh, it, stt in zip(ctxs, ds, (a, b), hb, hists, iters, status):
        h1, hh1, it1, st1 = c.solve(d, sp.alpha, 10, rtol)
        assert (it, stt) == (it1, st1)
        assert torch.equal(h, h1)
        np.testing.assert_array_equal(hh, hh1)
