"""Failure paths of Algorithm 1 on the GPU, made on the host (no GPU fault):
non-finite data, and a breakdown or a non-finite curvature injected through
the library's test hook on the device scalar path. Each returns its status
code, leaves the context usable, and leaves h at the last good iterate."""
import numpy as np
import pytest
import torch

from paper_2203_16573_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2203_16573_gb300 import build, ssx
    build.build()
    spec = W.small(order=8, nt=300)
    ctx = ssx.Context.for_problem(spec, W.velocity(spec))
    w = torch.as_tensor(W.ricker(spec), device="cuda")
    d = ctx.point_source_data(spec.x_d, spec.z_d, w).clone()
    return ssx, spec, ctx, d


def test_nan_in_the_data_gives_nonfinite_and_a_zero_source(setup):
    ssx, spec, ctx, d = setup
    bad = d.clone()
    bad[spec.nt // 2, spec.n_rec // 3] = float("nan")
    h, hist, iters, status = ctx.solve(bad, spec.alpha, 5, 0.0, allow_breakdown=True)
    assert status == "SSX_ERR_NONFINITE" and iters == 0
    assert not np.isfinite(hist[0])
    assert float(h.abs().max()) == 0.0            # h_0 = 0 is the last good iterate
    h2, _, it2, st2 = ctx.solve(d, spec.alpha, 2, 0.0)   # the context is still usable
    assert st2 == "SSX_ERR_NOT_CONVERGED" and it2 == 2 and torch.isfinite(h2).all()


@pytest.mark.parametrize("hook,code", [("BREAKDOWN", "SSX_ERR_BREAKDOWN"),
                                       ("NONFINITE", "SSX_ERR_NONFINITE")])
@pytest.mark.parametrize("mode", ["pcg", "cg"])
def test_injected_curvature_failure_keeps_the_last_good_iterate(setup, hook, code, mode):
    ssx, spec, ctx, d = setup
    m = ssx.MODE_PCG if mode == "pcg" else ssx.MODE_CG
    k = 2
    ref, ref_hist, ref_it, _ = ctx.solve(d, spec.alpha, k, 0.0, m)   # h_k of an undisturbed solve
    ref = ref.clone()
    ctx.set_test_hook(getattr(ssx, "HOOK_" + hook), k)
    h, hist, iters, status = ctx.solve(d, spec.alpha, 6, 0.0, m, allow_breakdown=True)
    assert status == code and iters == k and ref_it == k
    assert torch.equal(h, ref)
    np.testing.assert_array_equal(hist, ref_hist)
    msg = ctx._lib.ssx_last_error(ctx._c).decode()
    assert ("breakdown at k=2" in msg) if hook == "BREAKDOWN" else ("non-finite" in msg), msg
    with pytest.raises(ssx.SSXError):           # without allow_breakdown the binding raises
        ctx.set_test_hook(getattr(ssx, "HOOK_" + hook), 0)
        ctx.solve(d, spec.alpha, 3, 0.0, m)
    # the hook fired once: the next solve runs undisturbed
    h3, _, it3, st3 = ctx.solve(d, spec.alpha, 4, 0.0, m)
    assert it3 == 4 and st3 == "SSX_ERR_NOT_CONVERGED"


def test_hook_arguments_are_checked(setup):
    ssx, spec, ctx, d = setup
    for hook, k in ((7, 0), (ssx.HOOK_BREAKDOWN, -1)):
        with pytest.raises(ssx.SSXError) as e:
            ctx.set_test_hook(hook, k)
        assert e.value.code == 1
    ctx.set_test_hook(ssx.HOOK_NONE, -1)
