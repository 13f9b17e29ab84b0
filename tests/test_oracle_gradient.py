"""Pins of the oracle's reduced-objective gradient (variable projection:
eqn:esi, eqn:esis) against what the mathematics fixes, independent of the
oracle's own adjoint code:

* central finite differences of Phi(v) = ||S[v] h - d||^2 + alpha ||A h||^2
  along random directions, with the sponge strength held fixed, agree with
  <grad, dv> to second order in the step (any dropped term, wrong time index,
  missing sponge factor or wrong fold onto the model fails this);
* a direction confined to the model's edge rows and columns (whose values
  the sponge copies) checks the fold;
* the gradient vanishes when the data are fitted exactly (d = S h).
"""
import numpy as np
import pytest

from paper_2203_16573_gb300 import workloads as W


def _setup(order, seed=5):
    spec = W.tiny(order)
    rng = np.random.default_rng(seed)
    v = W.velocity(spec) * (1.0 + 0.05 * rng.standard_normal((spec.nz, spec.nx)))
    v_max = float(v.max()) * 1.05         # fixed sponge strength for the differences
    h = W.random_gather(spec.nt, spec.n_line, 3)
    d = 0.01 * W.random_gather(spec.nt, spec.n_rec, 4)
    return spec, v, v_max, h, d, rng


def _phi(oracle, spec, v, v_max, h, d, alpha):
    return oracle.objective(oracle.Problem(spec, v, v_max=v_max), h, d, alpha)


@pytest.mark.parametrize("order", [4, 8])
def test_gradient_matches_central_differences(oracle, order):
    spec, v, v_max, h, d, rng = _setup(order)
    alpha = 0.3
    g = oracle.velocity_gradient(oracle.Problem(spec, v, v_max=v_max), h, d)
    assert g.shape == (spec.nz, spec.nx)
    for _ in range(3):
        dv = rng.standard_normal(v.shape)
        an = float(np.sum(g * dv))
        errs = []
        for eps in (1e-2, 1e-3):
            fd = (_phi(oracle, spec, v + eps * dv, v_max, h, d, alpha)
                  - _phi(oracle, spec, v - eps * dv, v_max, h, d, alpha)) / (2 * eps)
            errs.append(abs(fd - an) / abs(an))
        assert errs[1] < 1e-4, errs
        assert errs[1] < errs[0] / 30, errs   # second order in eps (truncation-dominated)


def test_fold_onto_edge_model_points(oracle):
    """The sponge repeats the model's edge rows and columns: perturbing only
    those points must still match finite differences."""
    spec, v, v_max, h, d, rng = _setup(4, seed=7)
    g = oracle.velocity_gradient(oracle.Problem(spec, v, v_max=v_max), h, d)
    dv = np.zeros_like(v)
    dv[0, :] = rng.standard_normal(spec.nx)
    dv[-1, :] = rng.standard_normal(spec.nx)
    dv[:, 0] += rng.standard_normal(spec.nz)
    dv[:, -1] += rng.standard_normal(spec.nz)
    eps = 1e-3
    fd = (_phi(oracle, spec, v + eps * dv, v_max, h, d, 0.0)
          - _phi(oracle, spec, v - eps * dv, v_max, h, d, 0.0)) / (2 * eps)
    an = float(np.sum(g * dv))
    # without the sponge copies the edge gradient would be off by O(1)
    assert abs(fd - an) / abs(an) < 1e-4


def test_gradient_vanishes_at_exact_fit(oracle):
    spec, v, v_max, h, _, _ = _setup(4)
    P = oracle.Problem(spec, v, v_max=v_max)
    d = P.S(h)
    g = oracle.velocity_gradient(P, h, d)
    assert np.max(np.abs(g)) == 0.0
    assert oracle.objective(P, h, d, 0.0) == 0.0
