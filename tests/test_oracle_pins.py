"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one part of the oracle to the paper's statements, a closed
form, an invariant, a library routine or a textbook table, so that a dropped
term, a wrong sign, a shifted index or a transposed operand in the oracle
fails at least one of them. All run on the CPU (no GPU marker).
"""
import dataclasses
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, linalg

from paper_2203_16573_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_weights():
    out = {}
    for line in open(os.path.join(GOLDEN, "staggered_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        out[int(parts[0])] = [float(Fraction(t)) for t in parts[1:]]
    return out


def _golden_constants():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


# ---------------------------------------------------------------- stencil --
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_staggered_weights_match_textbook_table(oracle, order):
    """Weights equal the textbook staggered Taylor values (golden table)."""
    np.testing.assert_allclose(oracle.staggered_weights(order), _golden_weights()[order],
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_staggered_difference_exact_on_polynomials(oracle, order):
    """sum_m c_m (u(x+(m-1/2)h) - u(x-(m-1/2)h))/h = u'(x) exactly for
    polynomials of degree <= 2k, and not for degree 2k+1."""
    c = oracle.staggered_weights(order)
    k = order // 2
    h, x = 0.37, 0.81
    for deg in range(0, 2 * k + 2):
        u = lambda y: y ** deg
        du = deg * x ** (deg - 1) if deg > 0 else 0.0
        approx = sum(cm * (u(x + (m + 0.5) * h) - u(x - (m + 0.5) * h)) for m, cm in enumerate(c)) / h
        if deg <= 2 * k:
            assert abs(approx - du) <= 1e-11 * max(1.0, abs(du))
        else:
            assert abs(approx - du) > 1e-8


# ------------------------------------------------------------ adjointness --
def _grid_with_lines(oracle, order, frac=True, nsp=6):
    rng = np.random.default_rng(7)
    vel = 1.5 + 0.5 * rng.random((23, 29))
    g = oracle.Grid(vel, 0.01, 1.1e-3, order, nsp, 1.3)
    src = g.line(0.137 if frac else 0.13, 3, 21)
    rec = g.line(0.041 if frac else 0.04, 1, 25)
    return g, src, rec


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("frac", [True, False])
def test_dot_product_2x2_modelling_operator(oracle, order, frac):
    """<S(h,f), (yp,yv)> = <(h,f), S^T(yp,yv)> to 1e-12 (section "Synthetic
    models and simulation": computed adjoints pass the inner-product test
    "with errors well under machine precision"; eqn:sadj1)."""
    g, src, rec = _grid_with_lines(oracle, order, frac)
    nt = 57
    rng = np.random.default_rng(11)
    h, f = rng.standard_normal((2, nt, src.n))
    yp, yv = rng.standard_normal((2, nt, rec.n))
    tp, tv = oracle.simulate(g, nt, src, rec, h=h, f=f, want_p=True, want_v=True)
    hb, fb = oracle.simulate_adj(g, nt, src, rec, yp=yp, yv=yv, want_h=True, want_f=True)
    lhs = np.sum(tp * yp) + np.sum(tv * yv)
    rhs = np.sum(h * hb) + np.sum(f * fb)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300)
    # each block separately as well
    for a, b in [(np.sum(oracle.simulate(g, nt, src, rec, h=h)[0] * yp),
                  np.sum(h * oracle.simulate_adj(g, nt, src, rec, yp=yp)[0])),
                 (np.sum(oracle.simulate(g, nt, src, rec, f=f, want_p=False, want_v=True)[1] * yv),
                  np.sum(f * oracle.simulate_adj(g, nt, src, rec, yv=yv, want_h=False, want_f=True)[1]))]:
        assert abs(a - b) <= 1e-12 * abs(a)


def test_point_source_dot_product(oracle):
    g, _, rec = _grid_with_lines(oracle, 8)
    pt = g.line(0.11, 14, 1, scale=1.0 / 0.01)
    nt = 40
    rng = np.random.default_rng(3)
    w = rng.standard_normal((nt, 1))
    y = rng.standard_normal((nt, rec.n))
    a = np.sum(oracle.simulate(g, nt, pt, rec, h=w)[0] * y)
    b = np.sum(w * oracle.simulate_adj(g, nt, pt, rec, yp=y)[0])
    assert abs(a - b) <= 1e-12 * abs(a)



def test_lines_between_rows_interpolate_linearly_in_depth(oracle):
    """Trace sampling and source injection interpolate linearly in z: p lives
    on rows at k h and v_z on rows at (k + 1/2) h. So a pressure line at depth
    (k + 0.3) h is 0.7 x the line on row k plus 0.3 x the line on row k + 1,
    and a v_z line at the p-row depth k h is the mean of the v_z lines at
    (k - 1/2) h and (k + 1/2) h. Swapped weights, or a v_z line placed on the
    p rows, fails this. The dot tests cannot see either mistake, since each
    keeps injection and sampling transposes of one another."""
    g, _, _ = _grid_with_lines(oracle, 4, nsp=6)
    h, nt, k = 0.01, 40, 9
    rng = np.random.default_rng(11)
    hs = rng.standard_normal((nt, 21))
    fs = rng.standard_normal((nt, 21))

    def traces(z_src, z_rec, **kw):
        return oracle.simulate(g, nt, g.line(z_src, 3, 21), g.line(z_rec, 1, 25), want_v=True, **kw)

    def close(a, b):
        return np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    # pressure injection between rows
    a = traces((k + 0.3) * h, 0.05, h=hs)[0]
    b = 0.7 * traces(k * h, 0.05, h=hs)[0] + 0.3 * traces((k + 1) * h, 0.05, h=hs)[0]
    assert close(a, b)
    # pressure and v_z sampling between rows
    pa, va = traces(k * h, 0.043, h=hs)
    p0, v0 = traces(k * h, 0.04, h=hs)
    p1, v1 = traces(k * h, 0.05, h=hs)
    assert close(pa, 0.7 * p0 + 0.3 * p1)
    vlo = traces(k * h, 0.035, h=hs)[1]            # v_z row at 0.035 = (3 + 1/2) h
    vhi = traces(k * h, 0.045, h=hs)[1]            # v_z row at 0.045
    assert close(v0, 0.5 * vlo + 0.5 * vhi)
    # v_z (velocity) injection on a p-row depth: mean of the two v_z rows
    fa = traces(k * h, 0.05, f=fs)[0]
    flo = traces((k - 0.5) * h, 0.05, f=fs)[0]
    fhi = traces((k + 0.5) * h, 0.05, f=fs)[0]
    assert close(fa, 0.5 * flo + 0.5 * fhi)
    assert np.linalg.norm(fa) > 0 and np.linalg.norm(pa) > 0

# ------------------------------------------------------------------ energy --
@pytest.mark.parametrize("order", [4, 8])
def test_leapfrog_energy_is_conserved_without_sponge(oracle, order):
    """With no sponge and no sources (closed box, zero extension) the discrete
    energy 1/2 [sum p^n^2/kappa + rho sum v^{n-1/2} . v^{n+1/2}] of the
    staggered leapfrog is invariant (discrete form of eqn:defae0's balance)."""
    rng = np.random.default_rng(5)
    vel = 1.5 + rng.random((30, 34))
    g = oracle.Grid(vel, 0.01, 1.5e-3, order, 0, 1.7)
    p = np.ascontiguousarray(W.smooth_random_gather(g.NZ, g.NX, 9, 2, 2))
    vx = np.zeros_like(p)
    vz = np.zeros_like(p)
    E = []
    for n in range(400):
        p_old, vx_old, vz_old = p.copy(), vx.copy(), vz.copy()
        oracle.step(g, p, vx, vz)
        E.append(0.5 * (np.sum(p_old ** 2 / g.kappa)
                        + g.rho * (np.sum(vx_old * vx) + np.sum(vz_old * vz))))
    E = np.array(E)
    assert np.abs(E - E[0]).max() <= 1e-12 * E[0]
    # and the sponge removes energy (sanity that the pin is not vacuous)
    g2 = oracle.Grid(vel, 0.01, 1.5e-3, order, 6, 1.7)
    p2 = np.ascontiguousarray(W.smooth_random_gather(g2.NZ, g2.NX, 9, 2, 2))
    z2, z3 = np.zeros_like(p2), np.zeros_like(p2)
    e0 = np.sum(p2 ** 2 / g2.kappa)
    for n in range(400):
        oracle.step(g2, p2, z2, z3)
    assert np.sum(p2 ** 2 / g2.kappa) < 0.5 * e0


# ------------------------------------------------------- Green's function --
def _ricker_deriv(t, f, t0):
    tau = t - t0
    a = (math.pi * f * tau) ** 2
    return (2 * a - 3) * math.exp(-a) * 2 * math.pi ** 2 * f ** 2 * tau


def _greens_pressure(r, t, c, kappa, f, t0):
    """p(r,t) for (1/kappa) p_t + div v = s(t) delta(x), rho v_t + grad p = 0:
    p_tt - c^2 Lap p = kappa s'(t) delta(x), 2D Green's function
    H(ct - r) / (2 pi c sqrt(c^2 t^2 - r^2)); with t - tau = (r/c) cosh u the
    time convolution is kappa/(2 pi c^2) int_0^{acosh(ct/r)} s'(t - (r/c) cosh u) du."""
    if c * t <= r:
        return 0.0
    U = math.acosh(c * t / r)
    val, _ = integrate.quad(lambda u: _ricker_deriv(t - (r / c) * math.cosh(u), f, t0),
                            0.0, U, limit=400, epsabs=1e-13)
    return kappa / (2 * math.pi * c * c) * val


@pytest.mark.parametrize("order", [4, 8])
def test_point_source_converges_to_2d_greens_function(oracle, order):
    """Pressure trace of a point pressure source (scale 1/h^2, the discrete
    delta(x) delta(z)) converges to the closed-form 2D solution at second
    order in (h, dt), CFL fixed."""
    c, f, L, r, T = 1.5, 8.0, 1.6, 0.3, 0.55
    t0 = 1.5 / f
    errs = []
    for h in (0.02, 0.01, 0.005):
        dt = 0.2 * h
        n, nt = int(round(L / h)) + 1, int(round(T / dt))
        g = oracle.Grid(np.full((n, n), c), h, dt, order, 20, 1.0)
        ic = n // 2
        src = g.line(ic * h, ic, 1, scale=1.0 / h)
        rec = g.line(ic * h, ic + int(round(r / h)), 1)
        tt = (np.arange(nt) + 0.5) * dt - t0
        w = (1 - 2 * (math.pi * f * tt) ** 2) * np.exp(-(math.pi * f * tt) ** 2)
        tr = oracle.simulate(g, nt, src, rec, h=w.reshape(-1, 1))[0][:, 0]
        m = int(round(0.004 / dt))
        idx = np.arange(m - 1, nt, m)
        ex = np.array([_greens_pressure(r, (k + 1) * dt, c, c * c, f, t0) for k in idx])
        errs.append(np.abs(tr[idx] - ex).max() / np.abs(ex).max())
    assert errs[0] / errs[1] > 2.2 and errs[1] / errs[2] > 2.2, errs
    assert errs[2] < 5e-3, errs


# ------------------------------------------------- thin-slab weights -------
@pytest.fixture(scope="module")
def plane_problem(oracle):
    """Homogeneous medium, source line across the whole width: in the middle
    columns the fields are 1D plane waves, so the weights have closed forms."""
    s = dataclasses.replace(W.small(order=8, nt=500, model="homogeneous"), nx=301,
                            ix_line0=0, n_line=301, n_rec=301, rho=2.0)
    P = oracle.Problem(s, W.velocity(s))
    t = (np.arange(s.nt) + 0.5) * s.dt - 0.1
    a = (math.pi * 12.0 * t) ** 2
    x = np.tile(((1 - 2 * a) * np.exp(-a))[:, None], (1, s.n_line))
    return s, P, x, slice(120, 181)


def _ratio(y, x, mid):
    return np.sum(y[:, mid] * x[:, mid]) / np.sum(x[:, mid] ** 2)


def test_weights_match_plane_wave_impedance(plane_problem):
    """For a vertically travelling plane wave (impedance Z = rho c) a pressure
    prescribed on a plane needs the source 2 p / Z (eqn:deflam, jump of v_z),
    so sym Lambda ~ 2/Z and its inverse ~ Z/2: W~_m^{-1}, W~_d ~ 2/Z
    (eqn:winvcomp, eqn:wdef) and W~_m ~ Z/2 (eqn:laminv/wcomp, prefactor -1).
    Linear interpolation across half rows costs a few percent, hence the bands."""
    s, P, x, mid = plane_problem
    Z = s.rho * s.v0
    assert 0.85 * 2 / Z < _ratio(P.Wminv(x), x, mid) < 1.02 * 2 / Z
    assert 0.85 * 2 / Z < _ratio(P.Wd(x), x, mid) < 1.02 * 2 / Z
    assert 0.93 * Z / 2 < _ratio(P.Wm(x), x, mid) < 1.02 * Z / 2
    # W~_m is an approximate inverse of W~_m^{-1} (the paper's claim after wcomp)
    y = P.Wm(P.Wminv(x))
    assert np.linalg.norm(y[:, mid] - x[:, mid]) < 0.2 * np.linalg.norm(x[:, mid])


def test_time_reversal_approximate_inverse(oracle, plane_problem):
    """eqn:approxinv: 4 (V+)^T S+ ~ I on downgoing data (plane wave)."""
    s, _, _, mid = plane_problem
    s = dataclasses.replace(s, nt=1000)
    P = oracle.Problem(s, W.velocity(s))
    t = (np.arange(s.nt) + 0.5) * s.dt - 0.1
    a = (math.pi * 12.0 * t) ** 2
    x = np.tile(((1 - 2 * a) * np.exp(-a))[:, None], (1, s.n_line))
    d = P.S(x)                                              # S+ h
    _, fb = oracle.simulate_adj(P.g, s.nt, P.src, P.rec, yv=d, want_h=False, want_f=True)
    y = 4.0 * fb                                            # 4 (V+)^T S+ h
    assert 0.85 < _ratio(y, x, mid) < 1.05
    assert np.linalg.norm(y[:, mid] - x[:, mid]) < 0.2 * np.linalg.norm(x[:, mid])
    assert _golden_constants()["approxinv_factor"] == 0.25


def test_weight_quadratic_form_identity(oracle):
    """<f, W~_m^{-1} f> = -4 <S Pi_1^T f, (swap) S Pi_1^T f> = -8 <P p, P v_z>
    at the datum (eqn:winvcomp), the right side from a forward sweep only."""
    s = W.small(order=4, nt=200)
    P = oracle.Problem(s, W.velocity(s))
    f = W.smooth_random_gather(s.nt, s.n_line, 21)
    slab = P.slab_s
    g = slab.grid
    pl, dl = g.line(slab.z0, s.ix_line0, s.n_line), g.line(slab.zd, s.ix_line0, s.n_line)
    tp, tv = oracle.simulate(g, s.nt, pl, dl, f=f, want_p=True, want_v=True)
    lhs = np.sum(f * P.Wminv(f))
    rhs = _golden_constants()["winvcomp_prefactor"] * 2.0 * P.sgn * np.sum(tp * tv)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert lhs > 0
    # datum distance is the paper's 100 m
    assert abs(s.dz_datum - _golden_constants()["thin_slab_dz_km"]) < 1e-15


def test_symmetrised_lambda_tilde_is_Wminv(oracle):
    """eqn:winvcomp is the mean of eqn:lamtilde and eqn:lamtransp:
    (Lambda~ + Lambda~^T)/2 = W~_m^{-1} to rounding; Lambda~ and Lambda~^T are
    transposes of each other."""
    s = W.small(order=4, nt=150)
    P = oracle.Problem(s, W.velocity(s))
    a, b = W.random_gather(s.nt, s.n_line, 31), W.random_gather(s.nt, s.n_line, 32)
    sym = 0.5 * (P.lambda_tilde(a) + P.lambda_tilde(a, transpose=True))
    ref = P.Wminv(a)
    assert np.abs(sym - ref).max() <= 1e-12 * np.abs(ref).max()
    x, y = np.sum(b * P.lambda_tilde(a)), np.sum(a * P.lambda_tilde(b, transpose=True))
    assert abs(x - y) <= 1e-12 * abs(x)
    assert _golden_constants()["lamtilde_prefactor"] == -8


def test_lambda_tilde_maps_pressure_trace_to_source(oracle, plane_problem):
    """eqn:tracejump10 / eqn:lamnear: for a plane wave the pressure-to-source
    map is multiplication by 2/Z (asymptotically symmetric, so Lambda~ and
    Lambda~^T agree)."""
    s, P, x, mid = plane_problem
    Z = s.rho * s.v0
    for tr in (False, True):
        assert 0.85 * 2 / Z < _ratio(P.lambda_tilde(x, transpose=tr), x, mid) < 1.05 * 2 / Z


@pytest.mark.parametrize("which", ["Wminv", "Wm", "Wd"])
def test_weights_symmetric(oracle, which):
    """Symmetrised thin-slab weights are symmetric to rounding (eqn:winvcomp,
    wcomp: B^T J B with the exchange J symmetric)."""
    s = W.small(order=4, nt=150)
    P = oracle.Problem(s, W.velocity(s))
    n = s.n_rec if which == "Wd" else s.n_line
    a, b = W.random_gather(s.nt, n, 1), W.random_gather(s.nt, n, 2)
    op = getattr(P, which)
    x, y = np.sum(b * op(a)), np.sum(a * op(b))
    assert abs(x - y) <= 1e-12 * np.sqrt(np.sum(a * op(a)) ** 2 + np.sum(b * op(b)) ** 2)


def test_normal_operator_and_preconditioner_symmetric(oracle):
    s = W.small(order=4, nt=150)
    P = oracle.Problem(s, W.velocity(s))
    a, b = W.random_gather(s.nt, s.n_line, 3), W.random_gather(s.nt, s.n_line, 4)
    for mode in ("pcg", "cg"):
        for op in (lambda v: P.N(v, 0.3, mode), lambda v: P.Minv(v, 0.3, mode)):
            x, y = np.sum(b * op(a)), np.sum(a * op(b))
            assert abs(x - y) <= 1e-11 * (abs(x) + abs(y))


# ---------------------------------------------------- dense brute force ----
@pytest.fixture(scope="module")
def dense_tiny(oracle):
    s = W.tiny(order=4)
    P = oracle.Problem(s, W.velocity(s))
    nt = s.nt

    def dense(op, nin, nout):
        M = np.zeros((nout * nt, nin * nt))
        for j in range(nin * nt):
            e = np.zeros(nin * nt)
            e[j] = 1.0
            M[:, j] = op(e.reshape(nt, nin)).ravel()
        return M

    mats = dict(S=dense(P.S, s.n_line, s.n_rec), Wd=dense(P.Wd, s.n_rec, s.n_rec),
                Wm=dense(P.Wm, s.n_line, s.n_line), Wmi=dense(P.Wminv, s.n_line, s.n_line),
                A=np.diag(np.tile(P.dist, nt)))
    return s, P, mats


def test_dense_S_transpose_is_ST(dense_tiny):
    s, P, m = dense_tiny
    y = W.random_gather(s.nt, s.n_rec, 5)
    np.testing.assert_allclose(m["S"].T @ y.ravel(), P.ST(y).ravel(), rtol=0,
                               atol=1e-13 * np.abs(P.ST(y)).max())


def test_normal_operator_composition_dense(dense_tiny):
    """eqn:normpart with eqn:sadjwt: N = S^T W_d S + alpha A^T W_m A and
    S^* d = S^T W_d d, M^{-1} = D W~_m^{-1} D (eqn:defprecond), each compared
    with the product of separately extracted dense factors."""
    s, P, m = dense_tiny
    al = 0.7
    v = W.random_gather(s.nt, s.n_line, 6)
    d = W.random_gather(s.nt, s.n_rec, 7)
    N = m["S"].T @ m["Wd"] @ m["S"] + al * m["A"].T @ m["Wm"] @ m["A"]
    ref = N @ v.ravel()
    np.testing.assert_allclose(P.N(v, al).ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    ref = m["S"].T @ m["Wd"] @ d.ravel()
    np.testing.assert_allclose(P.rhs(d).ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    D = np.diag(1.0 / np.sqrt(1.0 + al * np.diag(m["A"]) ** 2))
    ref = D @ m["Wmi"] @ D @ v.ravel()
    np.testing.assert_allclose(P.Minv(v, al).ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    NE = m["S"].T @ m["S"] + al * m["A"].T @ m["A"]
    np.testing.assert_allclose(P.N(v, al, "cg").ravel(), NE @ v.ravel(), rtol=0,
                               atol=1e-12 * np.abs(NE @ v.ravel()).max())


class _DenseProblem:
    """Algorithm 1's inputs as dense SPD matrices (to pin the recurrences
    independently of the wave operators)."""

    def __init__(self, N, Minv, b, nt, n):
        self.Nm, self.Mm, self.b, self.nt = N, Minv, b, nt
        self.spec = type("S", (), {"n_line": n})

    def rhs(self, d, mode):
        return self.b.reshape(self.nt, -1).copy()

    def N(self, p, alpha, mode):
        return (self.Nm @ p.ravel()).reshape(p.shape)

    def Minv(self, r, alpha, mode):
        return (self.Mm @ r.ravel()).reshape(r.shape)


def test_pcg_matches_direct_solve_and_krylov_optimality(oracle):
    """Algorithm 1 on SPD (N, M): converges to scipy's direct solve, and the
    k-th iterate minimises the N-energy error over the Krylov space
    K_k(M^{-1} N, M^{-1} r_0) (the defining property of PCG)."""
    rng = np.random.default_rng(12)
    n, nt, nl = 60, 10, 6
    G = rng.standard_normal((n, n))
    N = G @ G.T + 0.5 * np.eye(n)
    H = rng.standard_normal((n, n))
    Mi = H @ H.T / n + np.eye(n)
    b = rng.standard_normal(n)
    prob = _DenseProblem(N, Mi, b, nt, nl)
    x_direct = linalg.solve(N, b, assume_a="pos")
    x, hist = oracle.pcg(prob, None, 0.0, 400, 1e-13)
    assert np.linalg.norm(x.ravel() - x_direct) <= 1e-9 * np.linalg.norm(x_direct)
    # Krylov optimality for a few k
    for k in (1, 3, 7):
        xk, _ = oracle.pcg(prob, None, 0.0, k, 0.0)
        K = [Mi @ b]
        for _ in range(k - 1):
            K.append(Mi @ (N @ K[-1]))
        Q, _ = np.linalg.qr(np.array(K).T)
        y = linalg.solve(Q.T @ N @ Q, Q.T @ b)
        np.testing.assert_allclose(xk.ravel(), Q @ y, rtol=0, atol=1e-9 * np.linalg.norm(Q @ y))


def test_plain_cg_matches_least_squares(dense_tiny, oracle):
    """Plain CG (W_m = W_d = I, M = I) reaches the minimiser of
    ||S h - d||^2 + alpha ||A h||^2 (eqn:esis) computed by lstsq on the
    stacked system [S; sqrt(alpha) A] h = [d; 0]."""
    s, P, m = dense_tiny
    al = 0.5
    # make the problem well posed: penalise every column (x_s off the line)
    P2 = oracle.Problem(dataclasses.replace(s, x_s=-0.05), W.velocity(s))
    A = np.diag(np.tile(P2.dist, s.nt))
    d = W.random_gather(s.nt, s.n_rec, 8)
    Sd = m["S"] * 1e3   # rescale so that both terms matter (same h for both sides)
    K = np.vstack([Sd, math.sqrt(al) * A])
    ref = np.linalg.lstsq(K, np.concatenate([d.ravel(), np.zeros(A.shape[0])]), rcond=None)[0]
    P2.S = lambda h: 1e3 * oracle.Problem.S(P2, h)
    P2.ST = lambda y: 1e3 * oracle.Problem.ST(P2, y)
    h, hist = oracle.pcg(P2, d, al, 800, 1e-12, mode="cg")
    assert np.linalg.norm(h.ravel() - ref) <= 1e-6 * np.linalg.norm(ref)


# --------------------------------------------------- known minimiser -------
def test_known_minimiser_objective_decreases(oracle):
    """Data from a point source on the source line in the same medium are fit
    exactly by h* = (wavelet/h) delta_{x = x_s}, which has A h* = 0: S h* = d,
    so h* minimises both objectives (eqn:esis, eqn:einv) and CG drives the
    N-energy error ||h_k - h*||_N^2 (the objective itself) down monotonically."""
    s = W.small(order=4, nt=350)
    P = oracle.Problem(s, W.velocity(s))
    w = W.ricker(s)
    d = P.point_source_data(w, s.x_d, s.z_d)
    hstar = np.zeros((s.nt, s.n_line))
    hstar[:, round(s.x_s / s.h) - s.ix_line0] = w / s.h
    assert np.linalg.norm(P.S(hstar) - d) <= 1e-13 * np.linalg.norm(d)
    assert np.abs(P.A(hstar)).max() == 0.0
    for mode in ("cg", "pcg"):
        J = []

        def cb(k, h, r):
            e = h - hstar
            J.append(np.sum(e * P.N(e, s.alpha, mode)))
        oracle.pcg(P, d, s.alpha, 5, 0.0, mode=mode, callback=cb)
        J0 = np.sum(hstar * P.N(hstar, s.alpha, mode))
        assert J[0] < J0 and all(b < a for a, b in zip(J, J[1:])), (mode, J0, J)


# ------------------------------------------------ mirror symmetry ----------
def _mirror_problem(oracle, order, nt=160):
    """The reduced lens case (133 x 71, x_s on the centre column, source line
    and receivers centred on it) with the model made exactly symmetric about
    x_s."""
    s = W.small(order=order, nt=nt)
    v = W.velocity(s)
    v = 0.5 * (v + v[:, ::-1])
    return s, oracle.Problem(s, v)


def _mirror_err(a, b):
    """relative error of b against the reflection of a about the centre column"""
    return float(np.linalg.norm(a[:, ::-1] - b) / np.linalg.norm(a))


@pytest.mark.parametrize("order", [4, 8])
def test_operators_commute_with_the_mirror_about_x_s(oracle, order):
    """Reflecting x about a p column maps the staggered grid onto itself
    (p and v_z stay, v_x changes sign), the sponge ramps onto themselves and
    |x - x_s| onto itself. With the model, the source line and the receivers
    symmetric about x_s, S, S^T, W~_d, W~_m and W~_m^{-1} therefore commute
    with reflecting the gathers, and S is linear. A sponge ramp shifted by
    half a cell at the v_x points, a one-sided x difference or a line placed
    one column off breaks the reflection."""
    s, P = _mirror_problem(oracle, order)
    h = W.random_gather(s.nt, s.n_line, 51)
    d = W.random_gather(s.nt, s.n_rec, 52)
    for op, x in ((P.S, h), (P.ST, d), (P.Wd, d), (P.Wm, h), (P.Wminv, h)):
        y, ym = op(x), op(x[:, ::-1].copy())
        assert np.linalg.norm(y) > 0
        assert _mirror_err(y, ym) <= 1e-13, op.__name__
    h2 = W.random_gather(s.nt, s.n_line, 53)
    lin = P.S(2.5 * h - 0.75 * h2)
    ref = 2.5 * P.S(h) - 0.75 * P.S(h2)
    assert np.linalg.norm(lin - ref) <= 1e-13 * np.linalg.norm(ref)


def test_pcg_solution_of_mirrored_data_is_the_mirrored_solution(oracle):
    """Every operator of Algorithm 1 commutes with the reflection, so the
    iterates for reflected data are the reflected iterates (up to the
    rounding of the inner products' summation order), for both modes."""
    s, P = _mirror_problem(oracle, 4, nt=120)
    d = W.smooth_random_gather(s.nt, s.n_rec, 54)
    for mode in ("pcg", "cg"):
        h, hist = oracle.pcg(P, d, s.alpha, 4, 0.0, mode=mode)
        hm, histm = oracle.pcg(P, d[:, ::-1].copy(), s.alpha, 4, 0.0, mode=mode)
        assert _mirror_err(h, hm) <= 1e-10, mode
        np.testing.assert_allclose(histm, hist, rtol=1e-10)

# ------------------------------------------------------------- sponge ------
def _sponge_trace(oracle, n, nsp, sigma_scale=None, nt=700):
    """Pressure trace 30 cells from a 10 Hz point source at the centre of an
    n x n homogeneous grid (1.5 km/s, h = 10 m) with an nsp-point sponge;
    sigma_scale multiplies the damping profiles (planted mistakes)."""
    c, h, f = 1.5, 0.01, 10.0
    dt = 0.3 * h / c
    g = oracle.Grid(np.full((n, n), c), h, dt, 4, nsp, 1.0)
    keep = []
    if sigma_scale is not None:
        for name in ("sx_i", "sx_h", "sz_i", "sz_h"):
            keep.append(getattr(g, name) * sigma_scale)
            setattr(g._c, name, oracle._ptr(keep[-1]))
    mid = n // 2
    src, rec = g.line(mid * h, mid, 1, scale=1 / h), g.line(mid * h, mid - 30, 1)
    t = (np.arange(nt) + 0.5) * dt - 1.5 / f
    w = (1 - 2 * (math.pi * f * t) ** 2) * np.exp(-(math.pi * f * t) ** 2)
    return oracle.simulate(g, nt, src, rec, h=w.reshape(-1, 1))[0][:, 0]


def test_sponge_absorbs_outgoing_waves(oracle):
    """The quadratic sponge, sigma_max = 3 v_max ln(1000) / (2 L): on an
    81 x 81 grid with a 20-point sponge the trace matches, within 2 %, the
    trace on a 401 x 401 grid whose edges are too far away to echo back
    within the 1.4 s window. Rigid walls (no sponge) give an O(1) error, and
    narrower sponges reflect more. Damping 10 x too weak or 10 x too strong
    (the wave then reflects off the sponge's own steep front), or of the
    wrong sign, fails the bound."""
    free = _sponge_trace(oracle, 401, 0)

    def err(nsp, scale=None):
        return np.linalg.norm(_sponge_trace(oracle, 81, nsp, scale) - free) / np.linalg.norm(free)
    e = [err(nsp) for nsp in (0, 5, 10, 20)]
    assert e[0] > 1.0 and e[1] > e[2] > e[3]
    assert e[3] < 0.02
    for scale in (0.1, 10.0, -1.0):
        assert not err(20, scale) < 0.02, scale

# ------------------------------------------------- planted mistakes --------
def test_pins_catch_planted_mistakes(oracle, plane_problem):
    """A wrong sign in c_2, a dropped component exchange, the paper's
    printed -1/16 in place of -1, or the sponge ramp of the v_x points taken
    at the p points each break a pin above."""
    s, P, x, mid = plane_problem
    Z = s.rho * s.v0
    # (1) dropped exchange: S^T S instead of S^T J S -> negative form
    slab = P.slab_s
    g = slab.grid
    pl, dl = g.line(slab.z0, s.ix_line0, s.n_line), g.line(slab.zd, s.ix_line0, s.n_line)
    tp, tv = oracle.simulate(g, s.nt, pl, dl, f=x, want_p=True, want_v=True)
    _, fb = oracle.simulate_adj(g, s.nt, pl, dl, yp=tp, yv=tv, want_h=False, want_f=True)
    assert not (0.85 * 2 / Z < _ratio(-4 * P.sgn * fb, x, mid) < 1.02 * 2 / Z)
    # (2) -1/16 prefactor for W~_m
    assert not (0.93 * Z / 2 < _ratio(P.Wm(x) / 16.0, x, mid) < 1.02 * Z / 2)
    # (3) wrong sign of c_2 (the scheme stays skew, so energy is still
    #     conserved): the Green's-function error becomes large
    c, f, h = 1.5, 8.0, 0.01
    n = 161
    g3 = oracle.Grid(np.full((n, n), c), h, 0.2 * h, 4, 20, 1.0)
    g3._c.c[1] = -g3._c.c[1]
    src, rec = g3.line(80 * h, 80, 1, scale=1 / h), g3.line(80 * h, 110, 1)
    nt = 275
    tt = (np.arange(nt) + 0.5) * 0.2 * h - 1.5 / f
    w = (1 - 2 * (math.pi * f * tt) ** 2) * np.exp(-(math.pi * f * tt) ** 2)
    tr = oracle.simulate(g3, nt, src, rec, h=w.reshape(-1, 1))[0][:, 0]
    idx = np.arange(1, nt, 2)
    ex = np.array([_greens_pressure(0.3, (k + 1) * 0.2 * h, c, c * c, f, 1.5 / f) for k in idx])
    assert np.abs(tr[idx] - ex).max() / np.abs(ex).max() > 0.05
    # (4) sponge ramp of the v_x points (half-integer x) read at integer x:
    #     the reflection about x_s no longer maps the sponge onto itself
    s4, P4 = _mirror_problem(oracle, 4)
    bad = P4.g.sx_i.copy()
    P4.g._c.sx_h = oracle._ptr(bad)
    h4 = W.random_gather(s4.nt, s4.n_line, 55)
    assert _mirror_err(P4.S(h4), P4.S(h4[:, ::-1].copy())) > 1e-6
