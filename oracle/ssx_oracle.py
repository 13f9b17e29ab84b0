"""FP64 CPU oracle of the surface-source-extension subproblem solver.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline / reference legs may import this module; the product (the CUDA
library and its binding) never does, and this module never imports the
product. Inputs come from the seeded generators in
``paper_2203_16573_gb300.workloads`` only through the caller.

Each function restates one step of W. W. Symes, "Efficient Computation of
Extended Surface Sources" (arXiv 2203.16573), in the paper's notation:

* ``Grid`` / ``simulate`` / ``simulate_adj``: the 2x2 modelling operator
  S_{z_s,z_r}(h_s, f_s) = (P_r p, P_r v_z) of eqn:fwd for the acoustic system
  eqn:awepm, and its exact discrete transpose (eqn:sadj1, Appendix A). The
  time stepping is the C code in ``ssx_oracle.c``.
* ``Problem.S`` / ``Problem.ST``: S = Pi_0 S Pi_0^T (eqn:sdef) and S^T.
* ``Problem.Wminv``: W~_m^{-1} = -4 Pi_1 S^T (Pi_0^T Pi_1 + Pi_1^T Pi_0) S Pi_1^T
  on the thin slab z_s .. z_s + dz (eqn:winvcomp, eqn:lamnear).
* ``Problem.Wd``: the same construction at the receiver line (eqn:wdef,
  "with a similar definition for W~_d").
* ``Problem.Wm``: W~_m = -Pi_0 S^T (Pi_1^T Pi_0 + Pi_0^T Pi_1) S Pi_0^T
  (eqn:laminv, wcomp; prefactor read from eqn:snull2mod + eqn:approxinv).
* ``Problem.A``: (A f)(x, t) = |x - x_s| f(x, t) (eqn:penop).
* ``Problem.N``: N = S^T W~_d S + alpha A^T W~_m A (eqn:normpart, eqn:sadjwt).
* ``Problem.Minv``: M^{-1} = (I + alpha A^T A)^{-1/2} W~_m^{-1}
  (I + alpha A^T A)^{-1/2} (eqn:defprecond).
* ``pcg``: Algorithm 1 (standard preconditioned CG).

Readings where the paper is silent or inconsistent are listed in the
repository's design notes; the ones that change arithmetic are:
the penalty weight alpha multiplies ||A h||^2 (eqn:esis), so the paper's
alpha^2 of eqn:einv is this alpha; the right-hand side of eqn:norm1 uses
W_d (eqn:normpart); W~_m uses the thin slab like W~_m^{-1}; its prefactor is
-1 (not -1/16), which is what eqn:snull2mod and the second line of
eqn:approxinv give and what makes W~_m an approximate inverse of W~_m^{-1}
as the paper states; the prefactors' signs hold for the geometry of the
paper's examples (datum reached by travelling towards smaller z) and flip
for the mirrored geometry.
"""
from __future__ import annotations

import ctypes
import math
import os
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libssx_oracle.so")
_lib = None


class _CGrid(ctypes.Structure):
    _fields_ = [("NX", ctypes.c_int), ("NZ", ctypes.c_int), ("R", ctypes.c_int),
                ("c", ctypes.c_double * 8), ("dt", ctypes.c_double),
                ("h", ctypes.c_double), ("rho", ctypes.c_double),
                ("kappa", ctypes.c_void_p), ("sx_i", ctypes.c_void_p),
                ("sx_h", ctypes.c_void_p), ("sz_i", ctypes.c_void_p),
                ("sz_h", ctypes.c_void_p)]


class _CLine(ctypes.Structure):
    _fields_ = [("i0", ctypes.c_int), ("n", ctypes.c_int), ("kp", ctypes.c_int),
                ("wp0", ctypes.c_double), ("wp1", ctypes.c_double),
                ("kv", ctypes.c_int), ("wv0", ctypes.c_double),
                ("wv1", ctypes.c_double), ("scale", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ssx_oracle.c into a shared library next to it (gcc, OpenMP if
    available, no FMA contraction so x86 and Arm round alike)."""
    import subprocess
    src = os.path.join(_HERE, "ssx_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.og_step_fwd.argtypes = [P(_CGrid), vp, vp, vp, P(_CLine), vp, vp, P(_CLine), vp, vp]
        L.og_step_adj.argtypes = [P(_CGrid), vp, vp, vp, P(_CLine), vp, vp, vp, vp, vp]
        L.og_forward.argtypes = [P(_CGrid), ctypes.c_int, P(_CLine), vp, vp, P(_CLine), vp, vp]
        L.og_adjoint.argtypes = [P(_CGrid), ctypes.c_int, P(_CLine), vp, vp, P(_CLine), vp, vp]
        L.og_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().og_num_threads()


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


# --------------------------------------------------------------------------
# Discretisation ("Synthetic models and simulation"): staggered differences
# of order 2k; the weights are the Taylor conditions written out and solved
# exactly in rational arithmetic.
# --------------------------------------------------------------------------
def staggered_weights(order: int) -> list[float]:
    """c_1..c_k with sum_m c_m (2m-1)^(2l+1) = [l == 0], l = 0..k-1, so that
    sum_m c_m (u(x+(m-1/2)h) - u(x-(m-1/2)h)) / h = u'(x) + O(h^2k)."""
    k = order // 2
    A = [[Fraction(2 * m - 1) ** (2 * l + 1) for m in range(1, k + 1)] for l in range(k)]
    b = [Fraction(1 if l == 0 else 0) for l in range(k)]
    # Gauss-Jordan elimination in exact arithmetic
    for col in range(k):
        piv = next(r for r in range(col, k) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(k):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
                b[r] -= f * b[col]
    return [float(b[i] / A[i][i]) for i in range(k)]


def sponge_profile(n_phys: int, nsp: int, h: float, sigma_max: float):
    """sigma at integer and half-integer padded positions: a quadratic ramp
    sigma_max (d / (nsp h))^2 in the distance d beyond the physical edge."""
    N = n_phys + 2 * nsp

    def sig(pos):
        d = np.maximum(0.0, np.maximum(nsp - pos, pos - (nsp + n_phys - 1)))
        return sigma_max * (d / max(nsp, 1)) ** 2 if nsp > 0 else np.zeros_like(pos)

    pos_i = np.arange(N, dtype=np.float64)
    return np.ascontiguousarray(sig(pos_i)), np.ascontiguousarray(sig(pos_i + 0.5))


def sigma_max(v_max: float, nsp: int, h: float) -> float:
    """Peak damping rate: 3 v_max ln(1000) / (2 L), L = nsp h the sponge width."""
    if nsp == 0:
        return 0.0
    return 3.0 * v_max * math.log(1000.0) / (2.0 * nsp * h)


def row_weights(zeta: float):
    """Linear interpolation at fractional row coordinate zeta: (k, w0, w1)."""
    k = math.floor(zeta + 1e-6)
    w1 = zeta - k
    if w1 < 1e-6:
        w1 = 0.0
    return k, 1.0 - w1, w1


class Grid:
    """A padded simulation grid: physical model vel[nz][nx] (km/s) with
    n_sponge absorbing points outside it on every side; the model is extended
    into the sponge by edge replication. kappa = rho v^2."""

    def __init__(self, vel, h, dt, order, n_sponge, rho, v_max=None, z_origin=0.0):
        vel = np.asarray(vel, dtype=np.float64)
        self.nz, self.nx = vel.shape
        self.h, self.dt, self.order, self.nsp, self.rho = h, dt, order, n_sponge, rho
        self.z_origin = z_origin          # depth of physical row 0, km
        self.NZ, self.NX = self.nz + 2 * n_sponge, self.nx + 2 * n_sponge
        vpad = np.pad(vel, n_sponge, mode="edge")
        self.kappa = np.ascontiguousarray(rho * vpad ** 2)
        self.v_max = float(vel.max()) if v_max is None else float(v_max)
        smax = sigma_max(self.v_max, n_sponge, h)
        self.sx_i, self.sx_h = sponge_profile(self.nx, n_sponge, h, smax)
        self.sz_i, self.sz_h = sponge_profile(self.nz, n_sponge, h, smax)
        self.c = staggered_weights(order)
        cg = _CGrid()
        cg.NX, cg.NZ, cg.R = self.NX, self.NZ, order // 2
        for i, v in enumerate(self.c):
            cg.c[i] = v
        cg.dt, cg.h, cg.rho = dt, h, rho
        cg.kappa, cg.sx_i, cg.sx_h = _ptr(self.kappa), _ptr(self.sx_i), _ptr(self.sx_h)
        cg.sz_i, cg.sz_h = _ptr(self.sz_i), _ptr(self.sz_h)
        self._c = cg

    def line(self, z, ix0, n, scale=1.0):
        """Injection / sampling line at depth z (km), physical columns
        ix0..ix0+n-1. Pressure lives on rows k, velocity v_z on rows k+1/2."""
        zeta = (z - self.z_origin) / self.h + self.nsp
        kp, wp0, wp1 = row_weights(zeta)
        kv, wv0, wv1 = row_weights(zeta - 0.5)
        if not (0 <= kp and kp + 1 < self.NZ and 0 <= kv and kv + 1 < self.NZ - 1):
            raise ValueError("line outside the grid")
        if ix0 < 0 or ix0 + n > self.nx:
            raise ValueError("line columns outside the physical grid")
        L = _CLine()
        L.i0, L.n, L.kp, L.wp0, L.wp1 = ix0 + self.nsp, n, kp, wp0, wp1
        L.kv, L.wv0, L.wv1, L.scale = kv, wv0, wv1, scale
        return L


def simulate(g: Grid, nt: int, src, rec, h=None, f=None, want_p=True, want_v=False):
    """The 2x2 modelling operator of eqn:fwd: sources (h_s, f_s) on line
    `src` -> traces (P p, P v_z) on line `rec`, gathers [nt][n]."""
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    f = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    outp = np.zeros((nt, rec.n)) if want_p else None
    outv = np.zeros((nt, rec.n)) if want_v else None
    lib().og_forward(ctypes.byref(g._c), nt, ctypes.byref(src), _ptr(h), _ptr(f),
                     ctypes.byref(rec), _ptr(outp), _ptr(outv))
    return outp, outv


def simulate_adj(g: Grid, nt: int, src, rec, yp=None, yv=None, want_h=True, want_f=False):
    """Exact transpose of ``simulate`` (Appendix A, by reverse-time sweep)."""
    yp = None if yp is None else np.ascontiguousarray(yp, dtype=np.float64)
    yv = None if yv is None else np.ascontiguousarray(yv, dtype=np.float64)
    hb = np.zeros((nt, src.n)) if want_h else None
    fb = np.zeros((nt, src.n)) if want_f else None
    lib().og_adjoint(ctypes.byref(g._c), nt, ctypes.byref(src), _ptr(hb), _ptr(fb),
                     ctypes.byref(rec), _ptr(yp), _ptr(yv))
    return hb, fb


class Slab:
    """Thin-slab grid around a plane z0 and its datum z0 + dir * dz
    (eqn:lamnear): physical rows from the shallower to the deeper of the two
    plus k rows of margin each side, taken from the full model (rows outside it
    repeat its edge rows), with the same sponge on every side."""

    def __init__(self, full: Grid, vel_full, z0, zd, order):
        h, R = full.h, order // 2
        kmin = math.floor(min(z0, zd) / h + 1e-6) - R
        kmax = math.ceil(max(z0, zd) / h - 1e-6) + R
        rows = np.clip(np.arange(kmin, kmax + 1), 0, vel_full.shape[0] - 1)
        self.grid = Grid(vel_full[rows, :], h, full.dt, order, full.nsp, full.rho,
                         v_max=full.v_max, z_origin=kmin * h)
        self.z0, self.zd = z0, zd


class Problem:
    """One source subproblem (eqn:esis) on a full grid with its two slabs."""

    def __init__(self, spec, vel, v_max=None):
        self.spec = spec
        self.vel = np.asarray(vel, dtype=np.float64)
        s = spec
        self.nt = s.nt
        # v_max sets the sponge strength; fixing it keeps the sponge constant
        # when the model is perturbed (finite-difference checks)
        self.g = Grid(self.vel, s.h, s.dt, s.order, s.n_sponge, s.rho, v_max=v_max)
        self.src = self.g.line(s.z_s, s.ix_line0, s.n_line)
        self.rec = self.g.line(s.z_r, s.ix_rec0, s.n_rec)
        # propagation direction from the source line towards the receivers;
        # both data are placed one dz further along it.
        self.dir = 1.0 if s.z_r > s.z_s else -1.0
        # the paper's prefactors hold for its examples' geometry (dir = -1)
        self.sgn = -self.dir
        self.slab_s = Slab(self.g, self.vel, s.z_s, s.z_s + self.dir * s.dz_datum, s.order)
        self.slab_r = Slab(self.g, self.vel, s.z_r, s.z_r + self.dir * s.dz_datum, s.order)
        x = (s.ix_line0 + np.arange(s.n_line)) * s.h
        self.dist = np.abs(x - s.x_s)            # |x - x_s|, km (eqn:penop)

    # -- S and S^T (eqn:sdef, eqn:sadj1) --------------------------------
    def S(self, h):
        return simulate(self.g, self.nt, self.src, self.rec, h=h)[0]

    def ST(self, d):
        return simulate_adj(self.g, self.nt, self.src, self.rec, yp=d)[0]

    # -- thin-slab weights ------------------------------------------------
    def _sym_lambda(self, slab: Slab, ix0, n, r):
        """-4 Pi_1 S^T (Pi_0^T Pi_1 + Pi_1^T Pi_0) S Pi_1^T on a slab
        (eqn:winvcomp): velocity-source injection of r on the plane, both
        traces at the datum, components exchanged, transpose sweep, velocity
        injection's adjoint read out."""
        g = slab.grid
        pl, dl = g.line(slab.z0, ix0, n), g.line(slab.zd, ix0, n)
        tp, tv = simulate(g, self.nt, pl, dl, f=r, want_p=True, want_v=True)
        _, fb = simulate_adj(g, self.nt, pl, dl, yp=tv, yv=tp, want_h=False, want_f=True)
        return -4.0 * self.sgn * fb

    def Wminv(self, r):
        s = self.spec
        return self._sym_lambda(self.slab_s, s.ix_line0, s.n_line, r)

    def Wd(self, d):
        s = self.spec
        return self._sym_lambda(self.slab_r, s.ix_rec0, s.n_rec, d)

    def Wm(self, h):
        """-Pi_0 S^T (Pi_1^T Pi_0 + Pi_0^T Pi_1) S Pi_0^T on the z_s slab."""
        s, slab = self.spec, self.slab_s
        g = slab.grid
        pl, dl = g.line(slab.z0, s.ix_line0, s.n_line), g.line(slab.zd, s.ix_line0, s.n_line)
        tp, tv = simulate(g, self.nt, pl, dl, h=h, want_p=True, want_v=True)
        hb, _ = simulate_adj(g, self.nt, pl, dl, yp=tv, yv=tp, want_h=True, want_f=False)
        return -1.0 * self.sgn * hb

    # -- unsymmetrised pressure-to-source and time-reversal inverse ---------
    def lambda_tilde(self, r, transpose=False):
        """eqn:lamtilde: Lambda~ = -8 (V+_{zs,zs+dz})^T Pi_0 S+ Pi_1^T r (velocity
        injection of r on the plane, the pressure trace at the datum taken back
        through V^T); with transpose=True eqn:lamtransp:
        Lambda~^T = -8 Pi_1 S^T Pi_0^T V r (the v_z trace at the datum taken
        back through the pressure-trace adjoint)."""
        s, slab = self.spec, self.slab_s
        g = slab.grid
        pl, dl = g.line(slab.z0, s.ix_line0, s.n_line), g.line(slab.zd, s.ix_line0, s.n_line)
        tp, tv = simulate(g, self.nt, pl, dl, f=r, want_p=True, want_v=True)
        if transpose:
            _, fb = simulate_adj(g, self.nt, pl, dl, yp=tv, want_h=False, want_f=True)
        else:
            _, fb = simulate_adj(g, self.nt, pl, dl, yv=tp, want_h=False, want_f=True)
        return -8.0 * self.sgn * fb

    def time_reversal_inverse(self, d):
        """eqn:approxinv: h ~ 4 (V+_{zs,zr})^T d -- the data injected as a
        vertical load at the receivers, propagated back in time, the v_z
        response read on the source line."""
        _, fb = simulate_adj(self.g, self.nt, self.src, self.rec, yv=d, want_h=False, want_f=True)
        return 4.0 * fb

    # -- penalty and normal operator ---------------------------------------
    def A(self, h):
        return h * self.dist[None, :]

    def N(self, p, alpha, mode="pcg"):
        """eqn:normpart: (S^T W_d S + alpha A^T W_m A) p, or the Euclidean
        S^T S + alpha A^T A for plain CG (W_m = W_d = I)."""
        if mode == "pcg":
            q = self.ST(self.Wd(self.S(p)))
            if alpha != 0.0:
                q = q + alpha * self.A(self.Wm(self.A(p)))
            return q
        q = self.ST(self.S(p))
        if alpha != 0.0:
            q = q + alpha * self.A(self.A(p))
        return q

    def rhs(self, d, mode="pcg"):
        """S^* d = S^T W_d d (eqn:sadjwt), or S^T d for plain CG."""
        return self.ST(self.Wd(d)) if mode == "pcg" else self.ST(d)

    def Minv(self, r, alpha, mode="pcg"):
        """eqn:defprecond: D W~_m^{-1} D with D = (I + alpha A^T A)^{-1/2};
        the identity for plain CG."""
        if mode != "pcg":
            return r.copy()
        D = 1.0 / np.sqrt(1.0 + alpha * self.dist ** 2)
        return D[None, :] * self.Wminv(D[None, :] * r)

    def point_source_data(self, wavelet, x_d, z_d):
        """Pressure gather at the receivers from a point pressure source
        (constitutive defect) w(t) delta(x - x_d) delta(z - z_d)."""
        s = self.spec
        ix = round(x_d / s.h)
        if abs(ix * s.h - x_d) > 1e-9:
            raise ValueError("point source must sit on a grid column")
        pt = self.g.line(z_d, ix, 1, scale=1.0 / s.h)
        return simulate(self.g, self.nt, pt, self.rec,
                        h=np.asarray(wavelet, dtype=np.float64).reshape(-1, 1))[0]


def pcg(prob: Problem, d, alpha, maxit, rtol, mode="pcg", callback=None):
    """Algorithm 1 (preconditioned CG, standard version) on N h = S^* d.

    Returns (h, history) with history[k] = ||r_k||_2. The loop stops as soon
    as ||r_{k+1}|| <= rtol ||r_0|| or after maxit updates of h; this yields
    the same iterates as testing at the bottom of the loop. A non-positive
    <p_k, q_k> or <g_k, r_k> raises ArithmeticError (breakdown: N or M^{-1}
    not positive on the Krylov space)."""
    vdot = lambda a, b: float(np.sum(a * b))
    h = np.zeros((prob.nt, prob.spec.n_line))
    r = prob.rhs(d, mode)
    p = prob.Minv(r, alpha, mode)
    g = p.copy()
    q = prob.N(p, alpha, mode)
    gr = vdot(g, r)
    hist = [math.sqrt(vdot(r, r))]
    for k in range(maxit):
        pq = vdot(p, q)
        if not (pq > 0.0 and gr > 0.0):
            raise ArithmeticError(f"PCG breakdown at k={k}: <p,q>={pq}, <g,r>={gr}")
        a = gr / pq
        h = h + a * p
        r = r - a * q
        hist.append(math.sqrt(vdot(r, r)))
        if callback is not None:
            callback(k + 1, h, r)
        if hist[-1] <= rtol * hist[0]:
            break
        g = prob.Minv(r, alpha, mode)
        gr_new = vdot(g, r)
        beta = gr_new / gr
        gr = gr_new
        p = g + beta * p
        q = prob.N(p, alpha, mode)
    return h, np.array(hist)


def step(g: Grid, p, vx, vz):
    """One source-free forward step in place on padded fields [NZ][NX]
    (vx valid for x index < NX-1, vz for z index < NZ-1)."""
    for a in (p, vx, vz):
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == (g.NZ, g.NX)
    lib().og_step_fwd(ctypes.byref(g._c), _ptr(p), _ptr(vx), _ptr(vz), None, None, None,
                      None, None, None)


# --------------------------------------------------------------------------
# Reduced objective of variable projection and its gradient in the velocity.
# --------------------------------------------------------------------------
def objective(prob: Problem, h, d, alpha):
    """Phi(c, h) = ||S[c] h - d||^2 + alpha ||A h||^2, the objective of the
    source subproblem eqn:esis (A of eqn:penop). Minimised over h it is the
    reduced objective J(c) that variable projection optimises over c
    (eqn:esi and the paragraph after eqn:esis)."""
    r = prob.S(h) - d
    return float(np.sum(r * r) + alpha * np.sum(prob.A(h) ** 2))


def velocity_gradient(prob: Problem, h, d):
    """d Phi / d v at fixed h: the gradient of ||S[v] h - d||^2 with respect
    to the physical velocity model v[nz][nx] (the penalty does not depend on
    v). At h = the minimiser of eqn:esis this is the gradient of the reduced
    objective, because Phi is stationary in h there (variable projection).

    Discrete adjoint state method (the paper's route to exact adjoints,
    section "Synthetic models and simulation" and Appendix A), in the
    discretisation's own steps:
      1. forward sweep of S h, keeping p^n for n = 0 .. nt;
      2. residual r = P p - d; the objective's derivative in the traces is 2 r;
      3. reverse sweep of the transposed step on 2 r. After the transposed
         sampling of sample n is added, the adjoint pressure pbar equals
         dPhi/dp^{n+1};
      4. p^{n+1} = A_p p^n + kappa (dt/h) B_p q^n with q^n independent of kappa
         (q^n = -D- v^{n+1/2} + injected h), so dp^{n+1}/dkappa at a point is
         (p^{n+1} - A_p p^n) / kappa there, and
         dPhi/dkappa = sum_n pbar^{n+1} (p^{n+1} - A_p p^n) / kappa;
      5. kappa = rho v_pad^2 on the padded grid, v_pad the model extended into
         the sponge by edge replication: dPhi/dv sums 2 rho v_pad dPhi/dkappa
         over the padded points that copy each model point.
    The sponge profile (it depends on max v) is held fixed."""
    g, src, rec, nt = prob.g, prob.src, prob.rec, prob.nt
    L = lib()
    h = np.ascontiguousarray(h, dtype=np.float64)
    shape = (g.NZ, g.NX)
    p, vx, vz = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    ps = [p.copy()]
    y = np.zeros((nt, rec.n))
    for n in range(nt):
        row = np.ascontiguousarray(h[n])
        yrow = np.zeros(rec.n)
        L.og_step_fwd(ctypes.byref(g._c), _ptr(p), _ptr(vx), _ptr(vz), ctypes.byref(src),
                      _ptr(row), None, ctypes.byref(rec), _ptr(yrow), None)
        y[n] = yrow
        ps.append(p.copy())
    ybar = 2.0 * (y - d)
    s_p = 0.5 * g.dt * (g.sz_i[:, None] + g.sx_i[None, :])
    a_p = (1.0 - s_p) / (1.0 + s_p)
    pb, vxb, vzb = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    q, wx, wz = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    gk = np.zeros(shape)
    cols = rec.i0 + np.arange(rec.n)
    for n in range(nt - 1, -1, -1):
        pb[rec.kp, cols] += rec.wp0 * ybar[n]
        if rec.wp1 != 0.0:
            pb[rec.kp + 1, cols] += rec.wp1 * ybar[n]
        gk += pb * (ps[n + 1] - a_p * ps[n]) / g.kappa
        L.og_step_adj(ctypes.byref(g._c), _ptr(pb), _ptr(vxb), _ptr(vzb), ctypes.byref(src),
                      None, None, _ptr(q), _ptr(wx), _ptr(wz))
    gv_pad = gk * 2.0 * np.sqrt(g.rho * g.kappa)          # 2 rho v dPhi/dkappa
    kk = np.clip(np.arange(g.NZ) - g.nsp, 0, g.nz - 1)
    ii = np.clip(np.arange(g.NX) - g.nsp, 0, g.nx - 1)
    out = np.zeros((g.nz, g.nx))
    np.add.at(out, (kk[:, None], ii[None, :]), gv_pad)
    return out
