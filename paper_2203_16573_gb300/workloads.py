"""Seeded synthetic inputs for the source-subproblem solver.

This module only *generates inputs*: velocity models, source wavelets,
acquisition geometry and random gathers. It holds none of the method's
arithmetic (no stencils, no operators, no Krylov steps), so both the CUDA
path and the FP64 CPU oracle can take their inputs from it without sharing
any computation.

Units throughout: km, s, km/s, g/cm^3 (so kappa = rho v^2 is in GPa).

Workload shapes follow the paper's synthetic media (Section "Synthetic
models and simulation": an 8 km x 4 km homogeneous medium and a low-velocity
lens in the middle of it, constant density) scaled to the two single-GPU
configurations this library is measured on:

* ``c1``: homogeneous 1.5 km/s, 201 x 101 points, h = 10 m, 20-point sponge,
  order 4, dt = 0.8 ms, 1000 steps; 10 Hz Ricker point source at
  (1000 m, 300 m); 201 receivers at 20 m depth; extended-source line at 300 m;
  alpha = 1e-2; 20 PCG iterations.
* ``c2``: 601 x 301 points, h = 10 m, v = 1.5 + 1.5 z/3 km/s with a -20 %
  Gaussian lens (sigma = 300 m) at (3.0 km, 1.5 km); order 8, 40-point sponge,
  dt = 0.5 ms, 3000 steps; 601 surface receivers; 15 Hz Ricker point source at
  (3.0 km, 2.4 km) on the extended-source line z = 2.4 km; alpha = 1e-2;
  30 PCG iterations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 20220331


@dataclasses.dataclass(frozen=True)
class Spec:
    """Grid, geometry and solve settings of one source-subproblem workload."""
    name: str
    nx: int            # physical grid points in x
    nz: int            # physical grid points in z
    h: float           # grid step, km
    dt: float          # time step, s
    nt: int            # time steps (= gather length)
    order: int         # spatial order 2k of the staggered differences
    n_sponge: int      # absorbing points padded outside the physical grid
    rho: float         # constant density, g/cm^3
    z_s: float         # extended-source line depth, km
    ix_line0: int      # first physical column of the source line
    n_line: int        # source-line points
    z_r: float         # receiver line depth, km
    ix_rec0: int       # first physical column of the receiver line
    n_rec: int         # receivers
    x_s: float         # physical source position (penalty centre), km
    x_d: float         # point source used to synthesise the data, km
    z_d: float
    f_peak: float      # Ricker peak frequency, Hz
    alpha: float       # penalty weight
    maxit: int         # PCG iteration cap
    rtol: float        # relative residual target
    dz_datum: float = 0.1   # thin-slab datum distance, km (the paper's 100 m)
    model: str = "homogeneous"  # "gradient", "gradient_lens", "gradient_perturbed"
    v0: float = 1.5

    @property
    def padded(self):
        return (self.nz + 2 * self.n_sponge, self.nx + 2 * self.n_sponge)


def c1() -> Spec:
    return Spec(name="c1_homog_201x101_o4_nt1000", nx=201, nz=101, h=0.01,
                dt=0.8e-3, nt=1000, order=4, n_sponge=20, rho=1.0,
                z_s=0.3, ix_line0=0, n_line=201, z_r=0.02, ix_rec0=0,
                n_rec=201, x_s=1.0, x_d=1.0, z_d=0.3, f_peak=10.0,
                alpha=1e-2, maxit=20, rtol=1e-3)


def c2() -> Spec:
    return Spec(name="c2_lens_601x301_o8_nt3000", nx=601, nz=301, h=0.01,
                dt=0.5e-3, nt=3000, order=8, n_sponge=40, rho=1.0,
                z_s=2.4, ix_line0=0, n_line=601, z_r=0.0, ix_rec0=0,
                n_rec=601, x_s=3.0, x_d=3.0, z_d=2.4, f_peak=15.0,
                alpha=1e-2, maxit=30, rtol=1e-3, model="gradient_lens")


def c3_shots(n_shots: int = 64, nt: int = 5000) -> list[Spec]:
    """Batched survey on one 2001 x 801 lens model (h = 5 m, 10 km x 4 km,
    order 8, 40-point sponge, dt = 0.4 ms, 5000 steps): shot i is a 15 Hz
    Ricker point source at x_i = (i + 1/2) 10 km / n at 50 m depth; its
    extended source lives on the line z = 50 m within 1 km of x_i (clipped to
    the model); every shot records on 2001 receivers on the line z = 3.5 km;
    alpha cycles through 1e-3, 1e-2, 1e-1."""
    out = []
    for i in range(n_shots):
        xs = (i + 0.5) * 10.0 / n_shots
        ixs = int(round(xs / 0.005))
        xs = ixs * 0.005
        i0 = max(0, ixs - 200)
        i1 = min(2000, ixs + 200)
        out.append(Spec(name=f"c3_shot{i:02d}_2001x801_o8_nt{nt}", nx=2001, nz=801, h=0.005,
                        dt=0.4e-3, nt=nt, order=8, n_sponge=40, rho=1.0, z_s=0.05,
                        ix_line0=i0, n_line=i1 - i0 + 1, z_r=3.5, ix_rec0=0, n_rec=2001,
                        x_s=xs, x_d=xs, z_d=0.05, f_peak=15.0,
                        alpha=(1e-3, 1e-2, 1e-1)[i % 3], maxit=30, rtol=1e-3,
                        model="gradient_lens"))
    return out


def c4_shots(n_shots: int = 32, nt: int = 4000) -> list[Spec]:
    """Gradient workload: 1001 x 401 grid (8 km x 3.2 km, h = 8 m), order 8,
    40-point sponge, dt = 0.6 ms, 4000 steps. Shot i: a 15 Hz Ricker point
    source at x_i = (i + 1/2) 8 km / n at 40 m depth, its extended source on
    the line z = 40 m within 1 km of x_i (clipped to the model), 1001
    receivers on the line z = 3.0 km; alpha = 1e-2. The data come from the
    "true" model (model "gradient_perturbed": the linear gradient 1.5 -> 3.0
    km/s times 1 + a smooth random perturbation of at most 10 %, correlation
    length 200 m); the gradient is taken at the unperturbed linear gradient
    (model "gradient", see ``background``)."""
    out = []
    for i in range(n_shots):
        xs = (i + 0.5) * 8.0 / n_shots
        ixs = int(round(xs / 0.008))
        xs = ixs * 0.008
        i0, i1 = max(0, ixs - 125), min(1000, ixs + 125)
        out.append(Spec(name=f"c4_shot{i:02d}_1001x401_o8_nt{nt}", nx=1001, nz=401, h=0.008,
                        dt=0.6e-3, nt=nt, order=8, n_sponge=40, rho=1.0, z_s=0.04,
                        ix_line0=i0, n_line=i1 - i0 + 1, z_r=3.0, ix_rec0=0, n_rec=1001,
                        x_s=xs, x_d=xs, z_d=0.04, f_peak=15.0, alpha=1e-2, maxit=10,
                        rtol=1e-3, model="gradient_perturbed"))
    return out


def paper_pcg(alpha: float = 0.0, lens: bool = True) -> Spec:
    """The setting of the paper's CG / PCG comparison ("Preconditioned CG
    iteration"): an 8 km x 4 km medium at h = 20 m (401 x 201), order 8,
    40-point sponge, dt = 2 ms, 1500 steps (3 s); receivers on z = 1 km and
    the extended-source line on z = 3 km, both over x = 2 .. 6 km (201
    points); a point source at (3.5 km, 3.5 km) with the paper's bandpass
    wavelet (``bandpass``); penalty centre x_s = 3.5 km. lens=True is the
    model the data are simulated in (``paper_lens``: kappa = 4 GPa with a
    central low-velocity lens down to 1.6 GPa); lens=False the homogeneous
    model (kappa = 4 GPa, v = 2 km/s) the problem is solved in."""
    return Spec(name=f"paper_pcg_401x201_o8_nt1500_{'lens' if lens else 'homog'}", nx=401, nz=201,
                h=0.02, dt=2e-3, nt=1500, order=8, n_sponge=40, rho=1.0, z_s=3.0,
                ix_line0=100, n_line=201, z_r=1.0, ix_rec0=100, n_rec=201, x_s=3.5, x_d=3.5,
                z_d=3.5, f_peak=7.5, alpha=alpha, maxit=60, rtol=0.0,
                model="paper_lens" if lens else "homogeneous", v0=2.0)


def background(spec: Spec) -> Spec:
    """The same workload on the unperturbed linear-gradient model."""
    return dataclasses.replace(spec, model="gradient")


def smooth_perturbation(nz: int, nx: int, h: float, corr: float, amp: float,
                        seed: int) -> np.ndarray:
    """Seeded smooth random field [nz][nx]: white noise blurred by a Gaussian
    of standard deviation corr (km), scaled so that max |field| = amp."""
    g = np.random.default_rng(SEED + seed).standard_normal((nz, nx))
    w = max(1, int(round(corr / h)))
    k = np.arange(-3 * w, 3 * w + 1)
    ker = np.exp(-0.5 * (k / w) ** 2)
    ker /= ker.sum()
    g = np.apply_along_axis(lambda s: np.convolve(np.pad(s, 3 * w, mode="wrap"), ker, "valid"), 0, g)
    g = np.apply_along_axis(lambda s: np.convolve(np.pad(s, 3 * w, mode="wrap"), ker, "valid"), 1, g)
    return amp * g / np.max(np.abs(g))


def small(order: int = 4, nt: int = 400, model: str = "gradient_lens",
          n_sponge: int = 12) -> Spec:
    """A reduced c2-like case (same structure, ~1/5 linear size) that the
    oracle finishes in seconds while still spanning many CUDA tiles with a
    ragged tail in both x and z."""
    return Spec(name=f"small_o{order}", nx=133, nz=71, h=0.01, dt=0.7e-3,
                nt=nt, order=order, n_sponge=n_sponge, rho=1.0, z_s=0.55,
                ix_line0=3, n_line=127, z_r=0.05, ix_rec0=0, n_rec=133,
                x_s=0.66, x_d=0.66, z_d=0.55, f_peak=15.0, alpha=1e-2,
                maxit=12, rtol=1e-3, model=model, v0=1.5)


def tiny(order: int = 4) -> Spec:
    """A grid small enough to build every operator densely column by column."""
    return Spec(name=f"tiny_o{order}", nx=14, nz=16, h=0.01, dt=1.0e-3,
                nt=36, order=order, n_sponge=5, rho=1.0, z_s=0.12,
                ix_line0=2, n_line=9, z_r=0.02, ix_rec0=1, n_rec=11,
                x_s=0.06, x_d=0.06, z_d=0.12, f_peak=40.0, alpha=5e-2,
                maxit=200, rtol=1e-12, dz_datum=0.04, model="homogeneous")


def velocity(spec: Spec) -> np.ndarray:
    """Physical velocity model v[nz][nx] in km/s (float64)."""
    z = np.arange(spec.nz) * spec.h
    x = np.arange(spec.nx) * spec.h
    if spec.model == "homogeneous":
        return np.full((spec.nz, spec.nx), spec.v0, dtype=np.float64)
    if spec.model == "gradient":
        zmax = (spec.nz - 1) * spec.h
        zz = np.repeat(z[:, None], spec.nx, axis=1)
        return spec.v0 * (1.0 + zz / zmax)
    if spec.model == "gradient_perturbed":
        zmax = (spec.nz - 1) * spec.h
        zz = np.repeat(z[:, None], spec.nx, axis=1)
        pert = smooth_perturbation(spec.nz, spec.nx, spec.h, 0.2, 0.1, seed=404)
        return spec.v0 * (1.0 + zz / zmax) * (1.0 + pert)
    if spec.model == "gradient_lens":
        # linear gradient v0 -> 2 v0 from top to bottom, times a -20 %
        # Gaussian lens at the centre with sigma = depth / 10 (300 m for 3 km)
        zmax = (spec.nz - 1) * spec.h
        xc, zc = 0.5 * (spec.nx - 1) * spec.h, 0.5 * zmax
        sig = 0.1 * zmax
        zz, xx = np.meshgrid(z, x, indexing="ij")
        v = spec.v0 * (1.0 + zz / zmax)
        lens = 1.0 - 0.2 * np.exp(-((xx - xc) ** 2 + (zz - zc) ** 2) / (2.0 * sig ** 2))
        return v * lens
    if spec.model == "paper_lens":
        # kappa = 4 GPa (rho = 1: v = 2 km/s) falling to 1.6 GPa at the centre
        # of the rectangle through a Gaussian of sigma = 0.5 km (the paper
        # gives the end values, not the lens profile)
        xc, zc = 0.5 * (spec.nx - 1) * spec.h, 0.5 * (spec.nz - 1) * spec.h
        zz, xx = np.meshgrid(z, x, indexing="ij")
        kappa = 4.0 - 2.4 * np.exp(-((xx - xc) ** 2 + (zz - zc) ** 2) / (2.0 * 0.5 ** 2))
        return np.sqrt(kappa / spec.rho)
    raise ValueError(spec.model)


def bandpass(spec: Spec, corners=(1.0, 2.5, 7.5, 12.5), delay: float = 0.4) -> np.ndarray:
    """The paper's source wavelet: a zero-phase bandpass filter with a
    trapezoidal amplitude spectrum (0 below 1 Hz, rising to 1 at 2.5 Hz, flat
    to 7.5 Hz, falling to 0 at 12.5 Hz), delayed by `delay` s and normalised
    to a unit peak, sampled at the half-step times (n + 1/2) dt; the first
    0.2 s are tapered by a half cosine so that the source starts from rest."""
    n = 1 << int(math.ceil(math.log2(8 * spec.nt)))
    f = np.fft.rfftfreq(n, spec.dt)
    f1, f2, f3, f4 = corners
    amp = np.clip(np.minimum((f - f1) / (f2 - f1), (f4 - f) / (f4 - f3)), 0.0, 1.0)
    w = np.fft.irfft(amp * np.exp(-2j * math.pi * f * (delay + 0.5 * spec.dt)), n)[: spec.nt]
    t = (np.arange(spec.nt) + 0.5) * spec.dt
    w = w * np.where(t < 0.2, 0.5 - 0.5 * np.cos(math.pi * t / 0.2), 1.0)
    return w / np.max(np.abs(w))


def ricker(spec: Spec) -> np.ndarray:
    """Ricker wavelet, peak frequency f_peak, delay 1.5/f_peak, sampled at the
    half-step times (n + 1/2) dt at which a pressure update integrates it."""
    t = (np.arange(spec.nt) + 0.5) * spec.dt - 1.5 / spec.f_peak
    a = (math.pi * spec.f_peak * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def random_gather(nt: int, n: int, seed: int) -> np.ndarray:
    """Standard-normal gather [nt][n] (float64), seeded."""
    return np.random.default_rng(SEED + seed).standard_normal((nt, n))


def smooth_random_gather(nt: int, n: int, seed: int, width_t: int = 6,
                         width_x: int = 3) -> np.ndarray:
    """A band-limited random gather (random normal field blurred by a
    separable Gaussian), for tests that need a source with little energy at
    the grid's Nyquist wavenumbers."""
    g = random_gather(nt, n, seed)

    def blur(a, w, axis):
        if w <= 0:
            return a
        k = np.arange(-3 * w, 3 * w + 1)
        ker = np.exp(-0.5 * (k / w) ** 2)
        ker /= ker.sum()
        return np.apply_along_axis(lambda s: np.convolve(s, ker, mode="same"), axis, a)

    return blur(blur(g, width_t, 0), width_x, 1)
