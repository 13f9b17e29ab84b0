"""The seeded input recipes (CPU): velocity models, shot layouts of the
batched-survey and gradient workloads, the smooth model perturbation and the
Ricker wavelet, against the numbers the workload descriptions state."""
import math

import numpy as np
import pytest

from paper_2203_16573_gb300 import workloads as W


def test_single_shot_lens_model():
    s = W.c2()
    v = W.velocity(s)
    assert v.shape == (301, 601)
    # linear gradient 1.5 -> 3.0 km/s, -20 % Gaussian lens centred at (3 km, 1.5 km)
    assert math.isclose(v[150, 300], (1.5 + 1.5 * 1.5 / 3.0) * 0.8, rel_tol=1e-12)
    assert np.unravel_index(np.argmin(v / (1.5 * (1 + np.arange(301)[:, None] * 0.01 / 3.0))),
                            v.shape) == (150, 300)
    assert math.isclose(v[0, 0], 1.5, rel_tol=1e-3) and math.isclose(v[-1, 0], 3.0, rel_tol=1e-3)
    assert math.isclose(v.max() * s.dt / s.h, 0.15, rel_tol=1e-3)   # CFL 0.15
    assert (s.x_d, s.z_d) == (s.x_s, s.z_s) == (3.0, 2.4)


def test_survey_shot_layout():
    shots = W.c3_shots(64)
    assert len(shots) == 64
    for i, s in enumerate(shots):
        x = (i + 0.5) * 10.0 / 64
        assert abs(s.x_s - x) <= s.h / 2 + 1e-12
        ixs = round(s.x_s / s.h)
        assert abs(s.x_s - ixs * s.h) < 1e-12
        assert s.ix_line0 == max(0, ixs - 200)
        assert s.ix_line0 + s.n_line - 1 == min(s.nx - 1, ixs + 200)     # 1 km each side, clipped
        assert (s.z_s, s.z_r, s.nt, s.nx, s.nz, s.h) == (0.05, 3.5, 5000, 2001, 801, 0.005)
        assert s.alpha == (1e-3, 1e-2, 1e-1)[i % 3]
        assert s.n_rec == 2001 and s.ix_rec0 == 0


def test_gradient_workload_models():
    shots = W.c4_shots(32)
    assert len(shots) == 32
    for i, s in enumerate(shots):
        assert abs(s.x_s - (i + 0.5) * 8.0 / 32) <= s.h / 2 + 1e-12
        assert s.model == "gradient_perturbed" and W.background(s).model == "gradient"
    s = shots[0]
    true, back = W.velocity(s), W.velocity(W.background(s))
    rel = true / back - 1.0
    assert math.isclose(np.abs(rel).max(), 0.1, rel_tol=1e-12)      # at most 10 %
    assert math.isclose(back[0, 0], 1.5) and math.isclose(back[-1, 0], 3.0)


def test_smooth_perturbation_amplitude_and_correlation():
    nz, nx, h, corr = 300, 400, 0.008, 0.2
    f = W.smooth_perturbation(nz, nx, h, corr, 0.1, seed=9)
    assert np.array_equal(f, W.smooth_perturbation(nz, nx, h, corr, 0.1, seed=9))
    assert math.isclose(np.abs(f).max(), 0.1, rel_tol=1e-12)
    w = round(corr / h)
    g = f - f.mean()

    def acf(lag):
        return float((g[:, lag:] * g[:, :-lag]).sum() / (g[:, lag:] ** 2).sum())
    # a Gaussian blur of width w gives correlation exp(-lag^2 / (4 w^2))
    assert 0.6 < acf(w) < 0.9
    assert acf(4 * w) < 0.15


def test_ricker_wavelet():
    s = W.c2()
    r = W.ricker(s)
    t = (np.arange(s.nt) + 0.5) * s.dt
    k = int(np.argmax(r))
    assert abs(t[k] - 1.5 / s.f_peak) <= s.dt
    assert math.isclose(r[k], 1.0, rel_tol=1e-3)
    assert abs(r.sum()) * s.dt < 1e-6          # zero mean


def test_paper_comparison_setting():
    """The setting of the paper's CG / PCG comparison: 8 km x 4 km at 20 m,
    lines at 1 km and 3 km over x = 2 .. 6 km, point source at (3.5, 3.5) km,
    kappa = 4 GPa falling to 1.6 GPa at the lens centre, and a bandpass
    wavelet whose spectrum is the 1 - 2.5 - 7.5 - 12.5 Hz trapezoid."""
    lens, homog = W.paper_pcg(lens=True), W.paper_pcg(lens=False)
    assert (lens.nx - 1) * lens.h == pytest.approx(8.0) and (lens.nz - 1) * lens.h == pytest.approx(4.0)
    assert lens.ix_line0 * lens.h == pytest.approx(2.0)
    assert (lens.ix_line0 + lens.n_line - 1) * lens.h == pytest.approx(6.0)
    assert (lens.z_r, lens.z_s, lens.x_d, lens.z_d) == (1.0, 3.0, 3.5, 3.5)
    kl = lens.rho * W.velocity(lens) ** 2
    kh = homog.rho * W.velocity(homog) ** 2
    assert np.allclose(kh, 4.0)
    assert kl[100, 200] == pytest.approx(1.6) and kl.min() == pytest.approx(1.6)
    assert kl[0, 0] == pytest.approx(4.0, abs=1e-6)
    w = W.bandpass(lens)
    assert abs(w[0]) < 1e-4 and np.max(np.abs(w)) == pytest.approx(1.0)
    F = np.abs(np.fft.rfft(w, 1 << 14))
    f = np.fft.rfftfreq(1 << 14, lens.dt)
    at = lambda fr: F[np.argmin(np.abs(f - fr))] / F.max()
    assert at(5.0) > 0.9 and at(7.0) > 0.9
    assert at(0.5) < 0.1 and at(14.0) < 0.05
    assert 0.3 < at(1.75) < 0.7 and 0.3 < at(10.0) < 0.7   # half way up and down the ramps
    # CFL of the order-8 scheme at the lens model's maximum speed
    assert W.velocity(lens).max() * lens.dt / lens.h * np.sqrt(2) * 1.3713 < 0.5
