"""The paper's speed-up of its preconditioned iteration over plain CG
(Algorithm 1 against CG on the Euclidean normal equation, in its examples
about 4-5 times fewer iterations) is a statement about its own geometry, so
it is reported here, not asserted. Run with `-s` to see the report: the
relative residual of each method in its own norm, and the Euclidean data
misfit, per iteration, on the oracle-sized configuration (201 x 101
homogeneous model, 1000 steps, data from a point source on the line).

What is asserted is what the mathematics fixes: the data are fitted
exactly by h* = (wavelet / h) delta_{x = x_s}, and CG lowers its objective
||S h - d||^2 + alpha ||A h||^2 at every iteration (it minimises it over
growing Krylov spaces)."""
import numpy as np

from paper_2203_16573_gb300 import workloads as W

ITERS = 12


def test_report_pcg_and_cg_on_the_oracle_sized_workload(oracle):
    s = W.c1()
    P = oracle.Problem(s, W.velocity(s))
    w = W.ricker(s)
    d = P.point_source_data(w, s.x_d, s.z_d)
    hstar = np.zeros((s.nt, s.n_line))
    hstar[:, round(s.x_s / s.h) - s.ix_line0] = w / s.h
    assert np.linalg.norm(P.S(hstar) - d) <= 1e-13 * np.linalg.norm(d)
    report = {}
    for mode in ("pcg", "cg"):
        misfit, obj = [], []

        def cb(k, h, r):
            res = P.S(h) - d
            misfit.append(np.linalg.norm(res) / np.linalg.norm(d))
            obj.append(np.sum(res ** 2) + s.alpha * np.sum(P.A(h) ** 2))
        _, hist = oracle.pcg(P, d, s.alpha, ITERS, 0.0, mode=mode, callback=cb)
        rel = np.asarray(hist) / hist[0]
        report[mode] = (rel, misfit)
        assert np.all(np.isfinite(rel))
        if mode == "cg":
            assert all(b < a for a, b in zip(obj, obj[1:])), obj
    print()
    for mode, (rel, misfit) in report.items():
        first = {tol: (int(np.argmax(rel <= tol)) if np.any(rel <= tol) else None)
                 for tol in (1e-1, 1e-2)}
        print(f"{mode}: relative residual {' '.join(f'{x:.2e}' for x in rel)}")
        print(f"{mode}: first iteration at 1e-1 / 1e-2: {first[1e-1]} / {first[1e-2]}")
        print(f"{mode}: data misfit {' '.join(f'{x:.3f}' for x in misfit)}")
