"""Thin Python binding of the C ABI in include/ssx.h (ctypes).

Argument marshalling only: every step of the solver runs in libssx's CUDA
kernels. PyTorch provides device memory and the stream. There is no CPU
fallback: constructing a Context without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libssx.so")

SSX_OK = 0
STATUS = {0: "SSX_OK", 1: "SSX_ERR_ARG", 2: "SSX_ERR_CUDA", 3: "SSX_ERR_CFL", 4: "SSX_ERR_OOM",
          5: "SSX_ERR_BREAKDOWN", 6: "SSX_ERR_NONFINITE", 7: "SSX_ERR_NOT_CONVERGED"}
ERR_ARG = 1
MODE_PCG, MODE_CG = 0, 1
SWEEP_AUTO, SWEEP_STEP, SWEEP_PERSISTENT, SWEEP_TEST_STALL = 0, 1, 2, 3
W_D, W_M, W_M_INV = 0, 1, 2
HOOK_NONE, HOOK_BREAKDOWN, HOOK_NONFINITE = 0, 1, 2

# every symbol the header declares, in declaration order
N_TILE_CONFIGS = 14   # SSX_NUM_TILE_CONFIGS of include/ssx.h
N_MARCH_CONFIGS = 4   # SSX_NUM_MARCH_CONFIGS: marching-kernel ids 2N .. 2N + N_MARCH_CONFIGS - 1
N_TWO_CONFIGS = 3     # SSX_NUM_TWO_CONFIGS: two-step kernel ids 2N + N_MARCH_CONFIGS + m

EXPORTS = ["ssx_version", "ssx_create", "ssx_destroy", "ssx_last_error",
           "ssx_set_velocity_model", "ssx_set_geometry", "ssx_forward", "ssx_adjoint",
           "ssx_weight_apply", "ssx_precond_apply", "ssx_normal_apply",
           "ssx_solve_source_subproblem", "ssx_point_source_data", "ssx_set_timing",
           "ssx_get_stats", "ssx_reset_stats", "ssx_forward_noalloc", "ssx_set_sweep_mode",
           "ssx_set_tile_config", "ssx_lambda_apply", "ssx_time_reversal_inverse",
           "ssx_solve_batch", "ssx_server_create", "ssx_server_submit", "ssx_server_step",
           "ssx_server_poll", "ssx_server_destroy", "ssx_server_last_error",
           "ssx_velocity_gradient", "ssx_last_objective", "ssx_set_test_hook",
           "ssx_server_set_timing", "ssx_server_get_stats", "ssx_server_set_cache_budget",
           "ssx_get_phase_stats"]


class SSXError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.msg = msg


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("space_order", ctypes.c_int),
                ("n_sponge", ctypes.c_int)]


class GeomDesc(ctypes.Structure):
    _fields_ = [("z_s", ctypes.c_double), ("ix_line0", ctypes.c_int), ("n_line", ctypes.c_int),
                ("z_r", ctypes.c_double), ("ix_rec0", ctypes.c_int), ("n_rec", ctypes.c_int),
                ("x_s", ctypes.c_double), ("dz_datum", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("point_updates", ctypes.c_longlong),
                ("sweeps", ctypes.c_longlong), ("sweep_ms", ctypes.c_double),
                ("timed_steps", ctypes.c_longlong), ("timed_point_updates", ctypes.c_double),
                ("tile_cfg", ctypes.c_int * 6)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["tile_cfg"] = list(self.tile_cfg)
        return d


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libssx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2203_16573_gb300.build`")
    L = ctypes.CDLL(path)
    P, vp, i, d = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ssx_version": ([], ctypes.c_char_p),
        "ssx_create": ([P(vp), P(GridDesc), vp], i),
        "ssx_destroy": ([vp], i),
        "ssx_last_error": ([vp], ctypes.c_char_p),
        "ssx_set_velocity_model": ([vp, vp, d], i),
        "ssx_set_geometry": ([vp, P(GeomDesc)], i),
        "ssx_forward": ([vp, vp, vp], i),
        "ssx_adjoint": ([vp, vp, vp], i),
        "ssx_weight_apply": ([vp, i, vp, vp], i),
        "ssx_precond_apply": ([vp, d, vp, vp], i),
        "ssx_normal_apply": ([vp, i, d, vp, vp], i),
        "ssx_solve_source_subproblem": ([vp, vp, d, i, d, i, vp, P(d), P(i)], i),
        "ssx_point_source_data": ([vp, d, d, vp, vp], i),
        "ssx_set_timing": ([vp, i], i),
        "ssx_get_stats": ([vp, P(Stats)], i),
        "ssx_reset_stats": ([vp], i),
        "ssx_get_phase_stats": ([vp, i, ctypes.c_char_p, i, P(ctypes.c_int), P(ctypes.c_int),
                                 P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double),
                                 P(ctypes.c_longlong)], i),
        "ssx_forward_noalloc": ([P(GridDesc), P(GeomDesc), vp, d, vp, vp, vp], i),
        "ssx_set_sweep_mode": ([vp, i], i),
        "ssx_set_tile_config": ([vp, i], i),
        "ssx_lambda_apply": ([vp, i, vp, vp], i),
        "ssx_time_reversal_inverse": ([vp, vp, vp], i),
        "ssx_solve_batch": ([P(vp), i, P(vp), P(d), i, d, i, P(vp), P(d), P(i), P(i)], i),
        "ssx_server_create": ([P(vp), i, ctypes.c_size_t, vp], i),
        "ssx_server_submit": ([vp, P(GridDesc), P(GeomDesc), vp, d, vp, d, i, d, i, vp, P(i)], i),
        "ssx_server_step": ([vp, P(i), P(i)], i),
        "ssx_server_poll": ([vp, i, P(i), P(i), P(i), P(d), P(d)], i),
        "ssx_server_destroy": ([vp], i),
        "ssx_server_last_error": ([vp], ctypes.c_char_p),
        "ssx_velocity_gradient": ([vp, vp, vp, d, i, vp, P(d)], i),
        "ssx_last_objective": ([vp, P(d)], i),
        "ssx_set_test_hook": ([vp, i, i], i),
        "ssx_server_set_timing": ([vp, i], i),
        "ssx_server_set_cache_budget": ([vp, ctypes.c_size_t], i),
        "ssx_server_get_stats": ([vp, P(Stats), P(ctypes.c_longlong), P(ctypes.c_longlong)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _dev_ptr(t: torch.Tensor, shape, dtype=torch.float64, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise TypeError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                        f"got {t.dtype} {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One grid (and its thin slabs) on the current CUDA device."""

    def __init__(self, nx, nz, h, dt, nt, space_order, n_sponge, stream=None):
        self._lib = load_library()
        self.nx, self.nz, self.h, self.dt, self.nt = nx, nz, h, dt, nt
        self.device = torch.device("cuda", torch.cuda.current_device())
        s = torch.cuda.current_stream() if stream is None else stream
        self.stream = s
        gd = GridDesc(nx, nz, h, dt, nt, space_order, n_sponge)
        self._c = ctypes.c_void_p()
        rc = self._lib.ssx_create(ctypes.byref(self._c), ctypes.byref(gd), ctypes.c_void_p(s.cuda_stream))
        if rc != SSX_OK:
            raise SSXError(rc, "ssx_create failed")
        self.n_line = self.n_rec = None

    @classmethod
    def from_spec(cls, spec, stream=None):
        return cls(spec.nx, spec.nz, spec.h, spec.dt, spec.nt, spec.order, spec.n_sponge, stream)

    def _check(self, rc):
        if rc != SSX_OK:
            raise SSXError(rc, self._lib.ssx_last_error(self._c).decode())
        return rc

    def close(self):
        if self._c:
            self._lib.ssx_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup ------------------------------------------------------------
    def set_velocity_model(self, v: torch.Tensor, rho: float):
        p = _dev_ptr(v, (self.nz, self.nx), torch.float32, "v")
        self._check(self._lib.ssx_set_velocity_model(self._c, p, float(rho)))

    def set_geometry(self, z_s, ix_line0, n_line, z_r, ix_rec0, n_rec, x_s, dz_datum=0.1):
        g = GeomDesc(z_s, ix_line0, n_line, z_r, ix_rec0, n_rec, x_s, dz_datum)
        self._check(self._lib.ssx_set_geometry(self._c, ctypes.byref(g)))
        self.n_line, self.n_rec = n_line, n_rec

    @classmethod
    def for_problem(cls, spec, vel, stream=None):
        """Context with the workload's model and geometry set (vel: numpy or
        tensor [nz][nx], km/s)."""
        ctx = cls.from_spec(spec, stream)
        v = torch.as_tensor(np.asarray(vel), dtype=torch.float32).to(ctx.device).contiguous()
        ctx.set_velocity_model(v, spec.rho)
        ctx.set_geometry(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0,
                         spec.n_rec, spec.x_s, spec.dz_datum)
        return ctx

    # -- operators ----------------------------------------------------------
    def _line(self, t, name):
        return _dev_ptr(t, (self.nt, self.n_line), name=name)

    def _rec(self, t, name):
        return _dev_ptr(t, (self.nt, self.n_rec), name=name)

    def _empty(self, n):
        return torch.empty((self.nt, n), dtype=torch.float64, device=self.device)

    def forward(self, h, out=None):
        out = self._empty(self.n_rec) if out is None else out
        self._check(self._lib.ssx_forward(self._c, self._line(h, "h"), self._rec(out, "d")))
        return out

    def adjoint(self, d, out=None):
        out = self._empty(self.n_line) if out is None else out
        self._check(self._lib.ssx_adjoint(self._c, self._rec(d, "d"), self._line(out, "h")))
        return out

    def weight_apply(self, which, x, out=None):
        chk = self._rec if which == W_D else self._line
        out = self._empty(self.n_rec if which == W_D else self.n_line) if out is None else out
        self._check(self._lib.ssx_weight_apply(self._c, which, chk(x, "in"), chk(out, "out")))
        return out

    def lambda_apply(self, x, transpose=False, out=None):
        out = self._empty(self.n_line) if out is None else out
        self._check(self._lib.ssx_lambda_apply(self._c, 1 if transpose else 0, self._line(x, "in"),
                                               self._line(out, "out")))
        return out

    def time_reversal_inverse(self, d, out=None):
        out = self._empty(self.n_line) if out is None else out
        self._check(self._lib.ssx_time_reversal_inverse(self._c, self._rec(d, "d"),
                                                        self._line(out, "h")))
        return out

    def precond_apply(self, alpha, r, out=None):
        out = self._empty(self.n_line) if out is None else out
        self._check(self._lib.ssx_precond_apply(self._c, float(alpha), self._line(r, "r"),
                                                self._line(out, "g")))
        return out

    def normal_apply(self, mode, alpha, p, out=None):
        out = self._empty(self.n_line) if out is None else out
        self._check(self._lib.ssx_normal_apply(self._c, mode, float(alpha), self._line(p, "p"),
                                               self._line(out, "q")))
        return out

    def velocity_gradient(self, h, d, alpha=0.0, checkpoint_every=50, out=None, wait=True):
        """dPhi/dc of Phi = ||S[c] h - d||^2 + alpha ||A h||^2 at fixed h
        (ssx_velocity_gradient): returns (gradient [nz][nx] float64, Phi).
        wait=False returns (gradient, None) as soon as the work is queued
        (Phi later from last_objective())."""
        out = (torch.empty((self.nz, self.nx), dtype=torch.float64, device=self.device)
               if out is None else out)
        if out.dtype != torch.float64 or not out.is_contiguous() or tuple(out.shape) != (self.nz, self.nx):
            raise TypeError("gradient buffer must be contiguous float64 [nz][nx]")
        obj = ctypes.c_double(0.0)
        self._check(self._lib.ssx_velocity_gradient(self._c, self._line(h, "h"), self._rec(d, "d"),
                                                    float(alpha), int(checkpoint_every),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    ctypes.byref(obj) if wait else None))
        return out, (obj.value if wait else None)

    def last_objective(self):
        """Phi of the last velocity_gradient (synchronises)."""
        obj = ctypes.c_double(0.0)
        self._check(self._lib.ssx_last_objective(self._c, ctypes.byref(obj)))
        return obj.value

    def solve(self, d, alpha, maxit, rtol, mode=MODE_PCG, out=None, allow_not_converged=True,
              allow_breakdown=False):
        """Algorithm 1. Returns (h, residual history (numpy), iterations, status).
        SSX_ERR_NOT_CONVERGED is returned as a status unless allow_not_converged
        is False; SSX_ERR_BREAKDOWN and SSX_ERR_NONFINITE raise unless
        allow_breakdown is True (h then holds the last good iterate)."""
        out = self._empty(self.n_line) if out is None else out
        hist = (ctypes.c_double * (maxit + 1))()
        iters = ctypes.c_int(0)
        rc = self._lib.ssx_solve_source_subproblem(self._c, self._rec(d, "d"), float(alpha),
                                                   int(maxit), float(rtol), int(mode),
                                                   self._line(out, "h"), hist, ctypes.byref(iters))
        if rc != SSX_OK and not ((allow_not_converged and rc == 7) or
                                 (allow_breakdown and rc in (5, 6))):
            self._check(rc)
        k = iters.value
        return out, np.array(hist[: k + 1]), k, STATUS[rc]

    def point_source_data(self, x_d, z_d, wavelet, out=None):
        w = _dev_ptr(wavelet, (self.nt,), name="wavelet")
        out = self._empty(self.n_rec) if out is None else out
        self._check(self._lib.ssx_point_source_data(self._c, float(x_d), float(z_d), w,
                                                    self._rec(out, "d")))
        return out

    def set_sweep_mode(self, mode: int):
        self._check(self._lib.ssx_set_sweep_mode(self._c, int(mode)))

    def set_test_hook(self, hook: int, k: int = 0):
        """Failure injection of the next solve (ssx_set_test_hook)."""
        self._check(self._lib.ssx_set_test_hook(self._c, int(hook), int(k)))

    def set_tile_config(self, cfg: int):
        self._check(self._lib.ssx_set_tile_config(self._c, int(cfg)))

    # -- instrumentation ------------------------------------------------------
    def set_timing(self, on: bool):
        self._check(self._lib.ssx_set_timing(self._c, 1 if on else 0))

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.ssx_get_stats(self._c, ctypes.byref(st)))
        return st.as_dict()

    def reset_stats(self):
        self._check(self._lib.ssx_reset_stats(self._c))

    def phase_stats(self) -> list:
        """Per-phase breakdown of the timed sweeps (ssx_get_phase_stats)."""
        rows = []
        name = ctypes.create_string_buffer(64)
        sw, tl, cfg, ch = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms, steps = ctypes.c_double(), ctypes.c_longlong()
        while True:
            rc = self._lib.ssx_get_phase_stats(self._c, len(rows), name, 64, ctypes.byref(sw),
                                               ctypes.byref(tl), ctypes.byref(cfg), ctypes.byref(ch),
                                               ctypes.byref(ms), ctypes.byref(steps))
            if rc == ERR_ARG:
                return rows
            self._check(rc)
            rows.append({"phase": name.value.decode(), "sweeps": sw.value, "tiles": tl.value,
                         "tile_config": cfg.value, "chain": ch.value, "ms": ms.value,
                         "steps": steps.value})


def solve_batch(ctxs, ds, alphas, maxit, rtol, mode=MODE_PCG, outs=None):
    """Solve one source subproblem per context in shared launches
    (ssx_solve_batch). Returns (list of h, list of residual histories,
    iterations, status names)."""
    n = len(ctxs)
    lib = load_library()
    outs = [c._empty(c.n_line) for c in ctxs] if outs is None else outs
    cptr = (ctypes.c_void_p * n)(*[c._c.value for c in ctxs])
    dptr = (ctypes.c_void_p * n)(*[c._rec(d, "d").value for c, d in zip(ctxs, ds)])
    hptr = (ctypes.c_void_p * n)(*[c._line(h, "h").value for c, h in zip(ctxs, outs)])
    al = (ctypes.c_double * n)(*[float(a) for a in alphas])
    hist = (ctypes.c_double * (n * (maxit + 1)))()
    iters = (ctypes.c_int * n)()
    status = (ctypes.c_int * n)()
    rc = lib.ssx_solve_batch(cptr, n, dptr, al, int(maxit), float(rtol), int(mode), hptr, hist,
                             iters, status)
    if rc != SSX_OK:
        raise SSXError(rc, lib.ssx_last_error(ctxs[0]._c).decode())
    hs = [np.array(hist[i * (maxit + 1): i * (maxit + 1) + iters[i] + 1]) for i in range(n)]
    return outs, hs, list(iters), [STATUS[st] for st in status]


class Server:
    """Continuous-batching solve server (ssx_server_*): submit requests, call
    step() repeatedly, poll results. Tensors given to submit() are kept alive
    until the request is done."""

    def __init__(self, space_order=8, hbm_budget_bytes=80 * 10 ** 9, stream=None):
        self._lib = load_library()
        s = torch.cuda.current_stream() if stream is None else stream
        self._s = ctypes.c_void_p()
        rc = self._lib.ssx_server_create(ctypes.byref(self._s), int(space_order),
                                         int(hbm_budget_bytes), ctypes.c_void_p(s.cuda_stream))
        if rc != SSX_OK:
            raise SSXError(rc, "ssx_server_create failed")
        self._keep = {}

    def submit(self, spec, vel, d, out, alpha=None, maxit=None, rtol=None, mode=MODE_PCG):
        gd = GridDesc(spec.nx, spec.nz, spec.h, spec.dt, spec.nt, spec.order, spec.n_sponge)
        gm = GeomDesc(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                      spec.x_s, spec.dz_datum)
        v = _dev_ptr(vel, (spec.nz, spec.nx), torch.float32, "vel")
        dp = _dev_ptr(d, (spec.nt, spec.n_rec), name="d")
        hp = _dev_ptr(out, (spec.nt, spec.n_line), name="out")
        rid = ctypes.c_int(0)
        rc = self._lib.ssx_server_submit(self._s, ctypes.byref(gd), ctypes.byref(gm), v, spec.rho, dp,
                                         float(spec.alpha if alpha is None else alpha),
                                         int(spec.maxit if maxit is None else maxit),
                                         float(spec.rtol if rtol is None else rtol), int(mode), hp,
                                         ctypes.byref(rid))
        if rc != SSX_OK:
            raise SSXError(rc, self._lib.ssx_server_last_error(self._s).decode())
        self._keep[rid.value] = (vel, d, out)
        return rid.value

    def step(self):
        a, q = ctypes.c_int(0), ctypes.c_int(0)
        rc = self._lib.ssx_server_step(self._s, ctypes.byref(a), ctypes.byref(q))
        if rc != SSX_OK:
            raise SSXError(rc, self._lib.ssx_server_last_error(self._s).decode())
        return a.value, q.value

    def poll(self, rid):
        done, st, it = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        lat, wait = ctypes.c_double(0), ctypes.c_double(0)
        rc = self._lib.ssx_server_poll(self._s, int(rid), ctypes.byref(done), ctypes.byref(st),
                                       ctypes.byref(it), ctypes.byref(lat), ctypes.byref(wait))
        if rc != SSX_OK:
            raise SSXError(rc, "unknown request")
        if done.value:
            self._keep.pop(rid, None)
        return {"done": bool(done.value), "status": STATUS[st.value], "iters": it.value,
                "latency_ms": lat.value, "queue_ms": wait.value}

    def set_cache_budget(self, nbytes: int):
        """Working-set admission limit in bytes (0: off; default: 4x the L2 size)."""
        rc = self._lib.ssx_server_set_cache_budget(self._s, int(nbytes))
        if rc != SSX_OK:
            raise SSXError(rc, "ssx_server_set_cache_budget failed")

    def set_timing(self, on: bool):
        rc = self._lib.ssx_server_set_timing(self._s, 1 if on else 0)
        if rc != SSX_OK:
            raise SSXError(rc, self._lib.ssx_server_last_error(self._s).decode())

    def stats(self) -> dict:
        """The shared launches' counters (ssx_server_get_stats)."""
        st, r, rr = Stats(), ctypes.c_longlong(0), ctypes.c_longlong(0)
        rc = self._lib.ssx_server_get_stats(self._s, ctypes.byref(st), ctypes.byref(r), ctypes.byref(rr))
        if rc != SSX_OK:
            raise SSXError(rc, self._lib.ssx_server_last_error(self._s).decode())
        d = st.as_dict()
        d["rounds"], d["request_rounds"] = r.value, rr.value
        return d

    def close(self):
        if self._s:
            self._lib.ssx_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load_library().ssx_version().decode()
