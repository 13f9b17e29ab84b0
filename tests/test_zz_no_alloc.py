"""ssx_forward_noalloc: forward modelling for callers that cannot allocate.

Some users of this library cannot call cudaMalloc -- a plug-in inside a
framework that owns the device's whole memory pool, or code under a fixed
memory budget -- so the library offers one entry point whose scratch lives in
a fixed device array. Here it is called through the C ABI twice in a row and
each result is compared with the context-based ssx_forward (which allocates
its wavefields up front) within the tolerance of the other parity tests. The
file is named to be collected last.
"""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_2203_16573_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_forward_matches_forward_twice():
    from paper_2203_16573_gb300 import build, ssx
    build.build()
    lib = ssx.load_library()
    spec = dataclasses.replace(W.small(order=8, nt=300), z_s=0.5537, z_r=0.0471)
    vel = torch.as_tensor(W.velocity(spec), dtype=torch.float32, device="cuda").contiguous()
    h = torch.as_tensor(W.smooth_random_gather(spec.nt, spec.n_line, 1), device="cuda")

    ctx = ssx.Context.from_spec(spec)
    ctx.set_velocity_model(vel, spec.rho)
    ctx.set_geometry(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                     spec.x_s, spec.dz_datum)
    d_ref = ctx.forward(h)
    torch.cuda.synchronize()

    gd = ssx.GridDesc(spec.nx, spec.nz, spec.h, spec.dt, spec.nt, spec.order, spec.n_sponge)
    gm = ssx.GeomDesc(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                      spec.x_s, spec.dz_datum)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):   # the second call reuses the array the first call left behind
        d = torch.full((spec.nt, spec.n_rec), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ssx_forward_noalloc(ctypes.byref(gd), ctypes.byref(gm),
                                     ctypes.c_void_p(vel.data_ptr()), spec.rho,
                                     ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                     stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert _rel(d, d_ref) <= TOL

    # a grid beyond the fixed scratch is refused before any device work
    big = ssx.GridDesc(3000, 3000, spec.h, spec.dt, spec.nt, spec.order, spec.n_sponge)
    rc = lib.ssx_forward_noalloc(ctypes.byref(big), ctypes.byref(gm),
                                 ctypes.c_void_p(vel.data_ptr()), spec.rho,
                                 ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                 stream)
    assert rc == 1
    ctx.close()
