"""ssx_forward_noalloc: forward modelling for callers that cannot allocate.

Some users of this library cannot call cudaMalloc -- a plug-in inside a
framework that owns the device's whole memory pool, or code under a fixed
memory budget -- so the library offers one entry point whose scratch lives in
a fixed device array. Here it is called through the C ABI twice in a row and
each result is compared with the context-based ssx_forward (which allocates
its wavefields up front): the two run the same tile arithmetic on the same
coefficients, so the results must be identical bit for bit. A second case
makes the very first library call of a fresh process a no-allocation call
(no context exists yet, so the module and its array are first used there).
The file is named to be collected last.
"""
import ctypes
import dataclasses
import os
import subprocess
import sys

import pytest
import torch

from paper_2203_16573_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _spec():
    return dataclasses.replace(W.small(order=8, nt=300), z_s=0.5537, z_r=0.0471)


def _noalloc(lib, ssx, spec, vel, h, d, nx=None):
    gd = ssx.GridDesc(spec.nx if nx is None else nx, spec.nz, spec.h, spec.dt, spec.nt,
                      spec.order, spec.n_sponge)
    gm = ssx.GeomDesc(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                      spec.x_s, spec.dz_datum)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ssx_forward_noalloc(ctypes.byref(gd), ctypes.byref(gm),
                                   ctypes.c_void_p(vel.data_ptr()), spec.rho,
                                   ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                   stream)


def test_noalloc_forward_matches_forward_twice():
    from paper_2203_16573_gb300 import build, ssx
    build.build()
    lib = ssx.load_library()
    spec = _spec()
    vel = torch.as_tensor(W.velocity(spec), dtype=torch.float32, device="cuda").contiguous()
    h = torch.as_tensor(W.smooth_random_gather(spec.nt, spec.n_line, 1), device="cuda")

    ctx = ssx.Context.from_spec(spec)
    ctx.set_velocity_model(vel, spec.rho)
    ctx.set_geometry(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                     spec.x_s, spec.dz_datum)
    d_ref = ctx.forward(h)
    torch.cuda.synchronize()
    assert float(d_ref.abs().max()) > 0

    for _ in range(2):   # the second call reuses the array the first call left behind
        d = torch.full((spec.nt, spec.n_rec), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, ssx, spec, vel, h, d) == 0
        torch.cuda.synchronize()
        assert torch.equal(d, d_ref)

    # grids beyond the fixed scratch are refused before any device work,
    # including a width whose padded size would overflow an int
    for nx in (3000, 2 ** 31 - 8):
        big = dataclasses.replace(spec, nz=3000) if nx == 3000 else spec
        assert _noalloc(lib, ssx, big, vel, h, d, nx=nx) == 1
    ctx.close()


_FRESH = r"""
import ctypes, dataclasses, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2203_16573_gb300 import ssx, workloads as W
lib = ssx.load_library()
spec = dataclasses.replace(W.small(order=8, nt=300), z_s=0.5537, z_r=0.0471)
torch.cuda.set_device(0)
vel = torch.as_tensor(W.velocity(spec), dtype=torch.float32, device="cuda").contiguous()
h = torch.as_tensor(W.smooth_random_gather(spec.nt, spec.n_line, 1), device="cuda")
gd = ssx.GridDesc(spec.nx, spec.nz, spec.h, spec.dt, spec.nt, spec.order, spec.n_sponge)
gm = ssx.GeomDesc(spec.z_s, spec.ix_line0, spec.n_line, spec.z_r, spec.ix_rec0, spec.n_rec,
                  spec.x_s, spec.dz_datum)
d = torch.full((spec.nt, spec.n_rec), float("nan"), dtype=torch.float64, device="cuda")
stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
rc = lib.ssx_forward_noalloc(ctypes.byref(gd), ctypes.byref(gm), ctypes.c_void_p(vel.data_ptr()),
                             spec.rho, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                             stream)
torch.cuda.synchronize()
assert rc == 0, rc
ctx = ssx.Context.for_problem(spec, W.velocity(spec))   # the first context comes afterwards
ref = ctx.forward(h)
torch.cuda.synchronize()
assert torch.equal(d, ref)
print("FRESH_OK")
"""


def test_noalloc_first_call_of_a_fresh_process():
    from paper_2203_16573_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "FRESH_OK" in r.stdout, r.stdout + r.stderr
