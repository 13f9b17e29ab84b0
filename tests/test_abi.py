"""The C-ABI library builds, loads and exports every symbol include/ssx.h
declares; the binding rejects bad arguments before any device work. CPU only:
no call here touches a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    text = open(os.path.join(ROOT, "include", "ssx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssx_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_16573_gb300 import build, ssx
    build.build()
    return ssx.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2203_16573_gb300 import ssx
    syms = _header_symbols()
    assert len(syms) >= 16
    assert sorted(ssx.EXPORTS) == syms
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_constants_match_the_header():
    from paper_2203_16573_gb300 import ssx
    text = open(os.path.join(ROOT, "include", "ssx.h")).read()
    n = int(re.search(r"#define SSX_NUM_TILE_CONFIGS (\d+)", text).group(1))
    assert ssx.N_TILE_CONFIGS == n
    src = open(os.path.join(ROOT, "paper_2203_16573_gb300", "csrc", "ssx_internal.cuh")).read()
    assert re.search(r"constexpr int kNumTileCfgs = (\d+);", src).group(1) == str(n)
    nm = int(re.search(r"#define SSX_NUM_MARCH_CONFIGS (\d+)", text).group(1))
    assert ssx.N_MARCH_CONFIGS == nm
    assert re.search(r"constexpr int kNumMarchCfgs = (\d+);", src).group(1) == str(nm)
    n2 = int(re.search(r"#define SSX_NUM_TWO_CONFIGS (\d+)", text).group(1))
    assert ssx.N_TWO_CONFIGS == n2
    assert re.search(r"constexpr int kNumTwoCfgs = (\d+);", src).group(1) == str(n2)


def test_version_string(lib):
    assert b"sm_103a" in lib.ssx_version()


def test_create_rejects_bad_descriptor_without_touching_the_device(lib):
    from paper_2203_16573_gb300 import ssx
    out = ctypes.c_void_p()
    for bad in [ssx.GridDesc(4, 100, 0.01, 1e-3, 10, 4, 5),      # nx too small
                ssx.GridDesc(100, 100, 0.01, 1e-3, 10, 5, 5),    # odd order
                ssx.GridDesc(100, 100, 0.01, 1e-3, 10, 10, 5),   # order > 8
                ssx.GridDesc(100, 100, -0.01, 1e-3, 10, 4, 5),   # h <= 0
                ssx.GridDesc(100, 100, 0.01, 1e-3, 0, 4, 5),     # nt = 0
                ssx.GridDesc(100, 100, 0.01, 1e-3, 10, 4, -1)]:  # sponge < 0
        assert lib.ssx_create(ctypes.byref(out), ctypes.byref(bad), None) == 1
        assert not out.value
    assert lib.ssx_create(None, None, None) == 1
    assert lib.ssx_destroy(None) == 1
    assert lib.ssx_last_error(None) == b"null context"


def test_oracle_shares_no_code_with_the_library():
    """The oracle and the CUDA path are independent: no file of one includes,
    imports or loads the other."""
    csrc = os.path.join(ROOT, "paper_2203_16573_gb300", "csrc")
    for f in os.listdir(csrc):
        t = open(os.path.join(csrc, f)).read()
        assert "oracle" not in t.lower(), f
    for f in ("ssx.py", "build.py", "__init__.py", "workloads.py"):
        t = open(os.path.join(ROOT, "paper_2203_16573_gb300", f)).read()
        assert "import oracle" not in t and "from oracle" not in t, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            t = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_2203_16573_gb300" not in t and "libssx.so" not in t, f


def test_every_entry_point_rejects_a_null_handle_without_touching_the_device(lib):
    """Each call on a context or server, and each call with only null
    buffers, returns SSX_ERR_ARG (1) before any CUDA work: the checks of the
    boundary's error behaviour that need no GPU."""
    import ctypes as C
    skip = {"ssx_version", "ssx_last_error", "ssx_server_last_error"}
    from paper_2203_16573_gb300 import ssx
    checked = []
    for name in ssx.EXPORTS:
        if name in skip:
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes:
            if t in (C.c_int, C.c_size_t):
                args.append(0)
            elif t is C.c_double:
                args.append(0.0)
            else:
                args.append(None)       # null handle, descriptor or buffer
        assert fn(*args) == 1, name
        checked.append(name)
    assert len(checked) == len(ssx.EXPORTS) - len(skip)
    assert lib.ssx_last_error(None) == b"null context"
    assert lib.ssx_server_last_error(None) == b"null server"


def test_bench_kernel_names_match_the_configuration_tables():
    """bench.py names each phase's kernel from its configuration id: its
    tables of shapes must be the library's."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_2203_16573_gb300", "csrc", "ssx_internal.cuh")).read()
    tile = re.findall(r"X\((\d+), (\d+), (\d+), (\d+), ([01])\)", src)
    march = re.findall(r"X\((\d+), (\d+), (\d+)\)\s", src)
    two = re.findall(r"X\((\d+), (\d+), (\d+), (\d+)\)\s", src)
    n = len(tile)
    assert n == 14 and len(march) == 4 and len(two) == 3
    for cid, tx, tz, nt, quads in tile:
        name = f"{tx}x{tz}/{nt}" + (" quads" if quads == "1" else "")
        assert bench._kernel_name(int(cid)) == f"k_multi {name}"
        assert bench._kernel_name(int(cid) + n) == f"k_multi_tma {name}"
    for cid, tx, tz in march:
        assert bench._kernel_name(int(cid) + 2 * n) == f"k_march {tx}x{tz}"
    for cid, tx, tz, nt in two:
        assert bench._kernel_name(int(cid) + 2 * n + len(march)) == f"k_two {tx}x{tz}/{nt}"
