"""The C ABI library builds for sm_103a, loads, and exports every entry point
include/gbspmv.h declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbspmv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbsp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_0910_4836_gb300 as g
    path = g.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("gbsp_crs_create", "gbsp_jds_plan", "gbsp_jds_build", "gbsp_spmv", "gbsp_spmm",
                 "gbsp_transpose_build", "gbsp_dval", "gbsp_batch_run", "gbsp_autotune"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_the_header():
    from paper_0910_4836_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_built_for_sm103a():
    from paper_0910_4836_gb300 import buildlib as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)


def test_host_side_checks_without_gpu():
    from paper_0910_4836_gb300 import _lib
    L = _lib.load()
    assert L.gbsp_status_string(-2) == b"GBSP_ERR_MATRIX"
    assert L.gbsp_version() >= 10000
    h = ctypes.c_void_p()
    # negative size, NULL row_ptr, bad dtype: rejected before any device work
    assert L.gbsp_crs_create(-1, 4, 0, None, None, None, 0, ctypes.byref(h)) == -1
    assert L.gbsp_crs_create(4, 4, 0, None, None, None, 0, ctypes.byref(h)) == -1
    assert L.gbsp_crs_create(4, 4, 0, ctypes.c_void_p(256), None, None, 7, ctypes.byref(h)) == -1
    assert b"dtype" in L.gbsp_last_error()
    # the largest nnz the int32 index arrays admit is 2^31 - 2^16 - 1
    p = ctypes.c_void_p(256)
    assert L.gbsp_crs_create(4, 4, 2 ** 31 - 2 ** 16, p, p, p, 0, ctypes.byref(h)) == -1
    assert b"int32" in L.gbsp_last_error()
    assert L.gbsp_crs_create(2 ** 31 - 1, 4, 0, p, None, None, 0, ctypes.byref(h)) == -1
    assert L.gbsp_spmv(None, 0, 0, 0, None, None, None) == -1
    assert L.gbsp_destroy(None) == 0


def test_kernel_option_checks_without_gpu():
    """gbsp_set_kernel's checks are host logic: a handle over placeholder
    device addresses (never dereferenced on the host) takes every VECTOR and
    RUNS shape the header admits and refuses the rest, and a RUNS request
    without a shape gets RUNS's own default, not a VECTOR leftover."""
    from paper_0910_4836_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    p = ctypes.c_void_p(256)
    assert L.gbsp_crs_create(64, 64, 0, p, None, None, 0, ctypes.byref(h)) == 0
    try:
        def opts(kernel, lanes=0, rows=0):
            return _lib.KernelOpts(_lib.KERNELS[kernel], lanes, rows, 0, 0, 0)

        def get():
            o = _lib.KernelOpts()
            assert L.gbsp_get_kernel(h, ctypes.byref(o)) == 0
            return o.kernel, o.lanes, o.rows_per_warp
        for lanes in (1, 2, 4, 8, 16, 32):
            for rows in (1, 2, 4):
                assert L.gbsp_set_kernel(h, ctypes.byref(opts("vector", lanes, rows))) == 0
                assert get() == (1, lanes, rows)
        for lanes, rows in ((1, 4), (1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 8)):
            assert L.gbsp_set_kernel(h, ctypes.byref(opts("runs", lanes, rows))) == 0
            assert get() == (3, lanes, rows)
        for lanes, rows in ((16, 8), (32, 8), (8, 4), (4, 2), (2, 1), (3, 4)):
            assert L.gbsp_set_kernel(h, ctypes.byref(opts("runs", lanes, rows))) == -1, (lanes, rows)
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("vector", 4, 8))) == -1  # a RUNS shape only
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("vector", 3, 4))) == -1
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("tiled"))) == -1        # no tile table prepared
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("vector", 16, 2))) == 0
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("runs"))) == 0
        assert get() == (3, 4, 4)
        assert L.gbsp_set_kernel(h, ctypes.byref(opts("runs", 8))) == 0
        assert get() == (3, 8, 8)
        bad = _lib.KernelOpts(4, 0, 0, 0, 0, 0)                                 # no such kernel
        assert L.gbsp_set_kernel(h, ctypes.byref(bad)) == -1
    finally:
        assert L.gbsp_destroy(h) == 0


def test_oracle_shares_no_code_with_the_library():
    """The oracle is independent: no include, import or link either way."""
    csrc = os.path.join(ROOT, "paper_0910_4836_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", src, flags=re.M)
                assert "oracle.c" not in src
    osrc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "gbspmv" not in osrc
    opy = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_0910_4836_gb300" not in opy
