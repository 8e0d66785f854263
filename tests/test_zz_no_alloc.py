"""The allocation-free entry point gbsp_crs_spmv_noalloc, called through the
C ABI, against the oracle and against the handle-based entry point on the
same matrices.

It exists for callers that cannot allocate device memory: its scratch (the
tile table) lives in a static array inside the library.  This file is
collected last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import dot2_bound
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-14  # per-entry tolerance of the FP64 tests: |dy| <= 1e-14 * sum |a||x|


def _dev(A, dtype):
    rp = torch.as_tensor(A.row_ptr).cuda()
    col = torch.as_tensor(A.col).cuda() if A.nnz else torch.zeros(4, dtype=torch.int32, device="cuda")
    val = (torch.as_tensor(A.val).to(dtype).cuda() if A.nnz
           else torch.zeros(4, dtype=dtype, device="cuda"))
    return rp, col, val


def _call(L, A, rp, col, val, x, y, accumulate=0):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.gbsp_crs_spmv_noalloc(A.n_rows, A.n_cols, A.nnz, ctypes.c_void_p(rp.data_ptr()),
                                   ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                   0 if val.dtype == torch.float64 else 1, accumulate,
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)


def _lib():
    import paper_0910_4836_gb300 as g
    from paper_0910_4836_gb300 import _lib
    g.build()
    return _lib.load()


def _edge_matrices():
    """A single row longer than the 1024-entry tile, rows of 63 and 64
    entries around it, and rows with no entries."""
    rows, cols = [], []
    for i, n in enumerate([63, 64, 0, 2500, 65, 1, 0, 1023, 1025]):
        rows += [i] * n
        cols += list(range(n))
    A = S.from_coo(9, 3000, rows, cols, S.uniform(41, 1, np.arange(len(rows)), -1, 1), name="tile_edges")
    one_long = S.from_coo(1, 5000, [0] * 4000, np.arange(4000), S.uniform(42, 1, np.arange(4000), -1, 1),
                          name="one_row_4000")
    return [A, one_long]


def test_noalloc_matches_oracle_and_handle_entry_point_two_calls():
    from paper_0910_4836_gb300 import CRSMatrix
    L = _lib()
    mats = [S.hh_like(300_000, 11), S.zipf_rows(200_000, 12, lmax=4000)] + _edge_matrices()
    for call, A in enumerate(mats):
        rp, col, val = _dev(A, torch.float64)
        xh = S.vector(A.n_cols, 20 + call)
        x = torch.as_tensor(xh).cuda()
        ref, s = O.crs_spmv_exact(A, xh)
        # two calls in a row on the same output: the second must not see the first's table
        for rep in range(2):
            y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
            assert _call(L, A, rp, col, val, x, y) == 0, L.gbsp_last_error()
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            err = np.abs(got - ref)
            assert np.all(err <= TOL64 * s), f"{A.name} call {rep}: max err vs oracle {err.max()}"
        handle = CRSMatrix(rp, col, val, A.n_cols).spmv(x)  # the existing entry point
        torch.cuda.synchronize()
        diff = np.abs(got - handle.cpu().numpy())
        assert np.all(diff <= TOL64 * s), f"{A.name}: max diff vs handle path {diff.max()}"


def test_noalloc_accumulate_and_fp32():
    L = _lib()
    A = S.hh_like(200_000, 13)
    xh = S.vector(A.n_cols, 31)
    # accumulate = 1 from a known y: y0 + A x
    rp, col, val = _dev(A, torch.float64)
    y0 = S.vector(A.n_rows, 32)
    y = torch.as_tensor(y0).cuda()
    for rep in range(2):
        y.copy_(torch.as_tensor(y0))
        assert _call(L, A, rp, col, val, torch.as_tensor(xh).cuda(), y, accumulate=1) == 0, L.gbsp_last_error()
        torch.cuda.synchronize()
        ref, s = O.crs_spmv_exact(A, xh, y=y0, accumulate=True)
        err = np.abs(y.cpu().numpy() - ref)
        assert np.all(err <= TOL64 * (s + np.abs(y0))), f"accumulate call {rep}: max err {err.max()}"
    # FP32 values and vector, compensated sums: the Dot2 bound against the
    # exact product of the FP32-rounded data
    rp, col, val32 = _dev(A, torch.float32)
    x32 = xh.astype(np.float32)
    A64 = S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64), "r32")
    ref, s = O.crs_spmv_exact(A64, x32.astype(np.float64))
    bound = dot2_bound(ref, s, np.diff(A.row_ptr))
    for rep in range(2):
        y = torch.full((A.n_rows,), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(L, A, rp, col, val32, torch.as_tensor(x32).cuda(), y) == 0, L.gbsp_last_error()
        torch.cuda.synchronize()
        err = np.abs(y.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= bound), f"FP32 call {rep}: max err {err.max()}"


def test_noalloc_empty_matrix():
    L = _lib()
    A = S.CRS(5, 3, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty_5x3")
    rp, col, val = _dev(A, torch.float64)
    x = torch.ones(3, dtype=torch.float64, device="cuda")
    y = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(L, A, rp, col, val, x, y) == 0, L.gbsp_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), np.zeros(5))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = _lib()
    fake = ctypes.c_void_p(4096)  # never dereferenced: the size check comes first
    st = L.gbsp_crs_spmv_noalloc(1, 1, 2_000_000_000, fake, fake, fake, 0, 0, fake, ctypes.c_void_p(8192),
                                 None)
    assert st == -1
    assert b"static scratch" in L.gbsp_last_error()
