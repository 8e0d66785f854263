"""The allocation-free entry point gbsp_crs_spmv_noalloc, called through the
C ABI, against the handle-based entry point on the same matrices.

It exists for callers that cannot allocate device memory: its scratch (the
tile table) lives in a static array inside the library.  This file is
collected last so that a run stopping at the first failure has run every
other test before it."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-14  # per-entry tolerance of the FP64 tests: |dy| <= 1e-14 * sum |a||x|


def _call(L, A, val, x, y, accumulate=0):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.gbsp_crs_spmv_noalloc(A.n_rows, A.n_cols, A.nnz, ctypes.c_void_p(A.rp.data_ptr()),
                                   ctypes.c_void_p(A.colt.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                   0 if val.dtype == torch.float64 else 1, accumulate,
                                   ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)


def test_noalloc_matches_handle_entry_point_two_calls():
    import paper_0910_4836_gb300 as g
    from paper_0910_4836_gb300 import CRSMatrix, _lib
    g.build()
    L = _lib.load()
    for call, A in enumerate([S.hh_like(300_000, 11), S.zipf_rows(200_000, 12, lmax=4000)]):
        A.rp = torch.as_tensor(A.row_ptr).cuda()
        A.colt = torch.as_tensor(A.col).cuda()
        val = torch.as_tensor(A.val).cuda()
        x = torch.as_tensor(S.vector(A.n_cols, 20 + call)).cuda()
        y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(L, A, val, x, y) == 0, L.gbsp_last_error()
        ref = CRSMatrix(A.rp, A.colt, val, A.n_cols).spmv(x)  # existing entry point
        torch.cuda.synchronize()
        s = O.crs_spmv_exact(A, S.vector(A.n_cols, 20 + call))[1]
        diff = np.abs(y.cpu().numpy() - ref.cpu().numpy())
        assert np.all(diff <= TOL64 * s), f"call {call}: max diff {diff.max()}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_0910_4836_gb300 import _lib
    L = _lib.load()
    fake = ctypes.c_void_p(4096)  # never dereferenced: the size check comes first
    st = L.gbsp_crs_spmv_noalloc(1, 1, 2_000_000_000, fake, fake, fake, 0, 0, fake, ctypes.c_void_p(8192),
                                 None)
    assert st == -1
    assert b"static scratch" in L.gbsp_last_error()
