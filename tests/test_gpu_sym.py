"""Symmetric SpMVM from the upper triangle on the GPU against the oracle.
The GPU scatters with FP64 atomics, so it is compared within the tolerance
(every row here has fewer than 60 terms, so any summation order stays
inside 1e-14 sum|a||x|) and exactly on integer data."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import assert_close64, crs, dev, host
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


def symmetric_random(n, seed, density):
    B = S.small_random(n, n, seed, density=density)
    D = B.to_dense()
    D = D + D.T
    r, c = np.nonzero(D)
    return S.from_coo(n, n, r, c, D[r, c])


MATS = [
    ("laplace", lambda: S.laplace2d(64, 64)),
    ("hh_like_100k", lambda: S.hh_like(100_000, 31)),
    ("stencil27_sym", lambda: S.stencil27(20, 4, symmetric_values=True)),
    ("random_sym", lambda: symmetric_random(700, 32, 0.02)),
    ("one", lambda: S.from_coo(1, 1, [0], [0], [2.5])),
    ("empty_rows", lambda: S.from_coo(5, 5, [1, 3], [3, 1], [1.0, 1.0])),
]


@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_upper_and_symmetric_products(name, make):
    A = make()
    M = crs(A)
    Uo = O.upper(A)
    U = M.upper()
    assert U.nnz == Uo.nnz
    assert np.array_equal(host(U.row_ptr), Uo.row_ptr)
    assert np.array_equal(host(U.col), Uo.col)
    assert np.array_equal(host(U.val).view(np.int64), Uo.val.view(np.int64))
    x = S.vector(A.n_rows, 33)
    ref, s = O.crs_spmv_exact(A, x)
    handles = [("crs", U)]
    for w, u in ((32, 2), (128, 4), (1024, 4)):
        handles.append((f"sell w={w} u={u}", U.to_jds("SELL", "row_only", window=w, unroll=u)))
    y0 = S.vector(A.n_rows, 34)
    for hname, H in handles:
        y = host(H.spmv_symmetric(dev(x)))
        assert_close64(y, ref, s, f"{name} {hname}")
        assert_close64(y, O.sym_spmv(Uo, x), s, f"{name} {hname} vs oracle loop")
        out = dev(y0)
        H.spmv_symmetric(dev(x), out=out, accumulate=True)
        assert_close64(host(out) - y0, ref, s + np.abs(y0), f"{name} {hname} accumulate")


def test_symmetric_integer_exact():
    A = S.hh_like(60_000, 35)
    D_vals = S.integer_values(A, 36, 1000).val
    # symmetric integer values: value of (i, j) from the upper copy
    rows = A.row_ids()
    key_lo = np.minimum(rows, A.col).astype(np.int64) * A.n_rows + np.maximum(rows, A.col)
    order = np.argsort(key_lo, kind="stable")
    first = np.ones(len(order), bool)
    first[1:] = key_lo[order][1:] != key_lo[order][:-1]
    grp = np.cumsum(first) - 1
    vals_sorted = D_vals[order][first][grp]
    vals = np.empty_like(D_vals)
    vals[order] = vals_sorted
    Ai = S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col, vals)
    xi = S.int_vector(A.n_rows, 37, 1000)
    ref = O.crs_spmv(Ai, xi)
    U = crs(Ai).upper()
    for H in (U, U.to_jds("SELL", "row_only", window=128, unroll=4)):
        assert np.array_equal(host(H.spmv_symmetric(dev(xi))), ref)


def test_symmetric_rejections():
    from paper_0910_4836_gb300 import GbspError
    A = S.laplace2d(16, 16)
    U = crs(A).upper()
    with pytest.raises(GbspError):
        U.to_jds("SELL", "symmetric", window=64).spmv_symmetric(dev(S.vector(A.n_rows, 1)))
    with pytest.raises(GbspError):
        U.to_jds("NUJDS", "row_only").spmv_symmetric(dev(S.vector(A.n_rows, 1)))
    U32 = crs(A, torch.float32).upper()
    with pytest.raises(GbspError):
        U32.spmv_symmetric(dev(S.vector(A.n_rows, 1).astype(np.float32)))
    with pytest.raises(GbspError):
        crs(S.small_random(10, 12, 3, density=0.3)).upper()
