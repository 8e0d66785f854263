"""Hybrid storage on the GPU (dense secondary diagonals in DIA form plus a
remainder): selection, arrays and products against the oracle."""
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


def planted(n=3000):
    rows, cols = [], []
    for k, o in enumerate((-50, 7, 123, 2999)):
        i = np.arange(max(0, -o), min(n, n - o))
        keep = S.uniform01(6, 40 + k, i) < 0.9
        rows += list(i[keep])
        cols += list(i[keep] + o)
    i = np.arange(n)
    rows += list(i) + list(i[:100])
    cols += list(S.randint(6, 50, i, 0, n - 1)) + list(i[:100] + 7)  # duplicates on offset 7
    vals = S.uniform(6, 51, np.arange(len(rows)), -1, 1)
    return S.from_coo(n, n, rows, cols, vals, dedupe=False)


MATS = [
    ("laplace", lambda: S.laplace2d(64, 64), 16, 0.5),
    ("hh_diagonals_300k", lambda: S.hh_diagonals(300_000, 5), 16, 2.0 / 3.0),
    ("hh_like_100k", lambda: S.hh_like(100_000, 3), 16, 2.0 / 3.0),
    ("planted_dups", planted, 8, 0.7),
    ("rect_none", lambda: S.small_random(500, 300, 7, density=0.02), 8, 1.01),
    ("empty", lambda: S.CRS(4, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty"), 8, 0.5),
]


@pytest.mark.parametrize("name,make,max_diags,min_fill", MATS, ids=[m[0] for m in MATS])
def test_hybrid_against_oracle(name, make, max_diags, min_fill):
    from paper_0910_4836_gb300 import HybridMatrix
    A = make()
    M = crs(A)
    offs = O.dia_select(A, max_diags, min_fill)
    dia_o, rem_o = O.dia_build(A, offs)
    x = S.vector(A.n_cols, 61)
    ref, s = O.crs_spmv_exact(A, x)
    y0 = S.vector(A.n_rows, 62)
    for remainder in ("CRS", "SELL"):
        H = HybridMatrix(M, max_diags, min_fill, remainder=remainder, window=128, unroll=4)
        assert H.offsets_host == list(offs), name
        assert H.nnz_rem == rem_o.nnz and H.nnz_dia == A.nnz - rem_o.nnz
        if len(offs):
            assert np.array_equal(host(H.dia).view(np.int64), dia_o.view(np.int64))
        assert np.array_equal(host(H.remainder.row_ptr), rem_o.row_ptr)
        assert np.array_equal(host(H.remainder.col), rem_o.col)
        assert np.array_equal(host(H.remainder.val).view(np.int64), rem_o.val.view(np.int64))
        y = host(H.spmv(dev(x)))
        assert_close64(y, ref, s, f"{name} {remainder}")
        assert_close64(y, O.dia_spmv(offs, dia_o, rem_o, x), s, f"{name} {remainder} vs oracle hybrid loop")
        out = dev(y0)
        H.spmv(dev(x), out=out, accumulate=True)
        assert_close64(host(out) - y0, ref, s + np.abs(y0), f"{name} {remainder} accumulate")


def test_hybrid_integer_exact():
    from paper_0910_4836_gb300 import HybridMatrix
    A = S.integer_values(S.hh_diagonals(200_000, 8), 9, 1000)
    xi = S.int_vector(A.n_cols, 10, 1000)
    for remainder in ("CRS", "SELL"):
        H = HybridMatrix(crs(A), 16, 2.0 / 3.0, remainder=remainder)
        assert len(H.offsets_host) == 7  # main diagonal + 3 outer offsets and their mirrors below n
        assert np.array_equal(host(H.spmv(dev(xi))), O.crs_spmv(A, xi))


def test_hybrid_rejections():
    from paper_0910_4836_gb300 import GbspError, HybridMatrix
    M = crs(S.laplace2d(16, 16))
    with pytest.raises(GbspError):
        HybridMatrix(M, 65, 0.5)
    H = HybridMatrix(M, 8, 0.5)
    with pytest.raises(GbspError):
        H.dia_part.spmm(dev(np.ones((256, 2))))
    with pytest.raises(GbspError):
        H.dia_part.spmv(dev(np.ones(256)), transpose=True)


def test_hybrid_fp32_compensated_within_dot2_bound():
    """FP32 values with compensated row sums through DIA + remainder: within
    the Dot2 bound of the exact product of the FP32-rounded data."""
    from gpu_util import dot2_bound
    from paper_0910_4836_gb300 import HybridMatrix
    A = S.hh_diagonals(200_000, 12)
    A32 = A.astype(np.float32)
    x32 = S.vector(A.n_cols, 13).astype(np.float32)
    ref, s = O.crs_spmv_exact(A32.astype(np.float64), x32.astype(np.float64))
    M = crs(A, torch.float32)
    M.set_kernel("vector", compensated=True)
    for remainder in ("CRS", "SELL"):
        H = HybridMatrix(M, 16, 2.0 / 3.0, remainder=remainder)
        y = host(H.spmv(dev(x32))).astype(np.float64)
        lens = np.diff(A.row_ptr.astype(np.int64))
        # the DIA sum is rounded to FP32 once before the remainder is added
        bound = dot2_bound(ref, s, lens) + 2.0 ** -24 * s
        assert np.all(np.abs(y - ref) <= bound), remainder
