"""Size limits on the GPU: the largest matrix the int32 index arrays admit,
and a windowed SELL sort whose (window, length) key does not fit 32 bits.

The index-limit matrix has nnz = 2^31 - 2^16 - 1 entries (25.8 GB in FP64
CRS) with integer values, so every product is exact in any summation
order: the formats must agree bit for bit on every row, sampled rows must
equal the oracle's CRS loop, and the adjoint must satisfy <A^T g, x> =
<g, A x> exactly."""
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


@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_sell_window_key_wider_than_32_bits(perm):
    """2^20 + 100 rows and a row of 140,001 entries: at windows of 32 and 64
    rows the (window, length) sort key needs 34 and 33 bits, so the build
    sorts in two stable stages; at 256 rows it fits (31 bits).  Arrays are
    bit-exact against the oracle's builder either way."""
    A = S.long_rows(2 ** 20 + 100, [140_001, 70_001], 5)
    M = crs(A)
    x = S.vector(A.n_cols, 91)
    ref, s = O.crs_spmv_exact(A, x)
    sym = perm == "symmetric"
    for fmt, window in (("SELL", 32), ("SELL", 64), ("SELL", 256), ("PSELL", 64), ("PSELL", 256)):
        Os = (O.sell_build if fmt == "SELL" else O.psell_build)(A, window, symmetric=sym)
        G = M.to_jds(fmt, perm, window=window, unroll=4)
        assert np.array_equal(host(G.perm), Os.perm), (fmt, window)
        assert np.array_equal(host(G.rlen), Os.rlen), (fmt, window)
        assert np.array_equal(host(G.blk_ptr), Os.blk_ptr), (fmt, window)
        assert np.array_equal(host(G.col), Os.col), (fmt, window)
        assert np.array_equal(host(G.val).view(np.int64), Os.val.view(np.int64)), (fmt, window)
        assert_close64(host(G.spmv_original(dev(x))), ref, s, f"{fmt} w={window}")
        del G


def _limit_matrix():
    """The index-limit CRS built on the device from the closed-form rows."""
    N = S.LIMIT_ROWS
    i = torch.arange(N, device="cuda", dtype=torch.int64)
    lens = S.limit_lengths(i)
    rp = torch.zeros(N + 1, dtype=torch.int64, device="cuda")
    torch.cumsum(lens, 0, out=rp[1:])
    assert int(rp[-1]) == S.LIMIT_NNZ
    col = torch.empty(S.LIMIT_NNZ, dtype=torch.int32, device="cuda")
    val = torch.empty(S.LIMIT_NNZ, dtype=torch.float64, device="cuda")
    step = 2 ** 20
    for r0 in range(0, N, step):
        r1 = min(r0 + step, N)
        k0, k1 = int(rp[r0]), int(rp[r1])
        rows = torch.repeat_interleave(i[r0:r1], lens[r0:r1])
        j = torch.arange(k0, k1, device="cuda", dtype=torch.int64) - rp[rows]
        col[k0:k1] = S.limit_cols(rows, j).to(torch.int32)
        val[k0:k1] = S.limit_vals(rows, j).to(torch.float64)
        del rows, j
    from paper_0910_4836_gb300 import CRSMatrix
    return CRSMatrix(rp.to(torch.int32), col, val, N), i


def test_index_limit_matrix_all_formats():
    props = torch.cuda.get_device_properties(0)
    if props.total_memory < 150 * 2 ** 30:
        pytest.skip("needs about 100 GB of device memory")
    M, i = _limit_matrix()
    assert M.nnz == S.LIMIT_NNZ and M.validate() == 0
    x = S.limit_x(i).to(torch.float64)
    y = M.spmv(x)
    # sampled rows, the ends of the index range among them, against the oracle
    N = S.LIMIT_ROWS
    rows = np.unique(np.concatenate([[0, 1, 2 ** 16, 2 ** 16 + 1, N // 2, N - 2, N - 1],
                                     S.randint(9, 1, np.arange(2000), 0, N - 1)]))
    sub = S.limit_rows_crs(rows)
    ref = O.crs_spmv(sub, S.limit_x(np.arange(N, dtype=np.int64)).astype(np.float64))
    assert np.array_equal(host(y[torch.as_tensor(rows, device="cuda")]), ref)
    # every other format, every row, bit for bit
    M.prepare_tiled(2048)
    assert torch.equal(M.spmv(x), y), "CRS tiled"
    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    assert torch.equal(M.spmv(x), y), "CRS vector 4x4"
    # rows of 8..248 entries: most warps take the runs kernel's cut-out step
    for l, r in ((4, 4), (2, 8)):
        M.set_kernel("runs", lanes=l, rows_per_warp=r)
        assert torch.equal(M.spmv(x), y), f"CRS runs {l}x{r}"
    # the value gradient at the top of the int32 entry range, on the sampled
    # rows: dval_k = g[row_k] x[col_k], exact for these integers
    g = S.limit_x(i + 5).to(torch.float64)
    d = M.dval(g, x)
    rt = torch.as_tensor(rows, device="cuda")
    k0 = M.row_ptr[rt].to(torch.int64).cpu().numpy()
    lens = S.limit_lengths(rows.astype(np.int64))
    ks = np.concatenate([np.arange(a, a + n) for a, n in zip(k0, lens)])
    rk = np.repeat(rows.astype(np.int64), lens)
    jk = ks - np.repeat(k0, lens)
    want = S.limit_x(rk + 5).astype(np.float64) * S.limit_x(S.limit_cols(rk, jk)).astype(np.float64)
    assert np.array_equal(host(d[torch.as_tensor(ks, device="cuda")]), want), "dval"
    del d
    for fmt, perm, kw in (("SELL", "row_only", dict(window=128, unroll=4)),
                          ("NUJDS", "symmetric", dict(unroll=2))):
        G = M.to_jds(fmt, perm, **kw)
        assert torch.equal(G.spmv_original(x), y), fmt
        del G
        torch.cuda.empty_cache()
    # the adjoint through the transposed structure: <A^T g, x> = <g, A x>,
    # exact (integers well below 2^53)
    M.transpose()
    g = S.limit_x(i + 3).to(torch.float64)
    z = M.spmv(g, transpose=True)
    assert float(torch.dot(z, x)) == float(torch.dot(g, y))
