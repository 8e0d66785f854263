"""JDS family on the GPU: conversion arrays bit-exact against the oracle's
builder (Sect. 2 JDS construction, RBJDS / SOJDS layouts) and products
against the oracle's JDS loops."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import adversarial_matrices, assert_close64, crs, dev, host
from paper_0910_4836_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import paper_0910_4836_gb300 as g
    g.build()


MATS = [
    lambda: S.laplace2d(),
    lambda: S.hh_like(100_000, 21),
    lambda: S.zipf_rows(60_000, 22, lmax=5000),
    lambda: S.small_random(500, 500, 23, density=0.02, empty_rows=0.3),
]


def check_arrays(J, Oj, fmt, block):
    assert np.array_equal(host(J.perm), Oj.perm)
    assert np.array_equal(host(J.iperm), Oj.iperm)
    assert np.array_equal(host(J.jd_ptr), Oj.jd_ptr)
    if fmt in ("RBJDS", "SOJDS"):
        bp, c, v = (O.rbjds_build if fmt == "RBJDS" else O.sojds_build)(Oj, block)
        assert np.array_equal(host(J.blk_ptr), bp)
        assert np.array_equal(host(J.col), c)
        assert np.array_equal(host(J.val).view(np.int64), v.view(np.int64))
    else:
        assert np.array_equal(host(J.col), Oj.col)
        assert np.array_equal(host(J.val).view(np.int64), Oj.val.view(np.int64))


@pytest.mark.parametrize("mi", range(len(MATS)))
@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_conversion_bit_exact(mi, perm):
    A = MATS[mi]()
    M = crs(A)
    Oj = O.jds_build(A, symmetric=perm == "symmetric")
    for fmt, block in [("JDS", 256), ("RBJDS", 256), ("RBJDS", 1000), ("SOJDS", 128),
                       ("SOJDS", 1000)]:
        J = M.to_jds(fmt, perm, block=block)
        assert J.n_diag == Oj.n_diag
        check_arrays(J, Oj, fmt, block)


@pytest.mark.parametrize("mi", range(len(MATS)))
@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_sell_conversion_and_products(mi, perm):
    A = MATS[mi]()
    M = crs(A)
    x = S.vector(A.n_cols, 51 + mi)
    ref, s = O.crs_spmv_exact(A, x)
    Jref = None
    for window in (32, 256, 1024, 32 * ((A.n_rows + 31) // 32)):
        Os = O.sell_build(A, window, symmetric=perm == "symmetric")
        G = M.to_jds("SELL", perm, window=window, value_map=True)
        assert np.array_equal(host(G.perm), Os.perm)
        assert np.array_equal(host(G.iperm), Os.iperm)
        assert np.array_equal(host(G.rlen), Os.rlen)
        assert np.array_equal(host(G.blk_ptr), Os.blk_ptr)
        assert np.array_equal(host(G.col), Os.col)
        assert np.array_equal(host(G.val).view(np.int64), Os.val.view(np.int64))
        xp = O.permute(Os.perm, x) if perm == "symmetric" else x
        for u in (1, 2, 4):
            G.set_format("SELL", unroll=u)
            yp = host(G.spmv(dev(xp)))
            assert_close64(yp, O.permute(Os.perm, ref), O.permute(Os.perm, s), f"SELL w={window} u={u}")
            assert_close64(host(G.spmv_original(dev(x))), ref, s, f"SELL w={window} u={u} original")
        # the value map re-gathers new values
        G.refresh_values(dev(A.val * 2.0))
        assert_close64(host(G.spmv_original(dev(x))) / 2.0, ref, s, "SELL refreshed values")
        if window >= A.n_rows:
            # one window: the JDS sort, so per-row sums match the JDS kernels bit for bit
            J = M.to_jds("JDS", perm)
            G2 = M.to_jds("SELL", perm, window=window)
            assert torch.equal(G2.spmv(dev(xp)), J.spmv(dev(xp)))


@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_deep_split(perm):
    """Long rows split over chunk threads: same product within tolerance,
    exact on integer data, for every walk that honours the split."""
    A = S.zipf_rows(50_000, 57, lmax=5000)
    x = S.vector(A.n_cols, 57)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    J = M.to_jds("JDS", perm)
    for depth, chunk in ((1, 1), (8, 32), (64, 128), (256, 64), (J.n_diag - 1, 7)):
        J.split(depth, chunk)
        for fmt, b, u, r in (("JDS", 0, 0, 1), ("NUJDS", 0, 2, 2), ("NUJDS", 0, 4, 1)):
            set_variant(J, fmt, b, u, r)
            assert_close64(host(J.spmv_original(dev(x))), ref, s, f"split {depth}/{chunk} {fmt} u{u} r{r}")
    # the split product forks its deep kernel onto a side stream: it must
    # still capture into a CUDA graph and replay to the same result
    J.split(16, 32)
    set_variant(J, "NUJDS", 0, 2, 1)
    xd = dev(x)
    yd = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    ref_split = host(J.spmv_original(xd, out=yd)).copy()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        J.spmv_original(xd, out=yd)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        J.spmv_original(xd, out=yd)
    yd.zero_()
    g.replay()
    assert np.array_equal(host(yd), ref_split)
    J.split(0)
    Ai = S.integer_values(A, 58, 1000)
    xi = S.int_vector(A.n_cols, 58, 1000)
    Ji = crs(Ai).to_jds("NUJDS", perm, unroll=2)
    Ji.split(32, 100)
    assert np.array_equal(host(Ji.spmv_original(dev(xi))), O.crs_spmv(Ai, xi))


def test_sell_spmm_and_integer():
    A = S.integer_values(S.hh_like(50_000, 53), 53, 512)
    X = np.stack([S.int_vector(A.n_cols, 60 + c, 512) for c in range(16)], axis=1)
    ref = O.crs_spmm(A, X)
    G = crs(A).to_jds("SELL", "row_only", window=512)
    for k in (1, 4, 16):
        Y = host(G.spmm(dev(X[:, :k].copy()), basis=1))
        assert np.array_equal(Y, ref[:, :k]), k


def test_golden_example_on_gpu():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "jds_5x5.json")))
    rows, cols, vals = [], [], []
    for i, cs in enumerate(g["rows"]):
        for j in cs:
            rows.append(i)
            cols.append(j)
            vals.append(10 * (i + 1) + (j + 1))
    A = S.from_coo(5, 5, rows, cols, vals)
    J = crs(A).to_jds("JDS", "symmetric")
    assert host(J.perm).tolist() == g["perm"]
    assert host(J.jd_ptr).tolist() == g["jd_ptr"]
    assert host(J.col).tolist() == g["col_jds_symmetric"]
    assert host(J.val).tolist() == g["val_jds"]
    xp = dev(np.array(g["x_permuted"], float))
    for fmt in ("JDS", "NBJDS", "NUJDS", "JDS_LITERAL"):
        J.set_format(fmt, block=2, unroll=2)
        assert host(J.spmv(xp)).tolist() == g["y_permuted"]
    R = crs(A).to_jds("RBJDS", "symmetric", block=g["rbjds_block"])
    assert host(R.blk_ptr).tolist() == g["rbjds_blk_ptr"]
    assert host(R.val).tolist() == g["rbjds_val"]
    assert host(R.spmv(xp)).tolist() == g["y_permuted"]


def variants():
    """(format, block, unroll, rows per thread)"""
    yield "JDS", 0, 0, 1
    yield "JDS", 0, 0, 4
    yield "JDS_LITERAL", 0, 0, 1
    for u in (2, 3, 4, 8, 16):
        for r in (1, 2, 4):
            yield "NUJDS", 0, u, r
    for b in (32, 100, 256, 1000, 2048, 5000):
        yield "NBJDS", b, 0, 1


def set_variant(J, fmt, b, u, r):
    J.set_format(fmt, block=b, unroll=u)
    J.set_kernel("vector", rows_per_warp=r)


@pytest.mark.parametrize("mi", range(len(MATS)))
def test_products_permuted_and_original(mi):
    A = MATS[mi]()
    x = S.vector(A.n_cols, 31 + mi)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    for perm in ("symmetric", "row_only"):
        Oj = O.jds_build(A, symmetric=perm == "symmetric")
        xp = O.permute(Oj.perm, x) if perm == "symmetric" else x
        ref_p = O.permute(Oj.perm, ref)
        s_p = O.permute(Oj.perm, s)
        J = M.to_jds("JDS", perm)
        xd, xpd = dev(x), dev(xp)
        first = None
        for fmt, b, u, r in variants():
            set_variant(J, fmt, b, u, r)
            yp = host(J.spmv(xpd))
            assert_close64(yp, ref_p, s_p, f"{perm} {fmt} b={b} u={u} r={r} permuted")
            yo = host(J.spmv_original(xd))
            assert_close64(yo, ref, s, f"{perm} {fmt} b={b} u={u} r={r} original")
            # every JDS-family kernel adds a row in slot order: identical bits
            if first is None:
                first = yp
            assert np.array_equal(yp.view(np.int64), first.view(np.int64)), fmt
        for fmt, b in [("RBJDS", 256), ("RBJDS", 1000), ("RBJDS", 1), ("SOJDS", 256)]:
            R = M.to_jds(fmt, perm, block=b)
            yp = host(R.spmv(xpd))
            assert_close64(yp, ref_p, s_p, f"{perm} {fmt} b={b}")
            if fmt == "RBJDS":
                assert np.array_equal(yp.view(np.int64), first.view(np.int64))
            assert_close64(host(R.spmv_original(xd)), ref, s, f"{perm} {fmt} original")


def test_integer_bit_exact_against_literal_loop():
    A = S.integer_values(S.zipf_rows(40_000, 41, lmax=3000), 41, 1024)
    x = S.int_vector(A.n_cols, 41, 1024)
    M = crs(A)
    Oj = O.jds_build(A, True)
    xp = O.permute(Oj.perm, x)
    ref = O.jds_spmv(Oj, xp)
    J = M.to_jds("JDS", "symmetric")
    xpd = dev(xp)
    for fmt, b, u, r in variants():
        set_variant(J, fmt, b, u, r)
        assert np.array_equal(host(J.spmv(xpd)), ref), (fmt, b, u, r)
    for fmt in ("RBJDS", "SOJDS"):
        assert np.array_equal(host(M.to_jds(fmt, "symmetric", block=500).spmv(xpd)), ref), fmt
    # unpermuted result equals CRS
    assert np.array_equal(host(J.spmv_original(dev(x))), O.crs_spmv(A, x))


def test_permute_roundtrip_and_rectangular():
    A = S.small_random(300, 77, 51, density=0.1, empty_rows=0.2)
    M = crs(A)
    J = M.to_jds("JDS", "row_only")
    x = S.vector(77, 51)
    ref, s = O.crs_spmv_exact(A, x)
    assert_close64(host(J.spmv_original(dev(x))), ref, s, "rect original")
    v = dev(S.vector(300, 52))
    assert torch.equal(J.permute(J.permute(v), back=True), v)
    from paper_0910_4836_gb300 import GbspError
    with pytest.raises(GbspError):
        M.to_jds("JDS", "symmetric")


def test_jds_spmm():
    A = S.hh_like(60_000, 61)
    X = np.stack([S.vector(A.n_cols, 70 + c) for c in range(16)], axis=1)
    Yref, Sref = O.crs_spmm_exact(A, X)
    M = crs(A)
    for fmt in ("JDS", "NBJDS", "RBJDS", "SOJDS"):
        J = M.to_jds(fmt, "symmetric", block=512)
        for k in (4, 5, 16):
            Y = host(J.spmm(dev(X[:, :k].copy()), basis=1))
            for c in range(k):
                assert_close64(Y[:, c], Yref[:, c], Sref[:, c], f"{fmt} k={k} col {c}")


@pytest.mark.parametrize("idx", range(9))
def test_adversarial(idx):
    A = adversarial_matrices()[idx]
    perm = "symmetric" if A.n_rows == A.n_cols else "row_only"
    x = S.vector(A.n_cols, 80 + idx)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    Oj = O.jds_build(A, symmetric=perm == "symmetric")
    for fmt, b in [("JDS", 0), ("NUJDS", 0), ("NBJDS", 64), ("RBJDS", 64), ("SOJDS", 64),
                   ("JDS_LITERAL", 0)]:
        J = M.to_jds(fmt, perm, block=b or 256)
        check_arrays(J, Oj, fmt, b or 256)
        assert_close64(host(J.spmv_original(dev(x))), ref, s, f"{A.name} {fmt}")


PSELL_MATS = MATS + [lambda: S.small_random(65, 65, 24, density=0.1),
                     lambda: S.small_random(127, 127, 25, density=0.05, empty_rows=0.5),
                     lambda: S.from_coo(3, 3, [1], [2], [1.5])]


@pytest.mark.parametrize("mi", range(len(PSELL_MATS)))
@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_psell_conversion_and_products(mi, perm):
    """Paired SELL: arrays bit-exact against the oracle's builder, products
    within tolerance for every unroll, in both bases, with accumulate."""
    A = PSELL_MATS[mi]()
    M = crs(A)
    x = S.vector(A.n_cols, 71 + mi)
    ref, s = O.crs_spmv_exact(A, x)
    for window in (64, 128, 1024):
        Op = O.psell_build(A, window, symmetric=perm == "symmetric")
        G = M.to_jds("PSELL", perm, window=window, value_map=True)
        assert G.n_blocks == (A.n_rows + 63) // 64
        assert np.array_equal(host(G.perm), Op.perm)
        assert np.array_equal(host(G.iperm), Op.iperm)
        assert np.array_equal(host(G.rlen), Op.rlen)
        assert np.array_equal(host(G.blk_ptr), Op.blk_ptr)
        assert np.array_equal(host(G.col), Op.col)
        assert np.array_equal(host(G.val).view(np.int64), Op.val.view(np.int64))
        xp = O.permute(Op.perm, x) if perm == "symmetric" else x
        for u in (1, 2, 4):
            G.set_format("PSELL", unroll=u)
            yp = host(G.spmv(dev(xp)))
            assert_close64(yp, O.permute(Op.perm, ref), O.permute(Op.perm, s), f"PSELL w={window} u={u}")
            yo = host(G.spmv_original(dev(x)))
            assert_close64(yo, ref, s, f"PSELL w={window} u={u} original")
            # y += A x on top of a known y
            y0 = S.vector(A.n_rows, 5)
            out = dev(O.permute(Op.perm, y0))
            G.spmv(dev(xp), out=out, accumulate=True)
            assert_close64(host(out) - O.permute(Op.perm, y0), O.permute(Op.perm, ref),
                           O.permute(Op.perm, s) + np.abs(O.permute(Op.perm, y0)), f"PSELL accumulate u={u}")
        # the oracle's own paired loop, in the permuted basis
        assert_close64(O.psell_spmv(Op, xp), O.permute(Op.perm, ref), O.permute(Op.perm, s), "oracle PSELL")
        G.refresh_values(dev(A.val * 2.0))
        assert_close64(host(G.spmv_original(dev(x))) / 2.0, ref, s, "PSELL refreshed values")


def test_psell_spmm_integer_and_rejections():
    A = S.integer_values(S.hh_like(50_000, 54), 54, 512)
    X = np.stack([S.int_vector(A.n_cols, 80 + c, 512) for c in range(16)], axis=1)
    ref = O.crs_spmm(A, X)
    M = crs(A)
    G = M.to_jds("PSELL", "row_only", window=128)
    for k in (1, 3, 4, 16):
        Y = host(G.spmm(dev(X[:, :k].copy()), basis=1))
        assert np.array_equal(Y, ref[:, :k]), k
    from paper_0910_4836_gb300 import GbspError
    with pytest.raises(GbspError):
        M.to_jds("PSELL", "row_only", window=96)  # not a multiple of 64
    with pytest.raises(GbspError):
        G.set_format("SELL")  # different storage


STAGE_MATS = [lambda: S.laplace2d(), lambda: S.hh_like(100_000, 21), lambda: S.zipf_rows(60_000, 22, lmax=3000),
              lambda: S.small_random(500, 700, 23, density=0.02, empty_rows=0.3),
              lambda: S.from_coo(3, 3, [1], [2], [1.5])]


@pytest.mark.parametrize("mi", range(len(STAGE_MATS)))
@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_sell_staged_x_is_bit_identical(mi, perm):
    """Staging pages of x in shared memory changes where x values are read,
    not the arithmetic: the staged SELL product equals the unstaged one bit
    for bit, in FP64 and compensated FP32, and matches the oracle."""
    A = STAGE_MATS[mi]()
    if perm == "symmetric" and A.n_rows != A.n_cols:
        pytest.skip("symmetric permutation needs a square matrix")
    x = S.vector(A.n_cols, 91 + mi)
    ref, s = O.crs_spmv_exact(A, x)
    for dtype in (torch.float64, torch.float32):
        M = crs(A, dtype)
        if dtype == torch.float32:
            M.set_kernel("vector", compensated=True)
        for w, u in ((128, 1), (128, 2), (1024, 4)):
            G = M.to_jds("SELL", perm, window=w, unroll=u)
            xd = dev(x).to(dtype)
            xp = G.permute(xd)  if perm == "symmetric" else xd
            plain = G.spmv(xp).clone()
            plain_o = G.spmv_original(xd).clone()
            for pages, refs in ((12, 32), (1, 1), (4, 10 ** 9)):
                G.stage_x(pages, refs)
                assert torch.equal(G.spmv(xp), plain), (mi, perm, dtype, w, u, pages, refs)
                assert torch.equal(G.spmv_original(xd), plain_o)
            G.stage_x(0)
            assert torch.equal(G.spmv(xp), plain)
            if dtype == torch.float64:
                assert_close64(host(plain_o), ref, s, f"staged SELL w={w} u={u}")


@pytest.mark.slow
@pytest.mark.parametrize("cfg", [1, 2, 4])
def test_full_size_step_kernels(cfg):
    """The schemes the benchmark times, at full size and in its launch
    configuration: every output entry against the accurate oracle (SELL-32-σ
    σ=128 u=4 and NUJDS on the HH-like matrix and the stencil; NUJDS split
    16/64 on the Zipf rows), and the staged-x SELL bit-identical to SELL."""
    from gpu_util import full_config
    A = full_config(cfg)
    x = S.vector(A.n_cols, cfg)
    ref, s = O.crs_spmv_exact(A, x)
    M = crs(A)
    xd = dev(x)
    if cfg == 2:
        J = M.to_jds("NUJDS", "row_only", unroll=2)
        J.split(16, 64)
        assert_close64(host(J.spmv_original(xd)), ref, s, "Zipf NUJDS split 16/64")
        return
    G = M.to_jds("SELL", "row_only", window=128, unroll=4)
    y = host(G.spmv_original(xd))
    assert_close64(y, ref, s, f"config {cfg} SELL w=128 u=4")
    G.stage_x(12, 32)
    assert np.array_equal(host(G.spmv_original(xd)), y)
    del G
    # the bench's step: the symmetric permutation, x and y in the permuted basis
    Gs = M.to_jds("SELL", "symmetric", window=128, unroll=4)
    perm = host(Gs.perm)
    yp = host(Gs.spmv(Gs.permute(xd)))
    assert_close64(yp, ref[perm], s[perm], f"config {cfg} SELL symmetric w=128 u=4, permuted basis")
    del Gs
    J = M.to_jds("NUJDS", "symmetric", unroll=2)
    assert_close64(host(J.spmv_original(xd)), ref, s, f"config {cfg} NUJDS u=2")


def test_psell_fp32_compensated_and_spmm():
    """Paired SELL in FP32 with compensated sums: within the Dot2 bound of
    the exact product of the FP32-rounded data, for one and several RHS."""
    from gpu_util import dot2_bound
    A = S.hh_like(50_000, 61)
    A32 = A.astype(np.float32)
    M = crs(A, torch.float32)
    M.set_kernel("vector", compensated=True)
    G = M.to_jds("PSELL", "row_only", window=128, unroll=4)
    G.set_kernel("vector", compensated=True)
    lens = np.diff(A.row_ptr.astype(np.int64))
    X = np.stack([S.vector(A.n_cols, 62 + c).astype(np.float32) for c in range(4)], axis=1)
    Y = host(G.spmm(dev(X), basis=1)).astype(np.float64)
    for c in range(4):
        ref, s = O.crs_spmv_exact(A32.astype(np.float64), X[:, c].astype(np.float64))
        assert np.all(np.abs(Y[:, c] - ref) <= dot2_bound(ref, s, lens)), c


REFRESH_MATS = [lambda: S.laplace2d(), lambda: S.zipf_rows(40_000, 31, lmax=3000),
                lambda: S.small_random(700, 700, 32, density=0.02, empty_rows=0.3),
                lambda: S.from_coo(3, 3, [1], [2], [1.5])]


@pytest.mark.parametrize("mi", range(len(REFRESH_MATS)))
@pytest.mark.parametrize("perm", ["symmetric", "row_only"])
def test_value_refresh_every_format(mi, perm):
    """Re-gathering new CRS values through the value map gives exactly the
    arrays a fresh conversion of the new values stores, for every layout
    (row-order re-gathers for JDS storage and SELL, entry order otherwise)."""
    A = REFRESH_MATS[mi]()
    v2 = S.vector(A.nnz, 33 + mi)
    M = crs(A)
    M2 = crs(S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col, v2, "new values"))
    for fmt, kw in (("JDS", {}), ("NBJDS", dict(block=128)), ("NUJDS", dict(unroll=2)),
                    ("RBJDS", dict(block=256)), ("SOJDS", dict(block=128)), ("JDS_LITERAL", {}),
                    ("SELL", dict(window=128)), ("PSELL", dict(window=128))):
        G = M.to_jds(fmt, perm, value_map=True, **kw)
        G.refresh_values(dev(v2))
        F = M2.to_jds(fmt, perm, **kw)
        assert np.array_equal(host(G.val).view(np.int64), host(F.val).view(np.int64)), fmt
        assert np.array_equal(host(G.col), host(F.col)), fmt
