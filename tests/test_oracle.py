"""Pins for the CPU oracle: each checks it against something other than
itself -- numpy dense products, exact rational arithmetic, closed forms, the
paper's stated special cases and a hand-worked example."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_0910_4836_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_matrix():
    g = json.load(open(os.path.join(GOLDEN, "jds_5x5.json")))
    n = g["n"]
    rows, cols, vals = [], [], []
    for i, cs in enumerate(g["rows"]):
        for j in cs:
            rows.append(i)
            cols.append(j)
            vals.append(10 * (i + 1) + (j + 1))
    return g, S.from_coo(n, n, rows, cols, vals)


def permuted_crs(A, J):
    """CRS of P A P^T (rows in JDS order, entries in their CRS order,
    columns renumbered), built with numpy only."""
    lens = A.row_lengths()[J.perm]
    rp = np.zeros(A.n_rows + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    src = np.concatenate([np.arange(A.row_ptr[p], A.row_ptr[p + 1]) for p in J.perm]) \
        if A.nnz else np.zeros(0, np.int64)
    col = A.col[src]
    if J.symmetric:
        col = J.iperm[col]
    return S.CRS(A.n_rows, A.n_cols, rp.astype(np.int32), col.astype(np.int32), A.val[src])


# ------------------------------------------------------------- CRS ------

@pytest.mark.parametrize("shape,seed", [((1, 1), 0), ((17, 23), 1), ((120, 120), 2),
                                        ((300, 77), 3), ((64, 300), 4)])
def test_crs_vs_dense(shape, seed):
    A = S.small_random(*shape, seed, density=0.1, empty_rows=0.1)
    x = S.vector(A.n_cols, seed)
    D = A.to_dense()
    y = O.crs_spmv(A, x)
    ye, s = O.crs_spmv_exact(A, x)
    ref = D @ x
    bound = 1e-14 * (np.abs(D) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= bound)
    assert np.all(np.abs(ye - ref) <= bound)
    np.testing.assert_allclose(s, np.abs(D) @ np.abs(x), rtol=1e-13)


def test_crs_accumulate_is_listing_update():
    A = S.small_random(50, 40, 5, density=0.2)
    x = S.vector(40, 5)
    y0 = S.vector(50, 6)
    y = O.crs_spmv(A, x, y0, accumulate=True)
    np.testing.assert_allclose(y, y0 + A.to_dense() @ x, rtol=0, atol=1e-13)
    ye, _ = O.crs_spmv_exact(A, x, y0, accumulate=True)
    exact = [float(Fraction(y0[i]) + sum(Fraction(v) * Fraction(x[c]) for v, c in
                                         zip(A.val[A.row_ptr[i]:A.row_ptr[i + 1]],
                                             A.col[A.row_ptr[i]:A.row_ptr[i + 1]])))
             for i in range(50)]
    assert np.array_equal(ye, np.array(exact))


def test_exact_oracle_is_correctly_rounded_on_cancellation():
    # rows built to cancel catastrophically: naive sums lose every digit
    rng_rows = []
    vals = []
    cols = []
    for i in range(40):
        big = S.uniform(7, 1, np.arange(i * 8, i * 8 + 8), 1e10, 1e12)
        small = S.uniform(7, 2, np.arange(i * 8, i * 8 + 8), -1, 1)
        v = np.concatenate([big, -big, small])
        vals.extend(v)
        cols.extend(range(24))
        rng_rows.extend([i] * 24)
    A = S.from_coo(40, 24, rng_rows, cols, vals, dedupe=False)
    x = np.concatenate([np.ones(8), np.ones(8), np.full(8, 0.5)])
    y, _ = O.crs_spmv_exact(A, x)
    for i in range(40):
        sl = slice(A.row_ptr[i], A.row_ptr[i + 1])
        exact = float(sum(Fraction(v) * Fraction(x[c]) for v, c in zip(A.val[sl], A.col[sl])))
        fs = math.fsum([float(v) * x[c] for v, c in zip(A.val[sl], A.col[sl])])
        assert y[i] == exact
        # x is 1 or 1/2, so every product is exact and fsum (correctly
        # rounded summation) is a second, library, pin on the same value
        assert fs == exact


def test_identity_and_diagonal_bit_exact():
    n = 257
    x = S.vector(n, 11)
    eye = S.from_coo(n, n, np.arange(n), np.arange(n), np.ones(n))
    assert np.array_equal(O.crs_spmv(eye, x), x)
    d = S.vector(n, 12, lo=-3, hi=3)
    D = S.from_coo(n, n, np.arange(n), np.arange(n), d)
    assert np.array_equal(O.crs_spmv(D, x), d * x)


def test_integer_inputs_exact_and_order_free():
    A = S.integer_values(S.random_rows(400, 13, 1, 60), 13, 1024)
    x = S.int_vector(400, 13, 1024)
    Ai = A.to_dense().astype(np.int64)
    ref = (Ai @ x.astype(np.int64)).astype(np.float64)
    assert np.array_equal(O.crs_spmv(A, x), ref)
    assert np.array_equal(O.crs_spmv_exact(A, x)[0], ref)
    assert np.array_equal(O.crs_spmv_omp(A, x), ref)


def test_omp_bit_identical_to_serial():
    A = S.zipf_rows(20000, 5, lmax=500)
    x = S.vector(A.n_cols, 5)
    assert np.array_equal(O.crs_spmv_omp(A, x), O.crs_spmv(A, x))


def test_f32_loop_matches_numpy_float32_for_short_rows():
    A = S.laplace2d(16, 16)
    x = S.int_vector(256, 3, 100)
    y = O.crs_spmv_f32(A, x)
    ref = (A.to_dense() @ x).astype(np.float32)
    assert np.array_equal(y, ref)


def test_spmm_columns_are_spmv():
    A = S.small_random(90, 70, 14, density=0.1)
    X = np.stack([S.vector(70, 20 + c) for c in range(5)], axis=1)
    Y = O.crs_spmm(A, X)
    np.testing.assert_allclose(Y, A.to_dense() @ X, rtol=0, atol=1e-13)
    for c in range(5):
        assert np.array_equal(Y[:, c], O.crs_spmv(A, X[:, c]))


# ------------------------------------------------- Laplacian closed forms --

def test_laplace_constant_and_linear_vectors():
    nx = ny = 64
    A = S.laplace2d(nx, ny)
    assert A.n_rows == 4096 and A.nnz == 20224
    gx, gy = np.arange(4096) % nx, np.arange(4096) // nx
    missing = (gx == 0).astype(int) + (gx == nx - 1) + (gy == 0) + (gy == ny - 1)
    assert np.array_equal(O.crs_spmv(A, np.ones(4096)), missing.astype(float))
    lin = 3.0 * gx + 5.0 * gy + 1.0
    y = O.crs_spmv(A, lin)
    interior = missing == 0
    assert np.all(y[interior] == 0.0)


@pytest.mark.parametrize("p,q", [(1, 1), (3, 7), (64, 1), (20, 33)])
def test_laplace_eigenvectors(p, q):
    A = S.laplace2d(64, 64)
    i, j = np.arange(4096) % 64 + 1, np.arange(4096) // 64 + 1
    # reduce p*i mod 130 first so every angle carries only one rounding
    v = np.sin(np.pi * ((p * i) % 130) / 65) * np.sin(np.pi * ((q * j) % 130) / 65)
    lam = 4 - 2 * np.cos(p * np.pi / 65) - 2 * np.cos(q * np.pi / 65)
    y, s = O.crs_spmv_exact(A, v)
    # the eigen-relation holds to the rounding of v itself (about 8 u |v| per row)
    assert np.all(np.abs(y - lam * v) <= 1e-14 * s + 1e-15)


# ------------------------------------------------------------- JDS ------

def test_golden_jds_hand_example():
    g, A = golden_matrix()
    assert np.array_equal(O.crs_spmv(A, np.array(g["x"], float)), np.array(g["y"], float))
    J = O.jds_build(A, symmetric=True)
    assert J.perm.tolist() == g["perm"]
    assert J.iperm.tolist() == g["iperm"]
    assert J.jd_ptr.tolist() == g["jd_ptr"]
    assert J.val.tolist() == g["val_jds"]
    assert J.col.tolist() == g["col_jds_symmetric"]
    xp = O.permute(J.perm, np.array(g["x"], float))
    assert xp.tolist() == g["x_permuted"]
    assert O.jds_spmv(J, xp).tolist() == g["y_permuted"]
    R = O.jds_build(A, symmetric=False)
    assert R.col.tolist() == g["col_jds_row_only"]
    assert O.jds_spmv(R, np.array(g["x"], float)).tolist() == g["y_permuted"]
    bp, c, v = O.rbjds_build(J, g["rbjds_block"])
    assert bp.tolist() == g["rbjds_blk_ptr"]
    assert v.tolist() == g["rbjds_val"]
    assert c.tolist() == g["rbjds_col_symmetric"]
    assert O.rbjds_spmv(J, bp, c, v, 2, xp).tolist() == g["y_permuted"]


@pytest.mark.parametrize("maker", [
    lambda: S.small_random(200, 200, 21, density=0.05, empty_rows=0.2),
    lambda: S.laplace2d(20, 20),
    lambda: S.zipf_rows(3000, 22, lmax=300),
    lambda: S.hh_like(2000, 23),
])
def test_jds_build_structure(maker):
    A = maker()
    lens = A.row_lengths()
    for sym in (True, False):
        J = O.jds_build(A, symmetric=sym)
        # perm is a permutation, iperm its inverse
        assert np.array_equal(np.sort(J.perm), np.arange(A.n_rows))
        assert np.array_equal(J.iperm[J.perm], np.arange(A.n_rows))
        # lengths non-increasing; equal lengths keep original order
        pl = lens[J.perm]
        assert np.all(np.diff(pl) <= 0)
        same = np.diff(pl) == 0
        assert np.all(np.diff(J.perm)[same] > 0)
        # closed form: diagLen(d) = #{i : len_i > d}
        nj = int(lens.max()) if A.n_rows else 0
        assert J.n_diag == nj
        expect = np.array([(lens > d).sum() for d in range(nj)])
        assert np.array_equal(J.diag_len(), expect)
        # round trip: every JDS entry maps back to the CRS entry it came from
        rows_back = []
        cols_back = []
        vals_back = []
        for d in range(nj):
            for r in range(J.diag_len()[d]):
                k = J.jd_ptr[d] + r
                rows_back.append(J.perm[r])
                cols_back.append(J.perm[J.col[k]] if sym else J.col[k])
                vals_back.append(J.val[k])
        B = S.from_coo(A.n_rows, A.n_cols, rows_back, cols_back, vals_back, dedupe=False)
        assert np.array_equal(B.row_ptr, A.row_ptr)
        assert np.array_equal(B.col, A.col)
        assert np.array_equal(B.val, A.val)


def test_jds_symmetric_rejects_rectangular():
    A = S.small_random(30, 40, 3)
    with pytest.raises(ValueError):
        O.jds_build(A, symmetric=True)
    J = O.jds_build(A, symmetric=False)
    x = S.vector(40, 3)
    y = O.permute(J.perm, O.jds_spmv(J, x), to_permuted=False)
    np.testing.assert_allclose(y, A.to_dense() @ x, rtol=0, atol=1e-14)


@pytest.mark.parametrize("sym", [True, False])
def test_jds_family_equals_crs_in_permuted_basis(sym):
    """JDS / NBJDS / NUJDS / RBJDS all add each row's entries in slot order
    from zero, so they are bit-identical to CRS on P A P^T; NUJDS with
    u = N_j is stated to be exactly that (Sect. 2), RBJDS with block 1 is
    row-by-row access and JDS is NBJDS with block = N (Sect. 4.2)."""
    A = S.hh_like(5000, 31)
    x = S.vector(A.n_cols, 31)
    J = O.jds_build(A, symmetric=sym)
    P = permuted_crs(A, J)
    xp = O.permute(J.perm, x) if sym else x
    ref = O.crs_spmv(P, xp)
    assert np.array_equal(O.jds_spmv(J, xp), ref)
    assert np.array_equal(O.nujds_spmv(J, xp, J.n_diag), ref)
    for u in (1, 2, 3, 4, 8):
        assert np.array_equal(O.nujds_spmv(J, xp, u), ref)
    assert np.array_equal(O.nbjds_spmv(J, xp, A.n_rows), O.jds_spmv(J, xp))
    for b in (1, 7, 128, 1000):
        assert np.array_equal(O.nbjds_spmv(J, xp, b), ref)
        bp, c, v = O.rbjds_build(J, b)
        assert np.array_equal(O.rbjds_spmv(J, bp, c, v, b, xp), ref)
    bp, c, v = O.rbjds_build(J, 1)
    assert np.array_equal(bp, P.row_ptr)
    assert np.array_equal(c, P.col)
    assert np.array_equal(v, P.val)
    # and the un-permuted result is A x
    y = O.permute(J.perm, ref, to_permuted=False)
    ye, s = O.crs_spmv_exact(A, x)
    assert np.all(np.abs(y - ye) <= 1e-14 * s)


def test_jds_integer_bit_exact_unpermuted():
    A = S.integer_values(S.zipf_rows(5000, 41, lmax=2000), 41, 1024)
    x = S.int_vector(A.n_cols, 41, 1024)
    ref = O.crs_spmv(A, x)
    J = O.jds_build(A, True)
    y = O.permute(J.perm, O.jds_spmv(J, O.permute(J.perm, x)), to_permuted=False)
    assert np.array_equal(y, ref)


def test_empty_and_degenerate():
    Z = S.CRS(5, 5, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert np.array_equal(O.crs_spmv(Z, np.ones(5)), np.zeros(5))
    J = O.jds_build(Z)
    assert J.n_diag == 0 and np.array_equal(J.perm, np.arange(5))
    assert np.array_equal(O.jds_spmv(J, np.ones(5)), np.zeros(5))
    one = S.from_coo(1, 1, [0], [0], [2.5])
    assert O.crs_spmv(one, np.array([4.0]))[0] == 10.0
    long_row = S.from_coo(3, 5000, [1] * 5000, np.arange(5000), np.ones(5000))
    y = O.crs_spmv(long_row, np.ones(5000))
    assert y.tolist() == [0.0, 5000.0, 0.0]


# ------------------------------------------------------------- SELL -----

@pytest.mark.parametrize("sym", [True, False])
def test_sell_one_window_is_rbjds_block32(sym):
    """With a single window the row sort is the JDS sort, so SELL-32 is the
    paper's RBJDS with block size 32 (Sect. 2), array for array."""
    A = S.hh_like(3000, 91)
    J = O.jds_build(A, symmetric=sym)
    bp, c, v = O.rbjds_build(J, 32)
    Sl = O.sell_build(A, window=32 * ((A.n_rows + 31) // 32), symmetric=sym)
    assert np.array_equal(Sl.perm, J.perm) and np.array_equal(Sl.iperm, J.iperm)
    assert np.array_equal(Sl.blk_ptr, bp)
    assert np.array_equal(Sl.col, c) and np.array_equal(Sl.val, v)
    assert np.array_equal(Sl.rlen, A.row_lengths()[J.perm])


@pytest.mark.parametrize("window", [32, 64, 1024])
def test_sell_windows(window):
    A = S.zipf_rows(5000, 92, lmax=300)
    Sl = O.sell_build(A, window, symmetric=False)
    lens = A.row_lengths()
    # perm only moves rows inside their window, longest first, stable
    assert np.array_equal(np.sort(Sl.perm), np.arange(A.n_rows))
    assert np.all(Sl.perm // window == np.arange(A.n_rows) // window)
    for w0 in range(0, A.n_rows, window):
        pl = lens[Sl.perm[w0:w0 + window]]
        assert np.all(np.diff(pl) <= 0)
        same = np.diff(pl) == 0
        assert np.all(np.diff(Sl.perm[w0:w0 + window])[same] > 0)
    # each permuted row's entries are the CRS row's entries in slot order
    x = S.vector(A.n_cols, 93)
    P = permuted_crs(A, O.JDS(A.n_rows, A.n_cols, False, Sl.perm, Sl.iperm, None, None, None))
    assert np.array_equal(O.sell_spmv(Sl, x), O.crs_spmv(P, x))
    Ai = S.integer_values(A, 94, 1000)
    xi = S.int_vector(A.n_cols, 94, 1000)
    Si = O.sell_build(Ai, window, symmetric=True)
    y = O.permute(Si.perm, O.sell_spmv(Si, O.permute(Si.perm, xi)), to_permuted=False)
    assert np.array_equal(y, O.crs_spmv(Ai, xi))


def test_sell_windows_with_rows_longer_than_2_17():
    """The matrix the GPU tests use for SELL sort keys wider than 32 bits:
    the oracle's builder still keeps every row in its window, longest
    first, ties in row order, and reproduces the exact product."""
    A = S.long_rows(2 ** 20 + 100, [140_001, 70_001], 5)
    lens = A.row_lengths()
    assert lens.max() == 140_001 and A.n_rows // 32 >= 2 ** 15
    for window in (32, 64):
        Sl = O.sell_build(A, window, symmetric=False)
        assert np.all(Sl.perm // window == np.arange(A.n_rows) // window)
        # along the permuted order: windows ascending, lengths descending
        # inside a window, equal lengths in ascending row order
        key = (np.arange(A.n_rows, dtype=np.int64) // window) * 2 ** 20 - lens[Sl.perm]
        step = np.diff(key)
        assert np.all(step >= 0)
        assert np.all(np.diff(Sl.perm)[step == 0] > 0)
        assert Sl.blk_ptr[-1] == A.nnz
    Ai = S.integer_values(A, 95, 1000)
    xi = S.int_vector(A.n_cols, 95, 1000)
    Si = O.sell_build(Ai, 32, symmetric=False)
    y = np.zeros(A.n_rows)
    y[Si.perm] = O.sell_spmv(Si, xi)
    assert np.array_equal(y, O.crs_spmv(Ai, xi))


def test_index_limit_matrix_closed_forms():
    """The index-limit generator: exactly 2^31 - 2^16 - 1 entries on 2^24
    rows of length 7..248, distinct columns in a row, and every row sum an
    integer below 2^12 in magnitude (exact in any order)."""
    i = np.arange(S.LIMIT_ROWS, dtype=np.int64)
    L = S.limit_lengths(i)
    assert int(L.sum()) == S.LIMIT_NNZ == 2 ** 31 - 2 ** 16 - 1
    assert L.min() == 7 and L.max() == 248
    assert np.all(L[0::2] + L[1::2] == 256 - (i[0::2] < 2 ** 16 + 1) - (i[1::2] < 2 ** 16 + 1))
    rows = np.array([0, 5, 2 ** 16, S.LIMIT_ROWS - 1])
    sub = S.limit_rows_crs(rows)
    for k, r in enumerate(rows):
        c = sub.col[sub.row_ptr[k]:sub.row_ptr[k + 1]]
        assert len(np.unique(c)) == len(c) == L[r]
    assert np.abs(sub.val).max() <= 3 and np.abs(S.limit_x(i)).max() <= 5
    assert 248 * 3 * 5 < 2 ** 12


# ------------------------------------------------------------ SOJDS -----

def test_sojds_is_row_permutation_and_same_product():
    A = S.hh_like(3000, 51)
    x = S.vector(A.n_cols, 51)
    J = O.jds_build(A, True)
    xp = O.permute(J.perm, x)
    for b in (1, 16, 100):
        bp, c, v = O.rbjds_build(J, b)
        bs, cs, vs = O.sojds_build(J, b)
        assert np.array_equal(bp, bs)
        # each row keeps its multiset of (col, val): compare per row
        lens = A.row_lengths()[J.perm]
        for k in range(len(bp) - 1):
            b0 = k * b
            rows = np.arange(b0, min(b0 + b, A.n_rows))
            seg_r = np.concatenate([rows[: (lens[rows] > d).sum()] for d in range(lens[b0])]) \
                if lens[b0] else np.zeros(0, int)
            sl = slice(bp[k], bp[k + 1])
            for r in rows:
                m = seg_r == r
                a = sorted(zip(c[sl][m], v[sl][m]))
                s = sorted(zip(cs[sl][m], vs[sl][m]))
                assert a == s
        y = O.rbjds_spmv(J, bs, cs, vs, b, xp)
        ref, sabs = O.crs_spmv_exact(permuted_crs(A, J), xp)
        assert np.all(np.abs(y - ref) <= 1e-14 * sabs)


def test_sojds_restores_unit_stride_on_shuffled_tridiagonal():
    """Closed case: interior rows of a tridiagonal matrix have columns
    {i-1, i, i+1}; with each row's entries stored in a shuffled order, the
    greedy rule must give stride exactly one down every block column."""
    n = 400
    rows, cols = [], []
    for i in range(n):
        cs = [c for c in (i - 1, i, i + 1) if 0 <= c < n]
        order = np.argsort(S.uniform01(61, 1, np.arange(3 * i, 3 * i + len(cs))))
        for o in order:
            rows.append(i)
            cols.append(cs[o])
    # unsorted entry order inside rows: build CRS directly, no sorting
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    A = S.CRS(n, n, rp, np.array(cols, np.int32), np.arange(len(cols), dtype=float))
    # row-only permutation keeps the original column numbers, so the interior
    # rows (all of length 3, kept in order by the stable sort) stay banded
    J = O.jds_build(A, False)
    b = 50
    bs, cs, vs = O.sojds_build(J, b)
    lens = A.row_lengths()[J.perm]
    nb = len(bs) - 1
    for k in range(nb):
        b0, b1 = k * b, min(k * b + b, n)
        if not np.all(lens[b0:b1] == 3):
            continue
        block = cs[bs[k]:bs[k + 1]].reshape(3, b1 - b0)   # slot-major, 3 full slots
        assert np.all(np.diff(block, axis=1) == 1)


# ------------------------------------------------ adjoint and gradients --

def test_adjoint_identity_and_transpose():
    A = S.small_random(150, 90, 71, density=0.08)
    g = S.vector(150, 71)
    x = S.vector(90, 72)
    at = O.crs_spmv_t(A, g)
    np.testing.assert_allclose(at, A.to_dense().T @ g, rtol=0, atol=1e-14)
    lhs = math.fsum(O.crs_spmv_t_exact(A, g)[0] * x)
    rhs = math.fsum(g * O.crs_spmv_exact(A, x)[0])
    assert abs(lhs - rhs) <= 1e-13 * math.fsum(np.abs(g) * (np.abs(A.to_dense()) @ np.abs(x)))
    # integer values: scatter adjoint == CRS of the explicit transpose, bit-exact
    Ai = S.integer_values(A, 71, 1000)
    gi = S.int_vector(150, 72, 1000)
    rid = Ai.row_ids()
    T = S.from_coo(90, 150, Ai.col, rid, Ai.val)
    assert np.array_equal(O.crs_spmv_t(Ai, gi), O.crs_spmv(T, gi))
    assert np.array_equal(O.crs_spmv_t_exact(Ai, gi)[0], O.crs_spmv(T, gi))


def test_dval_is_gradient_of_bilinear_form():
    A = S.small_random(40, 30, 81, density=0.2)
    g = S.vector(40, 81)
    x = S.vector(30, 82)
    dv = O.dval(A, g, x)
    rid = A.row_ids()
    assert np.array_equal(dv, g[rid] * x[A.col])
    # central difference of f(val) = g . (A x); f is linear in val, so the
    # difference quotient is exact up to rounding
    h = 1e-3
    for k in range(0, A.nnz, max(A.nnz // 25, 1)):
        vp, vm = A.val.copy(), A.val.copy()
        vp[k] += h
        vm[k] -= h
        fp = math.fsum(g * O.crs_spmv(S.CRS(40, 30, A.row_ptr, A.col, vp), x))
        fm = math.fsum(g * O.crs_spmv(S.CRS(40, 30, A.row_ptr, A.col, vm), x))
        assert abs((fp - fm) / (2 * h) - dv[k]) <= 1e-9


def test_power_gradient_finite_differences():
    A = S.stencil27(6, 4)
    x = S.vector(A.n_cols, 4)
    m = 3
    L, dv, dx = O.power_loss_grad(A, x, m)

    def loss(val, xx):
        B = S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col, val)
        return float(np.dot(O.power_forward(B, xx, m)[-1], O.power_forward(B, xx, m)[-1]))

    h = 1e-6
    for t in range(4):
        dvec = S.uniform(4, 90 + t, np.arange(A.nnz), -1, 1)
        fd = (loss(A.val + h * dvec, x) - loss(A.val - h * dvec, x)) / (2 * h)
        an = float(np.dot(dv, dvec))
        assert abs(fd - an) <= 1e-6 * abs(an)
        dxv = S.uniform(4, 95 + t, np.arange(A.n_cols), -1, 1)
        fd = (loss(A.val, x + h * dxv) - loss(A.val, x - h * dxv)) / (2 * h)
        an = float(np.dot(dx, dxv))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_power_gradient_closed_form_symmetric():
    """For symmetric A, d||A^m x||^2/dx = 2 A^{2m} x."""
    A = S.stencil27(6, 4, symmetric_values=True)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    x = S.vector(A.n_cols, 5)
    m = 4
    _, _, dx = O.power_loss_grad(A, x, m)
    ref = 2 * O.power_forward(A, x, 2 * m)[-1]
    np.testing.assert_allclose(dx, ref, rtol=1e-12, atol=1e-15)


# -------------------------------------------------------- generators ----

def test_splitmix64_published_sequence():
    """Draw t of a stream is mix(key + (t+1)*GAMMA); with key 0 that is the
    SplitMix64 generator started from state 0, whose first outputs are
    published (Steele, Lea & Flood 2014; Vigna's reference code)."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.array([np.uint64(t + 1) * gamma for t in range(4)], dtype=np.uint64)
    got = [int(v) for v in S._mix(z)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    # uniform01 uses the top 53 bits
    u = S.uniform01(0, 0, np.arange(4))
    assert np.all((u >= 0) & (u < 1))
    assert np.array_equal(u, (S.bits(0, 0, np.arange(4)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)


def test_generator_shapes():
    A = S.hh_like(20000, 1)
    D = A.to_dense() if A.n_rows <= 2000 else None
    assert D is None
    lens = A.row_lengths()
    # at this small size the far band offsets (up to 262144) mostly fall off
    # the matrix; the full 6e6 workload gives about 13 per row
    assert 7 <= lens.mean() <= 15
    # symmetric pattern and values
    T = S.from_coo(A.n_cols, A.n_rows, A.col, A.row_ids(), A.val)
    assert np.array_equal(T.row_ptr, A.row_ptr) and np.array_equal(T.col, A.col)
    assert np.array_equal(T.val, A.val)
    Z = S.zipf_rows(200000, 2)
    assert 5.3 <= Z.nnz / Z.n_rows <= 5.7
    assert Z.row_lengths().max() <= 5000
    assert S.stencil27(10).nnz == 28 ** 3
    assert S.laplace2d().nnz == 20224
    # rows come out column-sorted
    for M in (A, Z):
        d = np.diff(M.col.astype(np.int64))
        starts = M.row_ptr[1:-1]
        mask = np.ones(len(d), bool)
        mask[starts[(starts > 0) & (starts <= len(d))] - 1] = False
        assert np.all(d[mask] > 0)


# --------------------------------------------------------------------------
# Basic sparse vector operations (Sect. 4.1 table: ADD / SCP over PD, CS,
# IS, IR)
# --------------------------------------------------------------------------

def test_gather_dense_add_closed_form():
    n = 100_000
    b = np.arange(1, n + 1, dtype=np.float64)
    assert O.gather_sum("ADD", "PD", n, b) == n * (n + 1) // 2
    assert O.gather_sum_exact("ADD", "PD", n, b) == (n * (n + 1) // 2, n * (n + 1) // 2)


@pytest.mark.parametrize("k", [1, 8, 530])
def test_gather_constant_stride_closed_forms(k):
    """B(j) = j, A(i) = i + 1: ADD gives k n(n-1)/2, SCP gives
    k (sum i^2 + sum i) = k (n-1) n (2n-1)/6 + k n(n-1)/2 -- integers below
    2^53, so exact in every order."""
    n = 3000
    b = np.arange(k * (n - 1) + 1, dtype=np.float64)
    a = np.arange(1, n + 1, dtype=np.float64)
    add = k * n * (n - 1) // 2
    scp = k * (n - 1) * n * (2 * n - 1) // 6 + add
    assert O.gather_sum("ADD", "CS", n, b, k=k) == add
    assert O.gather_sum("SCP", "CS", n, b, a=a, k=k) == scp
    # IS: the same loop through an index array ind(i) = k i
    ind = S.stride_indices(n, k)
    assert O.gather_sum("ADD", "IND", n, b, ind=ind) == add
    assert O.gather_sum("SCP", "IND", n, b, a=a, ind=ind) == scp


def test_gather_scp_with_unit_a_is_add():
    n = 5000
    b = S.vector(4 * n, 7)
    ind = S.geometric_indices(n, 0.25, 7)
    ind = ind[ind < len(b)]
    m = len(ind)
    ones = np.ones(m)
    assert O.gather_sum("SCP", "IND", m, b, a=ones, ind=ind) == O.gather_sum("ADD", "IND", m, b, ind=ind)


def test_gather_exact_against_rationals():
    """Random A, B, IR indices: the accurate sum is within one rounding of
    the exact rational sum; the loop-order sum within n u sum|t|."""
    n = 600
    b = S.vector(5000, 11)
    a = S.vector(n, 12)
    ind = S.bernoulli_indices(5000, 0.15, 13)[:n]
    n = len(ind)
    exact = sum(Fraction(float(a[i])) * Fraction(float(b[ind[i]])) for i in range(n))
    s, abs_sum = O.gather_sum_exact("SCP", "IND", n, b, a=a, ind=ind)
    assert abs(Fraction(s) - exact) <= Fraction(2.0 ** -52) * abs(exact) + Fraction(2.0 ** -100) * Fraction(abs_sum)
    assert math.isclose(abs_sum, float(sum(abs(Fraction(float(a[i])) * Fraction(float(b[ind[i]])))
                                           for i in range(n))), rel_tol=1e-12)
    plain = O.gather_sum("SCP", "IND", n, b, a=a, ind=ind)
    assert abs(Fraction(plain) - exact) <= Fraction(n * 2.0 ** -53) * Fraction(abs_sum)
    # the ADD sum against math.fsum (correctly rounded)
    add_s, _ = O.gather_sum_exact("ADD", "IND", n, b, ind=ind)
    assert add_s == math.fsum(b[ind[:n]])


def test_bernoulli_indices_p1_is_dense():
    assert np.array_equal(S.bernoulli_indices(1000, 1.0, 3), np.arange(1000, dtype=np.int32))
    b = S.vector(1000, 3)
    assert O.gather_sum("ADD", "IND", 1000, b, ind=S.bernoulli_indices(1000, 1.0, 3)) == \
        O.gather_sum("ADD", "PD", 1000, b)


@pytest.mark.parametrize("k", [2, 8, 64])
def test_geometric_indices_follow_the_bernoulli_gap_law(k):
    """The IR arrays drawn gap by gap have the gap law of the paper's
    per-position draw: mean k, variance k(k-1), P(gap = 1) = 1/k."""
    p = 1.0 / k
    n = 200_000
    g = np.diff(np.concatenate([[-1], S.geometric_indices(n, p, 21).astype(np.int64)]))
    gb = np.diff(np.concatenate([[-1], S.bernoulli_indices(n * k, p, 22).astype(np.int64)]))
    for gaps in (g, gb):
        assert gaps.min() >= 1
        assert abs(gaps.mean() - k) < 0.02 * k
        assert abs(gaps.var() - k * (k - 1)) < 0.05 * k * k + 0.02
        assert abs(np.mean(gaps == 1) - p) < 0.01


def test_gaussian_indices_zero_variance_is_constant_stride():
    n, m = 10_000, 7
    ind = S.gaussian_indices(n, m, 0.0, 10 ** 6, 5)
    assert np.array_equal(ind, (np.arange(n, dtype=np.int64) * m % 10 ** 6).astype(np.int32))
    ind = S.gaussian_indices(n, 4.0, 400.0, 10 ** 6, 5)
    L = 10 ** 6
    steps = (np.diff(ind.astype(np.int64)) + L // 2) % L - L // 2  # undo the wrap
    assert (steps < 0).mean() > 0.3  # backward jumps appear at large variance
    assert abs(steps.mean() - 4.0) < 0.5 and abs(steps.var() - 400.0) < 20.0


# --------------------------------------------------------------------------
# Stride distribution (Sect. 4.2, Fig. 4a) and sectors per warp-wide gather
# --------------------------------------------------------------------------

def tridiagonal(n):
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
    return S.from_coo(n, n, rows, cols, np.ones(len(rows)))


def test_stride_hist_tridiagonal_closed_form():
    """CRS of a tridiagonal matrix read row by row: every jump inside a row
    is +1 (2n-2 of them) and every row change jumps back by 1 (n-1)."""
    n = 1000
    fwd, bwd = O.stride_hist(tridiagonal(n).col)
    assert fwd[1] == 2 * n - 2 and fwd.sum() == 2 * n - 2
    assert bwd[1] == n - 1 and bwd.sum() == n - 1


def test_stride_hist_power_of_two_bins():
    col = np.array([2 ** b - 1 for b in range(31)], dtype=np.int32)  # jumps 1, 2, 4, ..., 2^29
    fwd, bwd = O.stride_hist(col)
    assert list(fwd) == [0] + [1] * 30 + [0, 0] and bwd.sum() == 0
    fwd, bwd = O.stride_hist(col[::-1].copy())
    assert list(bwd) == [0] + [1] * 30 + [0, 0] and fwd.sum() == 0
    fwd, bwd = O.stride_hist(np.array([5, 5, 5, 4, 7], dtype=np.int32))  # 0, 0, -1, +3
    assert fwd[0] == 2 and fwd[2] == 1 and bwd[1] == 1 and fwd.sum() + bwd.sum() == 4
    # extremes of int32: one jump of 2^31 - 1 and one of -(2^31 - 1)
    fwd, bwd = O.stride_hist(np.array([0, 2 ** 31 - 1, 0], dtype=np.int32))
    assert fwd[31] == 1 and bwd[31] == 1


def test_warp_sectors_identity_closed_form():
    """A warp reading 32 consecutive aligned FP64 entries touches 256 bytes,
    i.e. 8 sectors (4 for FP32), in CRS with one lane per row, JDS and SELL."""
    n = 32 * 50
    A = S.from_coo(n, n, np.arange(n), np.arange(n), np.ones(n))
    for h in (O.warp_sectors_crs(A, 1), O.warp_sectors_jds(O.jds_build(A, True)),
              O.warp_sectors_sell(O.sell_build(A, 64, True))):
        assert h[8] == n // 32 and h.sum() == n // 32
    assert O.warp_sectors_crs(A, 1, elem_bytes=4)[4] == n // 32


def test_warp_sectors_crs_lanes_closed_forms():
    """Rows of 64 consecutive columns starting at multiples of 64: with 32
    lanes a row is read in two accesses of 8 sectors; with 8 lanes a warp
    reads 4 rows x 8 consecutive columns = 4 x 2 sectors per access.  Rows
    whose columns are 1000 apart: every lane its own sector."""
    n_rows = 40
    rows = np.repeat(np.arange(n_rows), 64)
    cols = (np.arange(n_rows)[:, None] * 64 + np.arange(64)[None, :]).ravel()
    A = S.from_coo(n_rows, 64 * n_rows, rows, cols, np.ones(len(rows)))
    h32 = O.warp_sectors_crs(A, 32)
    assert h32[8] == 2 * n_rows and h32.sum() == 2 * n_rows
    h8 = O.warp_sectors_crs(A, 8)
    assert h8[8] == (n_rows // 4) * 8 and h8.sum() == (n_rows // 4) * 8
    cols = (np.arange(n_rows)[:, None] * 32000 + np.arange(32)[None, :] * 1000).ravel()
    B = S.from_coo(n_rows, 32000 * n_rows, np.repeat(np.arange(n_rows), 32), cols, np.ones(32 * n_rows))
    h = O.warp_sectors_crs(B, 32)
    assert h[32] == n_rows and h.sum() == n_rows


def test_warp_sectors_sell_one_window_is_jds():
    """With one window SELL-32 reads, per 32-row block and slot, exactly the
    rows and columns the thread-per-row JDS walk reads per warp and
    diagonal (two loops over two different layouts)."""
    A = S.small_random(700, 700, 5, density=0.02)
    for sym in (True, False):
        hj = O.warp_sectors_jds(O.jds_build(A, sym))
        hs = O.warp_sectors_sell(O.sell_build(A, 704, sym))
        assert np.array_equal(hj, hs)
        assert hj.sum() > 0


def test_warp_sectors_crs_one_lane_equal_rows_is_jds():
    """Rows of equal length keep their order under the stable JDS sort, so
    the row-only JDS warp walk and CRS with one lane per row coincide."""
    n = 64 * 5
    rows = np.repeat(np.arange(n), 3)
    cols = ((np.arange(n)[:, None] + np.array([0, 97, 1003])[None, :]) % n).ravel()
    A = S.from_coo(n, n, rows, cols, np.ones(3 * n))
    assert np.array_equal(O.warp_sectors_crs(A, 1), O.warp_sectors_jds(O.jds_build(A, False)))


# --------------------------------------------------------------------------
# Paired SELL (a GPU layout of this library): rank q pairs with rank m-1-q
# --------------------------------------------------------------------------

def test_psell_hand_worked_example():
    """Rows of lengths 1, 3, 2, 0.  Sorted by decreasing length: rows 1, 2,
    0, 3.  Two lanes: lane 0 = (row 1, row 3), lane 1 = (row 2, row 0).
    Permuted rows: a-rows 1, 2 at 0, 1; b-rows 3, 0 at 2, 3.  Lane totals
    3 and 3; slots: t=0 (1.0, 2.0), t=1 (1.1, 2.1), t=2 (1.2, 0.0) where
    r.e is entry e of row r."""
    A = S.from_coo(4, 4, [0, 1, 1, 1, 2, 2], [0, 0, 1, 3, 2, 3], [1., 2, 3, 4, 5, 6])
    P = O.psell_build(A, 64, False)
    assert list(P.perm) == [1, 2, 3, 0]
    assert list(P.rlen) == [3, 2, 0, 1]
    assert list(P.blk_ptr) == [0, 6]
    assert list(P.col) == [0, 2, 1, 3, 3, 0]
    assert list(P.val) == [2., 5., 3., 6., 4., 1.]
    P = O.psell_build(A, 64, True)
    assert list(P.col) == [3, 1, 0, 2, 2, 3]  # iperm = [3, 0, 1, 2]


def test_psell_equal_lengths_closed_form():
    """Equal row lengths keep their order under the stable sort, so lane q
    of a full 64-row window pairs rows q and 63-q."""
    n = 64 * 3 + 10
    A = S.from_coo(n, n, np.repeat(np.arange(n), 2), np.stack([np.arange(n), (np.arange(n) + 5) % n], 1).ravel(),
                   np.ones(2 * n))
    P = O.psell_build(A, 64, False)
    for g in range(3):
        assert list(P.perm[64 * g:64 * g + 32]) == list(range(64 * g, 64 * g + 32))
        assert list(P.perm[64 * g + 32:64 * g + 64]) == list(range(64 * g + 63, 64 * g + 31, -1))
    # last window, 10 rows: 5 lanes (q, 9-q)
    assert list(P.perm[192:]) == [192, 193, 194, 195, 196, 201, 200, 199, 198, 197]
    assert np.array_equal(np.diff(P.blk_ptr), [128, 128, 128, 20])


@pytest.mark.parametrize("window", [64, 128, 256])
@pytest.mark.parametrize("n", [1, 63, 64, 65, 129, 1000])
def test_psell_product_and_invariants(window, n):
    A = S.small_random(n, n, 40 + n, density=min(0.5, 12.0 / n), empty_rows=0.1)
    for sym in (True, False):
        P = O.psell_build(A, window, sym)
        assert np.array_equal(np.sort(P.perm), np.arange(n))
        assert np.array_equal(P.iperm[P.perm], np.arange(n))
        assert all(P.perm[w0:w0 + window].min() >= w0 and P.perm[w0:w0 + window].max() < w0 + window
                   for w0 in range(0, n, window))
        assert P.rlen.sum() == A.nnz and P.blk_ptr[-1] == A.nnz
        x = S.vector(n, 3)
        xp = x[P.perm] if sym else x
        y = np.zeros(n)
        y[P.perm] = O.psell_spmv(P, xp)
        ref = A.to_dense() @ x
        s = np.abs(A.to_dense()) @ np.abs(x)
        assert np.all(np.abs(y - ref) <= 1e-13 * s + 1e-300)
        Ai = S.integer_values(A, 9, 1000)
        xi = S.int_vector(n, 10, 1000)
        Pi = O.psell_build(Ai, window, sym)
        yi = np.zeros(n)
        yi[Pi.perm] = O.psell_spmv(Pi, xi[Pi.perm] if sym else xi)
        assert np.array_equal(yi, (Ai.to_dense().astype(np.int64) @ xi.astype(np.int64)).astype(np.float64))


def test_psell_pairs_long_with_short():
    """In a full window the a-row of each lane is at least as long as its
    b-row, and lane totals vary less than row lengths (the point of it)."""
    A = S.hh_like(20_000, 1)
    P = O.psell_build(A, 64, False)
    a = P.rlen.reshape(-1, 64)[:, :32] if len(P.rlen) % 64 == 0 else P.rlen[:len(P.rlen) // 64 * 64].reshape(-1, 64)[:, :32]
    b = P.rlen[:len(P.rlen) // 64 * 64].reshape(-1, 64)[:, 32:]
    assert np.all(a >= b)
    tot = a + b
    assert tot.std(axis=1).mean() < 0.5 * P.rlen[:len(P.rlen) // 64 * 64].reshape(-1, 64).std(axis=1).mean()


# --------------------------------------------------------------------------
# Symmetric SpMVM from the upper triangle (Sect. 4.2's unused symmetry)
# --------------------------------------------------------------------------

def symmetric_random(n, seed, density):
    B = S.small_random(n, n, seed, density=density)
    D = B.to_dense()
    D = D + D.T  # symmetric values
    r, c = np.nonzero(D)
    return S.from_coo(n, n, r, c, D[r, c])


def test_upper_extract_is_triu():
    A = symmetric_random(300, 5, 0.03)
    U = O.upper(A)
    Ud = np.zeros((300, 300))
    rows = np.repeat(np.arange(300), np.diff(U.row_ptr))
    Ud[rows, U.col] = U.val
    assert np.array_equal(Ud, np.triu(A.to_dense()))
    assert U.nnz == np.count_nonzero(np.triu(A.to_dense()))


@pytest.mark.parametrize("n", [1, 2, 57, 300])
def test_sym_spmv_equals_full_product(n):
    A = symmetric_random(n, 6 + n, min(0.5, 8.0 / n))
    x = S.vector(n, 7)
    U = O.upper(A)
    y = O.sym_spmv(U, x)
    D = A.to_dense()
    assert np.all(np.abs(y - D @ x) <= 1e-14 * (np.abs(D) @ np.abs(x)) + 1e-300)
    Ai = S.integer_values(A, 8, 1000)
    Di = Ai.to_dense()
    Di = np.triu(Di) + np.triu(Di, 1).T  # integer symmetric values
    r, c = np.nonzero(Di)
    Ai = S.from_coo(n, n, r, c, Di[r, c])
    xi = S.int_vector(n, 9, 1000)
    assert np.array_equal(O.sym_spmv(O.upper(Ai), xi), (Di.astype(np.int64) @ xi.astype(np.int64)).astype(float))


def test_sym_spmv_hh_like_matches_crs():
    """The HH-like stand-in is symmetric by construction (mirrored pattern,
    equal values): the upper-triangle product equals the full CRS product."""
    A = S.hh_like(20_000, 1)
    x = S.vector(A.n_rows, 3)
    ref, s = O.crs_spmv_exact(A, x)
    U = O.upper(A)
    assert 2 * U.nnz - A.n_rows == A.nnz  # every off-diagonal entry has its mirror
    assert np.all(np.abs(O.sym_spmv(U, x) - ref) <= 1e-14 * s)


# --------------------------------------------------------------------------
# Hybrid storage: dense secondary diagonals in DIA form + remainder CRS
# (Sect. 4.2 names the dense secondary diagonals as candidates for dense storage)
# --------------------------------------------------------------------------

def dense_of(offs, dia, rem, n_cols):
    n = rem.n_rows
    D = np.zeros((n, n_cols))
    for k, o in enumerate(offs):
        for i in range(n):
            if 0 <= i + o < n_cols:
                D[i, i + o] += dia[k, i]
    rows = np.repeat(np.arange(n), np.diff(rem.row_ptr))
    np.add.at(D, (rows, rem.col), rem.val)
    return D


def test_dia_laplacian_closed_form():
    """nx x ny Laplacian: diagonal n entries, offsets +-1 hold (nx-1) ny,
    offsets +-nx hold n - nx; all five are full enough, nothing remains,
    and on integer data the product is exact."""
    nx, ny = 12, 9
    A = S.laplace2d(nx, ny)
    n = nx * ny
    offs = O.dia_select(A, 8, 0.5)
    assert list(offs) == [0, -1, 1, -nx, nx]  # counts n, (nx-1)ny twice, n-nx twice
    dia, rem = O.dia_build(A, offs)
    assert rem.nnz == 0
    assert np.array_equal(dense_of(offs, dia, rem, n), A.to_dense())
    assert np.count_nonzero(dia[1]) == (nx - 1) * ny and np.count_nonzero(dia[3]) == n - nx
    x = S.int_vector(n, 3, 1000)
    assert np.array_equal(O.dia_spmv(offs, dia, rem, x), A.to_dense() @ x)


def test_dia_none_selected_is_crs():
    A = S.small_random(200, 150, 4, density=0.05, empty_rows=0.2)
    offs = O.dia_select(A, 8, 1.01)  # no diagonal can be fuller than 1
    assert len(offs) == 0
    dia, rem = O.dia_build(A, offs)
    assert np.array_equal(rem.row_ptr, A.row_ptr) and np.array_equal(rem.col, A.col)
    x = S.vector(150, 5)
    assert np.array_equal(O.dia_spmv(offs, dia, rem, x), O.crs_spmv(A, x))


def test_dia_planted_diagonals_and_duplicates():
    """Planted diagonals of fill 0.9 are found (and a sparse band is not);
    DIA + remainder reproduce A, including a duplicated entry whose second
    copy stays in the remainder."""
    n = 400
    rng_rows, rng_cols, vals = [], [], []
    for k, o in enumerate((-50, 7, 123)):
        i = np.arange(max(0, -o), min(n, n - o))
        keep = S.uniform01(6, 40 + k, i) < 0.9
        rng_rows += list(i[keep]); rng_cols += list(i[keep] + o)
    i = np.arange(n)
    j = S.randint(6, 50, i, 0, n - 1)
    rng_rows += list(i); rng_cols += list(j)
    vals = S.uniform(6, 51, np.arange(len(rng_rows)), -1, 1)
    A = S.from_coo(n, n, rng_rows, rng_cols, vals, dedupe=False)
    offs = O.dia_select(A, 8, 0.7)
    assert sorted(offs) == [-50, 7, 123]
    dia, rem = O.dia_build(A, offs)
    assert np.allclose(dense_of(offs, dia, rem, n), _dense_sum(A), rtol=0, atol=1e-15)
    x = S.vector(n, 7)
    ref, s = O.crs_spmv_exact(A, x)
    assert np.all(np.abs(O.dia_spmv(offs, dia, rem, x) - ref) <= 1e-14 * s)


def _dense_sum(A):
    D = np.zeros((A.n_rows, A.n_cols))
    np.add.at(D, (A.row_ids(), A.col), A.val)
    return D


def test_dia_hh_diagonals_selects_the_outer_diagonals():
    A = S.hh_diagonals(200_000, 5)
    offs = O.dia_select(A, 16, 2.0 / 3.0)
    inside = [o for o in S.HH_OUTER_OFFSETS if o < A.n_rows]  # 65536, 131072, 196608
    assert sorted(np.abs(offs[1:]).tolist()) == sorted(2 * inside)
    assert offs[0] == 0
    dia, rem = O.dia_build(A, offs)
    assert rem.nnz + np.count_nonzero(dia) == A.nnz
    x = S.vector(A.n_rows, 8)
    ref, s = O.crs_spmv_exact(A, x)
    assert np.all(np.abs(O.dia_spmv(offs, dia, rem, x) - ref) <= 1e-14 * s)
