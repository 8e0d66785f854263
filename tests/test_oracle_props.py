"""Property-based pins of the oracle: random small matrices, every layout
checked against plain dense numpy and exact integer arithmetic."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
from paper_0910_4836_gb300 import synth as S  # noqa: E402


@st.composite
def int_matrices(draw, square=True):
    n = draw(st.integers(1, 40))
    m = n if square else draw(st.integers(1, 40))
    density = draw(st.sampled_from([0.0, 0.05, 0.2, 0.6]))
    seed = draw(st.integers(0, 10_000))
    A = S.small_random(n, m, seed, density=density) if density > 0 else \
        S.CRS(n, m, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")
    return S.integer_values(A, seed + 1, 1000) if A.nnz else A


def dense_int(A):
    return A.to_dense().astype(np.int64)


SETTINGS = settings(max_examples=60, deadline=None)


@SETTINGS
@given(int_matrices(square=False), st.integers(0, 1000))
def test_crs_loop_is_the_dense_product(A, seed):
    x = S.int_vector(A.n_cols, seed, 1000)
    assert np.array_equal(O.crs_spmv(A, x), (dense_int(A) @ x.astype(np.int64)).astype(float))


@SETTINGS
@given(int_matrices(), st.booleans(), st.integers(0, 1000))
def test_jds_family_products_match(A, sym, seed):
    x = S.int_vector(A.n_cols, seed, 1000)
    ref = (dense_int(A) @ x.astype(np.int64)).astype(float)
    J = O.jds_build(A, sym)
    assert np.array_equal(np.sort(J.perm), np.arange(A.n_rows))
    xp = O.permute(J.perm, x) if sym else x
    for y_p in (O.jds_spmv(J, xp), O.nbjds_spmv(J, xp, 3), O.nujds_spmv(J, xp, 2)):
        y = np.zeros(A.n_rows)
        y[J.perm] = y_p
        assert np.array_equal(y, ref)
    bp, c, v = O.rbjds_build(J, 4)
    y = np.zeros(A.n_rows)
    y[J.perm] = O.rbjds_spmv(J, bp, c, v, 4, xp)
    assert np.array_equal(y, ref)


@SETTINGS
@given(int_matrices(), st.booleans(), st.sampled_from([32, 64, 128]), st.integers(0, 1000))
def test_sell_and_paired_sell_match(A, sym, window, seed):
    x = S.int_vector(A.n_cols, seed, 1000)
    ref = (dense_int(A) @ x.astype(np.int64)).astype(float)
    G = O.sell_build(A, window, sym)
    y = np.zeros(A.n_rows)
    y[G.perm] = O.sell_spmv(G, x[G.perm] if sym else x)
    assert np.array_equal(y, ref)
    if window % 64 == 0:
        P = O.psell_build(A, window, sym)
        y = np.zeros(A.n_rows)
        y[P.perm] = O.psell_spmv(P, x[P.perm] if sym else x)
        assert np.array_equal(y, ref)
        assert P.blk_ptr[-1] == A.nnz


@SETTINGS
@given(int_matrices(), st.integers(1, 8), st.sampled_from([0.3, 0.6, 0.9]), st.integers(0, 1000))
def test_dia_hybrid_reconstructs(A, max_diags, min_fill, seed):
    offs = O.dia_select(A, max_diags, min_fill)
    dia, rem = O.dia_build(A, offs)
    x = S.int_vector(A.n_cols, seed, 1000)
    assert np.array_equal(O.dia_spmv(offs, dia, rem, x), (dense_int(A) @ x.astype(np.int64)).astype(float))
    # DIA + remainder hold exactly the matrix
    D = np.zeros((A.n_rows, A.n_cols))
    for k, o in enumerate(offs):
        for i in range(A.n_rows):
            if 0 <= i + o < A.n_cols:
                D[i, i + o] += dia[k, i]
    np.add.at(D, (np.repeat(np.arange(A.n_rows), np.diff(rem.row_ptr)), rem.col), rem.val)
    assert np.array_equal(D, A.to_dense()) and rem.nnz <= A.nnz


@SETTINGS
@given(int_matrices())
def test_stride_hist_counts_every_jump(A):
    fwd, bwd = O.stride_hist(A.col)
    assert fwd.sum() + bwd.sum() == max(A.nnz - 1, 0)
    steps = np.diff(A.col.astype(np.int64))
    assert bwd.sum() == (steps < 0).sum() and fwd[0] == (steps == 0).sum()


@SETTINGS
@given(st.integers(1, 3000), st.integers(1, 9), st.integers(0, 1000))
def test_gather_sums_exact_on_integers(n, k, seed):
    b = S.int_vector(k * n, seed, 1000)
    a = S.int_vector(n, seed + 1, 1000)
    ind = S.stride_indices(n, k)
    ref = int((a.astype(np.int64) * b[::k][:n].astype(np.int64)).sum())
    assert O.gather_sum("SCP", "CS", n, b, a=a, k=k) == ref
    assert O.gather_sum("SCP", "IND", n, b, a=a, ind=ind) == ref
    assert O.gather_sum_exact("SCP", "IND", n, b, a=a, ind=ind)[0] == ref


@SETTINGS
@given(int_matrices(square=False), st.integers(1, 6), st.integers(0, 1000))
def test_spmm_and_exact_spmm_are_dense_products(A, k, seed):
    """Every column of the SpMM loops, plain and exact (with its Σ|a||x|), is
    the dense integer product."""
    X = np.stack([S.int_vector(A.n_cols, seed + c, 1000) for c in range(k)], axis=1)
    D = dense_int(A)
    ref = (D @ X.astype(np.int64)).astype(float)
    assert np.array_equal(O.crs_spmm(A, X), ref)
    Y, Sabs = O.crs_spmm_exact(A, X)
    assert np.array_equal(Y, ref)
    assert np.array_equal(Sabs, (np.abs(D) @ np.abs(X.astype(np.int64))).astype(float))


@SETTINGS
@given(int_matrices(square=False), st.integers(0, 1000))
def test_adjoint_and_dval_are_their_definitions(A, seed):
    """A^T g is the dense transposed product; dval_k = g[row_k] x[col_k]."""
    g = S.int_vector(A.n_rows, seed, 1000)
    x = S.int_vector(A.n_cols, seed + 1, 1000)
    D = dense_int(A)
    assert np.array_equal(O.crs_spmv_t(A, g), (D.T @ g.astype(np.int64)).astype(float))
    t, st_ = O.crs_spmv_t_exact(A, g)
    assert np.array_equal(t, (D.T @ g.astype(np.int64)).astype(float))
    rid = A.row_ids().astype(np.int64)
    want = (g.astype(np.int64)[rid] * x.astype(np.int64)[A.col]).astype(float)
    assert np.array_equal(O.dval(A, g, x), want)


@SETTINGS
@given(int_matrices(square=False), st.integers(0, 1000))
def test_fp32_loop_exact_below_2_24(A, seed):
    """With |a|, |x| <= 64 and at most 40 entries a row every partial sum is
    an integer below 2^24, so the FP32 loop is exact."""
    Ai = S.integer_values(A, seed, 64) if A.nnz else A
    x = S.int_vector(A.n_cols, seed + 2, 64)
    ref = (dense_int(Ai) @ x.astype(np.int64))
    assert np.abs(ref).max(initial=0) < 2 ** 24
    assert np.array_equal(O.crs_spmv_f32(Ai, x), ref.astype(np.float32))
