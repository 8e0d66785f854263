"""Adjoint, value gradient and autograd on the GPU against the oracle."""
import math

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


@pytest.mark.parametrize("maker", [lambda: S.hh_like(50_000, 71), lambda: S.zipf_rows(40_000, 72, lmax=3000),
                                   lambda: S.small_random(300, 77, 73, density=0.1, empty_rows=0.2),
                                   lambda: S.stencil27(20, 4)])
def test_transpose_structure_bit_exact(maker):
    A = maker()
    M = crs(A)
    T = M.transpose()
    # reference: stable sort of the entries by column (numpy), rows in entry order
    order = np.argsort(A.col, kind="stable")
    rp = np.zeros(A.n_cols + 1, np.int64)
    np.cumsum(np.bincount(A.col, minlength=A.n_cols), out=rp[1:])
    assert np.array_equal(host(T.row_ptr), rp)
    assert np.array_equal(host(T.tmap), order)
    assert np.array_equal(host(T.col), A.row_ids()[order])
    assert np.array_equal(host(T.val), A.val[order])


@pytest.mark.parametrize("maker", [lambda: S.hh_like(60_000, 74), lambda: S.zipf_rows(40_000, 75, lmax=2000),
                                   lambda: S.small_random(300, 77, 76, density=0.1, empty_rows=0.2)])
def test_adjoint_against_oracle(maker):
    A = maker()
    g = S.vector(A.n_rows, 77)
    ref, s = O.crs_spmv_t_exact(A, g)
    M = crs(A)
    M.transpose()
    assert_close64(host(M.spmv(dev(g), transpose=True)), ref, s, "A^T g (CRS of transpose)")
    # transposed JDS: a JDS of the transposed structure attached as the adjoint
    T = M._transpose
    JT = T.to_jds("NUJDS", "row_only", unroll=4)
    M.attach_transpose(JT)
    assert_close64(host(M.spmv(dev(g), transpose=True, basis=1)), ref, s, "A^T g (transposed JDS)")
    # dot-product identity <A^T g, x> = <g, A x>
    x = S.vector(A.n_cols, 78)
    M.attach_transpose(T)
    lhs = math.fsum(host(M.spmv(dev(g), transpose=True)) * x)
    rhs = math.fsum(g * host(M.spmv(dev(x))))
    scale = math.fsum(np.abs(g) * (np.abs(A.to_dense()) @ np.abs(x))) if A.n_rows < 1000 else \
        math.fsum(np.abs(g) * O.crs_spmv_exact(S.CRS(A.n_rows, A.n_cols, A.row_ptr, A.col, np.abs(A.val)),
                                              np.abs(x))[0])
    assert abs(lhs - rhs) <= 1e-13 * scale


def test_adjoint_integer_bit_exact_and_value_refresh():
    A = S.integer_values(S.zipf_rows(30_000, 79, lmax=1000), 79, 512)
    g = S.int_vector(A.n_rows, 79, 512)
    M = crs(A)
    M.transpose()
    assert np.array_equal(host(M.spmv(dev(g), transpose=True)), O.crs_spmv_t(A, g))
    # new values, same pattern: refresh the gathered transposed values
    B = S.integer_values(A, 80, 256)
    newval = dev(B.val)
    M.set_values(newval)
    M.refresh_transpose_values()
    assert np.array_equal(host(M.spmv(dev(g), transpose=True)), O.crs_spmv_t(B, g))


def test_dval_and_multi():
    A = S.hh_like(40_000, 81)
    g = S.vector(A.n_rows, 81)
    x = S.vector(A.n_cols, 82)
    M = crs(A)
    d = host(M.dval(dev(g), dev(x)))
    assert np.array_equal(d, O.dval(A, g, x))  # fma(g, x, 0) is the rounded product
    # accumulate: one fma onto the old value
    d0 = S.vector(A.nnz, 83)
    d2 = host(M.dval(dev(g), dev(x), out=dev(d0), accumulate=True))
    rid = A.row_ids()
    np.testing.assert_allclose(d2, d0 + g[rid] * x[A.col], rtol=0, atol=4e-16)
    # multi: m pairs in one pass == sum of single calls, in a fixed order
    m = 5
    G = np.stack([S.vector(A.n_rows, 90 + t) for t in range(m)], axis=1)
    X = np.stack([S.vector(A.n_cols, 95 + t) for t in range(m)], axis=1)
    dm = host(M.dval_multi(dev(G), dev(X)))
    ref = sum(G[rid, t] * X[A.col, t] for t in range(m))
    np.testing.assert_allclose(dm, ref, rtol=0, atol=1e-15 * m)
    # splitting t over calls gives identical bits
    out = torch.zeros(A.nnz, dtype=torch.float64, device="cuda")
    M.dval_multi(dev(G[:, :2].copy()), dev(X[:, :2].copy()), out=out, accumulate=True)
    M.dval_multi(dev(G[:, 2:].copy()), dev(X[:, 2:].copy()), out=out, accumulate=True)
    assert np.array_equal(host(out).view(np.int64), dm.view(np.int64))
    # the same pairs laid out column-major (m contiguous vectors) through the
    # strided entry point: identical bits
    Gc = torch.as_tensor(np.ascontiguousarray(G.T), device="cuda").t()
    Xc = torch.as_tensor(np.ascontiguousarray(X.T), device="cuda").t()
    assert Gc.stride() == (1, A.n_rows) and Xc.stride() == (1, A.n_cols)
    dc = host(M.dval_multi(Gc, Xc))
    assert np.array_equal(dc.view(np.int64), dm.view(np.int64))


@pytest.mark.parametrize("idx", range(9))
def test_dval_edge_matrices(idx):
    """The one-step value gradient finds each entry's row from the warp's
    row starts: empty rows, rows of one entry, rows longer than a warp's
    chunks, a ragged last block and rectangular shapes, bit for bit."""
    from gpu_util import adversarial_matrices
    A = adversarial_matrices()[idx]
    if A.nnz == 0:
        return
    g = S.vector(A.n_rows, 300 + idx)
    x = S.vector(A.n_cols, 310 + idx)
    M = crs(A)
    assert np.array_equal(host(M.dval(dev(g), dev(x))), O.dval(A, g, x)), A.name
    d0 = S.vector(A.nnz, 320 + idx)
    d2 = host(M.dval(dev(g), dev(x), out=dev(d0), accumulate=True))
    rid = A.row_ids()
    # one fma onto the old value against a product and a sum, each rounded
    # (|g x|, |d0| <= 1): within half an ulp of 1 plus one ulp of 2
    np.testing.assert_allclose(d2, d0 + g[rid] * x[A.col], rtol=0, atol=6e-16, err_msg=A.name)


def _pattern(A, **kw):
    from paper_0910_4836_gb300.autograd import Pattern
    return Pattern.from_host(A, **kw)


@pytest.mark.parametrize("adjoint", ["crs", "jds", "sell"])
def test_spmv_function_gradcheck(adjoint):
    from paper_0910_4836_gb300.autograd import spmv
    A = S.small_random(30, 25, 84, density=0.2)
    p = _pattern(A, adjoint=adjoint)
    val = dev(A.val).requires_grad_(True)
    x = dev(S.vector(25, 84)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v, xx: spmv(p, v, xx), (val, x), eps=1e-6, atol=1e-9)


@pytest.mark.parametrize("adjoint,forward", [("crs", "crs"), ("jds", "jds"), ("sell", "sell"), ("auto", "auto")])
def test_power_gradients_against_oracle(adjoint, forward):
    from paper_0910_4836_gb300.autograd import power_apply
    A = S.stencil27(8, 4)
    x = S.vector(A.n_cols, 85)
    m = 6
    L_ref, dv_ref, dx_ref = O.power_loss_grad(A, x, m)
    p = _pattern(A, adjoint=adjoint, forward=forward)
    grads = []
    for c in (1, 2, 4, 6):
        val = dev(A.val).requires_grad_(True)
        xx = dev(x).requires_grad_(True)
        y = power_apply(p, val, xx, m, checkpoint=c)
        loss = (y * y).sum()
        loss.backward()
        assert abs(loss.item() - L_ref) <= 1e-12 * abs(L_ref)
        dv, dx = host(val.grad), host(xx.grad)
        np.testing.assert_allclose(dv, dv_ref, rtol=1e-11, atol=1e-14 * np.abs(dv_ref).max())
        np.testing.assert_allclose(dx, dx_ref, rtol=1e-11, atol=1e-14 * np.abs(dx_ref).max())
        grads.append((dv, dx))
    # recomputation is deterministic: identical bits for every interval
    for dv, dx in grads[1:]:
        assert np.array_equal(dv.view(np.int64), grads[0][0].view(np.int64))
        assert np.array_equal(dx.view(np.int64), grads[0][1].view(np.int64))


def test_power_gradient_finite_differences_and_closed_form():
    from paper_0910_4836_gb300.autograd import power_apply
    A = S.stencil27(6, 4, symmetric_values=True)
    x = S.vector(A.n_cols, 86)
    m = 3
    p = _pattern(A)
    val = dev(A.val).requires_grad_(True)
    xx = dev(x).requires_grad_(True)
    y = power_apply(p, val, xx, m, checkpoint=2)
    (y * y).sum().backward()
    # symmetric A: dL/dx = 2 A^{2m} x
    closed = 2 * O.power_forward(A, x, 2 * m)[-1]
    np.testing.assert_allclose(host(xx.grad), closed, rtol=1e-12, atol=1e-15)

    def loss(v):
        with torch.no_grad():
            yy = power_apply(p, v, dev(x), m)
            return float((yy * yy).sum())

    h = 1e-6
    for t in range(3):
        dvec = S.uniform(86, 100 + t, np.arange(A.nnz), -1, 1)
        fd = (loss(dev(A.val + h * dvec)) - loss(dev(A.val - h * dvec))) / (2 * h)
        an = float(np.dot(host(val.grad), dvec))
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_fp32_power_gradient_error_stated():
    from paper_0910_4836_gb300.autograd import power_apply
    A = S.stencil27(10, 4)
    x = S.vector(A.n_cols, 87)
    m = 5
    _, dv_ref, dx_ref = O.power_loss_grad(A, x, m)
    p = _pattern(A, dtype=torch.float32)
    val = dev(A.val.astype(np.float32)).requires_grad_(True)
    xx = dev(x.astype(np.float32)).requires_grad_(True)
    y = power_apply(p, val, xx, m, checkpoint=2)
    (y * y).sum().backward()
    rel_v = np.abs(host(val.grad) - dv_ref).max() / np.abs(dv_ref).max()
    rel_x = np.abs(host(xx.grad) - dx_ref).max() / np.abs(dx_ref).max()
    assert rel_v < 1e-5 and rel_x < 1e-5, (rel_v, rel_x)
