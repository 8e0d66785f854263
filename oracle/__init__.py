"""CPU oracle for CRS / JDS sparse matrix-vector multiplication.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark -- never by the product library, which
shares no code with it.

Thin numpy wrappers around the plain C loops in ``oracle.c`` (Schubert, Hager
& Fehske, Sect. 2), plus the power-iteration gradient written out with the
chain rule.  Everything is FP64 unless the name says otherwise.

Pins (see tests/test_oracle.py): dense matvec on tiny matrices, exact
rational sums, identity / diagonal / integer inputs, Laplacian closed forms,
the JDS special cases the paper states (NUJDS with u = N_j is CRS in the
permuted basis; RBJDS with block 1 is row-by-row access; JDS is NBJDS with
block = N), a hand-worked JDS example, the adjoint identity and finite
differences; the basic gather sums of Sect. 4.1 against closed forms
(dense and constant-stride sums of integers), exact rational sums and
math.fsum, with the IR index law checked against the paper's per-position
draw.  SOJDS: parity unpinned (the paper fixes no sorting rule), only
invariants and a closed-form banded case.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None

_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_F64 = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_F32 = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I64 = ctypes.c_int64
_INT = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "orc_crs_spmv": [_I64, _I32, _I32, _F64, _F64, _F64, _INT],
            "orc_crs_spmv_f32": [_I64, _I32, _I32, _F32, _F32, _F32, _INT],
            "orc_crs_spmv_omp": [_I64, _I32, _I32, _F64, _F64, _F64, _INT],
            "orc_crs_spmm": [_I64, _I32, _I32, _F64, _I64, _F64, _I64, _F64, _I64, _INT],
            "orc_crs_spmv_exact": [_I64, _I32, _I32, _F64, _F64, _F64, _F64, _INT],
            "orc_crs_spmv_t_exact": [_I64, _I64, _I32, _I32, _F64, _F64, _F64, _F64],
            "orc_crs_spmv_t": [_I64, _I64, _I32, _I32, _F64, _F64, _F64, _INT],
            "orc_dval": [_I64, _I32, _I32, _F64, _F64, _F64, _INT],
            "orc_max_row_len": [_I64, _I32],
            "orc_jds_build": [_I64, _I64, _I32, _I32, _F64, _INT, _I32, _I32, _I32, _I32, _F64],
            "orc_jds_spmv": [_I64, _I64, _I32, _I32, _F64, _F64, _F64, _INT],
            "orc_nbjds_spmv": [_I64, _I64, _I32, _I32, _F64, _I64, _F64, _F64, _INT],
            "orc_nujds_spmv": [_I64, _I64, _I32, _I32, _F64, _I64, _F64, _F64, _INT],
            "orc_rbjds_build": [_I64, _I64, _I32, _I32, _F64, _I64, _I32, _I32, _F64],
            "orc_rbjds_spmv": [_I64, _I64, _I32, _I32, _I32, _F64, _I64, _F64, _F64, _INT],
            "orc_sojds_build": [_I64, _I64, _I32, _I32, _F64, _I64, _I32, _I32, _F64],
            "orc_permute": [_I64, _I32, _F64, _F64, _INT],
            "orc_sell_build": [_I64, _I64, _I32, _I32, _F64, _INT, _I64, _I32, _I32, _I32, _I32, _I32,
                               _F64],
            "orc_sell_spmv": [_I64, _I32, _I32, _I32, _F64, _F64, _F64],
            "orc_gather_sum": [_INT, _INT, _I64, _I64, _F64, _F64, _I32],
            "orc_gather_sum_exact": [_INT, _INT, _I64, _I64, _F64, _F64, _I32, _F64],
            "orc_psell_build": [_I64, _I64, _I32, _I32, _F64, _INT, _I64, _I32, _I32, _I32, _I32, _I32,
                                _F64],
            "orc_psell_spmv": [_I64, _I32, _I32, _I32, _F64, _F64, _F64],
            "orc_upper_count": [_I64, _I32, _I32],
            "orc_upper_extract": [_I64, _I32, _I32, _F64, _I32, _I32, _F64],
            "orc_sym_spmv": [_I64, _I32, _I32, _F64, _F64, _F64],
            "orc_dia_select": [_I64, _I64, _I32, _I32, _I64, ctypes.c_double, _I32],
            "orc_dia_build": [_I64, _I32, _I32, _F64, _I64, _I32, _F64, _I32, _I32, _F64],
            "orc_dia_spmv": [_I64, _I64, _I64, _I32, _F64, _I32, _I32, _F64, _F64, _F64],
            "orc_stride_hist": [_I64, _I32, _I64P],
            "orc_warp_sectors_crs": [_I64, _I32, _I32, _INT, _INT, _I64P],
            "orc_warp_sectors_jds": [_I64, _I64, _I32, _I32, _INT, _I64P],
            "orc_warp_sectors_sell": [_I64, _I32, _I32, _I32, _INT, _I64P],
            "orc_num_threads": [],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _I64 if name in ("orc_max_row_len", "orc_jds_build", "orc_upper_count",
                                          "orc_dia_select", "orc_dia_build") else (
                _INT if name in ("orc_num_threads", "orc_sell_build", "orc_psell_build") else (
                    ctypes.c_double if name == "orc_gather_sum" else None))
        _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- CRS -----

def crs_spmv(A, x, y=None, accumulate=False):
    """Sect. 2 CRS loop, serial, literal order."""
    out = np.zeros(A.n_rows) if y is None else _f64(y).copy()
    lib().orc_crs_spmv(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x), out,
                       int(accumulate))
    return out


def crs_spmv_f32(A, x):
    """The CRS loop entirely in single precision."""
    out = np.zeros(A.n_rows, dtype=np.float32)
    lib().orc_crs_spmv_f32(A.n_rows, _i32(A.row_ptr), _i32(A.col),
                           np.ascontiguousarray(A.val, dtype=np.float32),
                           np.ascontiguousarray(x, dtype=np.float32), out, 0)
    return out


def crs_spmv_omp(A, x, out=None):
    """Sect. 5.2: CRS with an OpenMP static schedule (the CPU baseline)."""
    out = np.zeros(A.n_rows) if out is None else out
    lib().orc_crs_spmv_omp(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x), out, 0)
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


def crs_spmm(A, X, Y=None, accumulate=False):
    X = _f64(X)
    k = X.shape[1]
    out = np.zeros((A.n_rows, k)) if Y is None else _f64(Y).copy()
    lib().orc_crs_spmm(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(A.val), k, X, k, out, k,
                       int(accumulate))
    return out


def crs_spmv_exact(A, x, y=None, accumulate=False):
    """Accurate y = A x (Dot2 accumulation).  Returns (y, sum_j |a_ij||x_j|)."""
    out = np.zeros(A.n_rows) if y is None else _f64(y).copy()
    absrow = np.zeros(A.n_rows)
    lib().orc_crs_spmv_exact(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x),
                             out, absrow, int(accumulate))
    return out, absrow


def crs_spmm_exact(A, X):
    X = _f64(X)
    Y = np.zeros((A.n_rows, X.shape[1]))
    S = np.zeros_like(Y)
    for c in range(X.shape[1]):
        Y[:, c], S[:, c] = crs_spmv_exact(A, X[:, c])
    return Y, S


def crs_spmv_t(A, g, dx=None, accumulate=False):
    """dx = A^T g by a serial scatter over the stored entries."""
    out = np.zeros(A.n_cols) if dx is None else _f64(dx).copy()
    lib().orc_crs_spmv_t(A.n_rows, A.n_cols, _i32(A.row_ptr), _i32(A.col), _f64(A.val),
                         _f64(g), out, int(accumulate))
    return out


def crs_spmv_t_exact(A, g):
    out = np.zeros(A.n_cols)
    absc = np.zeros(A.n_cols)
    lib().orc_crs_spmv_t_exact(A.n_rows, A.n_cols, _i32(A.row_ptr), _i32(A.col), _f64(A.val),
                               _f64(g), out, absc)
    return out, absc


def dval(A, g, x, out=None, accumulate=False):
    """dval_k = g[row_k] * x[col_k]."""
    res = np.zeros(A.nnz) if out is None else _f64(out).copy()
    lib().orc_dval(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(g), _f64(x), res,
                   int(accumulate))
    return res


# ---------------------------------------------------------------- JDS -----

class JDS:
    """JDS arrays as built by :func:`jds_build`."""

    def __init__(self, n_rows, n_cols, symmetric, perm, iperm, jd_ptr, col, val):
        self.n_rows, self.n_cols, self.symmetric = n_rows, n_cols, symmetric
        self.perm, self.iperm, self.jd_ptr, self.col, self.val = perm, iperm, jd_ptr, col, val

    @property
    def n_diag(self):
        return len(self.jd_ptr) - 1

    def diag_len(self):
        return np.diff(self.jd_ptr.astype(np.int64))


def jds_build(A, symmetric=True):
    """Sect. 2 JDS construction, steps (i)-(v) (see oracle.c)."""
    rp = _i32(A.row_ptr)
    nj = int(lib().orc_max_row_len(A.n_rows, rp))
    perm = np.zeros(A.n_rows, np.int32)
    iperm = np.zeros(A.n_rows, np.int32)
    jd_ptr = np.zeros(nj + 1, np.int32)
    col = np.zeros(A.nnz, np.int32)
    val = np.zeros(A.nnz)
    r = lib().orc_jds_build(A.n_rows, A.n_cols, rp, _i32(A.col), _f64(A.val), int(symmetric),
                            perm, iperm, jd_ptr, col, val)
    if r < 0:
        raise ValueError("symmetric JDS needs a square matrix")
    return JDS(A.n_rows, A.n_cols, symmetric, perm, iperm, jd_ptr, col, val)


def jds_spmv(J, x_p, y=None, accumulate=False):
    """Sect. 2 JDS loop (diagonal-outer) in the permuted basis."""
    out = np.zeros(J.n_rows) if y is None else _f64(y).copy()
    lib().orc_jds_spmv(J.n_rows, J.n_diag, J.jd_ptr, J.col, J.val, _f64(x_p), out,
                       int(accumulate))
    return out


def nbjds_spmv(J, x_p, block):
    out = np.zeros(J.n_rows)
    lib().orc_nbjds_spmv(J.n_rows, J.n_diag, J.jd_ptr, J.col, J.val, block, _f64(x_p), out, 0)
    return out


def nujds_spmv(J, x_p, u):
    out = np.zeros(J.n_rows)
    lib().orc_nujds_spmv(J.n_rows, J.n_diag, J.jd_ptr, J.col, J.val, u, _f64(x_p), out, 0)
    return out


def n_blocks(n_rows, block):
    return (n_rows + block - 1) // block


def rbjds_build(J, block):
    """RBJDS layout: returns (blk_ptr, col_rb, val_rb)."""
    nb = n_blocks(J.n_rows, block)
    blk_ptr = np.zeros(nb + 1, np.int32)
    col = np.zeros(len(J.col), np.int32)
    val = np.zeros(len(J.val))
    lib().orc_rbjds_build(J.n_rows, J.n_diag, J.jd_ptr, J.col, J.val, block, blk_ptr, col, val)
    return blk_ptr, col, val


def rbjds_spmv(J, blk_ptr, col_rb, val_rb, block, x_p):
    out = np.zeros(J.n_rows)
    lib().orc_rbjds_spmv(J.n_rows, J.n_diag, J.jd_ptr, _i32(blk_ptr), _i32(col_rb),
                         _f64(val_rb), block, _f64(x_p), out, 0)
    return out


def sojds_build(J, block):
    """SOJDS layout (RBJDS layout with rows re-ordered by the greedy rule)."""
    nb = n_blocks(J.n_rows, block)
    blk_ptr = np.zeros(nb + 1, np.int32)
    col = np.zeros(len(J.col), np.int32)
    val = np.zeros(len(J.val))
    lib().orc_sojds_build(J.n_rows, J.n_diag, J.jd_ptr, J.col, J.val, block, blk_ptr, col, val)
    return blk_ptr, col, val


class SELL:
    """SELL-32-sigma arrays as built by :func:`sell_build`."""

    def __init__(self, n_rows, symmetric, window, perm, iperm, rlen, blk_ptr, col, val):
        self.n_rows, self.symmetric, self.window = n_rows, symmetric, window
        self.perm, self.iperm, self.rlen, self.blk_ptr, self.col, self.val = perm, iperm, rlen, blk_ptr, col, val


def sell_build(A, window, symmetric=True):
    """RBJDS with 32-row blocks and the row sort restricted to windows."""
    n = A.n_rows
    perm = np.zeros(n, np.int32)
    iperm = np.zeros(n, np.int32)
    rlen = np.zeros(n, np.int32)
    blk = np.zeros((n + 31) // 32 + 1, np.int32)
    col = np.zeros(A.nnz, np.int32)
    val = np.zeros(A.nnz)
    r = lib().orc_sell_build(n, A.n_cols, _i32(A.row_ptr), _i32(A.col), _f64(A.val), int(symmetric),
                             window, perm, iperm, rlen, blk, col, val)
    if r == -1:
        raise ValueError("symmetric permutation needs a square matrix")
    if r == -2:
        raise ValueError("window must be a positive multiple of 32")
    return SELL(n, symmetric, window, perm, iperm, rlen, blk, col, val)


def sell_spmv(S_, x_p):
    out = np.zeros(S_.n_rows)
    lib().orc_sell_spmv(S_.n_rows, S_.rlen, S_.blk_ptr, S_.col, S_.val, _f64(x_p), out)
    return out


def permute(perm, v, to_permuted=True):
    out = np.zeros(len(perm))
    lib().orc_permute(len(perm), _i32(perm), _f64(v), out, int(to_permuted))
    return out


# ------------------------------------------------- iterated products ------

def power_forward(A, x, m):
    """x_0 = x, x_t = A x_{t-1}; returns [x_0, ..., x_m]."""
    xs = [_f64(x)]
    for _ in range(m):
        xs.append(crs_spmv(A, xs[-1]))
    return xs


def power_loss_grad(A, x, m):
    """L = ||A^m x||^2 and its gradients by the chain rule:
    g_m = 2 x_m, g_{t-1} = A^T g_t, dL/dval = sum_t g_t[row] x_{t-1}[col],
    dL/dx = g_0.  Returns (L, dL/dval, dL/dx)."""
    xs = power_forward(A, x, m)
    L = float(np.dot(xs[-1], xs[-1]))
    g = 2.0 * xs[-1]
    dv = np.zeros(A.nnz)
    for t in range(m, 0, -1):
        dv = dval(A, g, xs[t - 1], dv, accumulate=True)
        g = crs_spmv_t(A, g)
    return L, dv, g


# ---------------------------------------------------------------------------
# Basic sparse vector operations (Sect. 4.1): ADD / SCP over PD, CS, IS / IR
# ---------------------------------------------------------------------------

GATHER_OPS = {"ADD": 0, "SCP": 1}
GATHER_ACCESS = {"PD": 0, "CS": 1, "IND": 2}


def gather_sum(op: str, access: str, n: int, b, a=None, k: int = 1, ind=None) -> float:
    """s = sum_i B(idx(i)) (ADD) or sum_i A(i) B(idx(i)) (SCP) in loop order,
    idx(i) = i (PD), k*i (CS) or ind(i) (IND)."""
    a_, b_, ind_ = _gather_inputs(op, access, n, b, a, k, ind)
    return float(lib().orc_gather_sum(GATHER_OPS[op], GATHER_ACCESS[access], n, k, a_, b_, ind_))


def gather_sum_exact(op: str, access: str, n: int, b, a=None, k: int = 1, ind=None):
    """(accurate sum, sum of |term|) for the same loop."""
    a_, b_, ind_ = _gather_inputs(op, access, n, b, a, k, ind)
    out = np.zeros(2)
    lib().orc_gather_sum_exact(GATHER_OPS[op], GATHER_ACCESS[access], n, k, a_, b_, ind_, out)
    return float(out[0]), float(out[1])


def _gather_inputs(op, access, n, b, a, k, ind):
    b_ = _f64(b)
    if op == "SCP":
        a_ = _f64(a)
        if len(a_) < n:
            raise ValueError("gather: A shorter than n")
    else:
        a_ = np.zeros(1)
    if access == "IND":
        ind_ = _i32(ind)
        if len(ind_) < n or (n and (ind_[:n].min() < 0 or ind_[:n].max() >= len(b_))):
            raise ValueError("gather: ind out of range")
    else:
        ind_ = np.zeros(1, dtype=np.int32)
        last = (n - 1) * (k if access == "CS" else 1)
        if n and last >= len(b_):
            raise ValueError("gather: B shorter than the strided range")
    return a_, b_, ind_


# ---------------------------------------------------------------------------
# Stride distribution (Sect. 4.2, Fig. 4a) and sectors per warp-wide gather
# ---------------------------------------------------------------------------

def stride_hist(col):
    """(forward[33], backward[33]) counts of the jumps col[i+1] - col[i] in
    storage order; bin 0 = no jump, bin b = 2^(b-1) <= |jump| < 2^b."""
    c = _i32(col)
    h = np.zeros(66, dtype=np.int64)
    lib().orc_stride_hist(len(c), c, h)
    return h[:33], h[33:]


def warp_sectors_crs(A, lanes, elem_bytes=8):
    """hist[c] = warp accesses touching c distinct 32-byte sectors of x, for
    the CRS kernel with `lanes` lanes per row."""
    h = np.zeros(33, dtype=np.int64)
    lib().orc_warp_sectors_crs(A.n_rows, _i32(A.row_ptr), _i32(A.col), lanes, elem_bytes, h)
    return h


def warp_sectors_jds(J, elem_bytes=8):
    h = np.zeros(33, dtype=np.int64)
    lib().orc_warp_sectors_jds(J.n_rows, J.n_diag, _i32(J.jd_ptr), _i32(J.col), elem_bytes, h)
    return h


def warp_sectors_sell(S_, elem_bytes=8):
    h = np.zeros(33, dtype=np.int64)
    lib().orc_warp_sectors_sell(S_.n_rows, _i32(S_.rlen), _i32(S_.blk_ptr), _i32(S_.col), elem_bytes, h)
    return h


# ---------------------------------------------------------------------------
# Paired SELL (rows of rank q and m-1-q of a sorted window share a lane)
# ---------------------------------------------------------------------------

def psell_build(A, window, symmetric=True):
    """Window sort, pairing and slot-major storage, see orc_psell_build."""
    n = A.n_rows
    perm = np.zeros(n, np.int32)
    iperm = np.zeros(n, np.int32)
    rlen = np.zeros(n, np.int32)
    blk = np.zeros((n + 63) // 64 + 1, np.int32)
    col = np.zeros(A.nnz, np.int32)
    val = np.zeros(A.nnz)
    r = lib().orc_psell_build(n, A.n_cols, _i32(A.row_ptr), _i32(A.col), _f64(A.val), int(symmetric),
                              window, perm, iperm, rlen, blk, col, val)
    if r == -1:
        raise ValueError("symmetric permutation needs a square matrix")
    if r == -2:
        raise ValueError("window must be a positive multiple of 64")
    return SELL(n, symmetric, window, perm, iperm, rlen, blk, col, val)


def psell_spmv(P, x_p):
    out = np.zeros(P.n_rows)
    lib().orc_psell_spmv(P.n_rows, _i32(P.rlen), _i32(P.blk_ptr), _i32(P.col), _f64(P.val), _f64(x_p), out)
    return out


# ---------------------------------------------------------------------------
# Symmetric SpMVM from the upper triangle
# ---------------------------------------------------------------------------

def upper(A):
    """CRS of the entries with col >= row, in their CRS order."""
    from types import SimpleNamespace
    rp, c = _i32(A.row_ptr), _i32(A.col)
    nu = int(lib().orc_upper_count(A.n_rows, rp, c))
    rpu = np.zeros(A.n_rows + 1, np.int32)
    cu = np.zeros(nu, np.int32)
    vu = np.zeros(nu)
    lib().orc_upper_extract(A.n_rows, rp, c, _f64(A.val), rpu, cu, vu)
    return SimpleNamespace(n_rows=A.n_rows, n_cols=A.n_cols, row_ptr=rpu, col=cu, val=vu, nnz=nu)


def sym_spmv(U, x):
    """y = (U + U^T - diag U) x from the upper triangle U."""
    out = np.zeros(U.n_rows)
    lib().orc_sym_spmv(U.n_rows, _i32(U.row_ptr), _i32(U.col), _f64(U.val), _f64(x), out)
    return out


# ---------------------------------------------------------------------------
# Hybrid storage: dense secondary diagonals in DIA form + remainder CRS
# ---------------------------------------------------------------------------

def dia_select(A, max_diags=16, min_fill=2.0 / 3.0):
    offs = np.zeros(max(max_diags, 1), np.int32)
    m = int(lib().orc_dia_select(A.n_rows, A.n_cols, _i32(A.row_ptr), _i32(A.col), max_diags, min_fill, offs))
    return offs[:m].copy()


def dia_build(A, offs):
    """(dia [len(offs), n_rows], remainder CRS as a SimpleNamespace)."""
    from types import SimpleNamespace
    offs = _i32(offs)
    nd = len(offs)
    dia = np.zeros(nd * A.n_rows)
    rp = np.zeros(A.n_rows + 1, np.int32)
    col = np.zeros(max(A.nnz, 1), np.int32)
    val = np.zeros(max(A.nnz, 1))
    m = int(lib().orc_dia_build(A.n_rows, _i32(A.row_ptr), _i32(A.col), _f64(A.val), nd,
                                offs if nd else np.zeros(1, np.int32), dia if nd else np.zeros(1), rp, col, val))
    rem = SimpleNamespace(n_rows=A.n_rows, n_cols=A.n_cols, row_ptr=rp, col=col[:m].copy(), val=val[:m].copy(),
                          nnz=m)
    return dia.reshape(nd, A.n_rows), rem


def dia_spmv(offs, dia, rem, x):
    out = np.zeros(rem.n_rows)
    nd = len(offs)
    lib().orc_dia_spmv(rem.n_rows, rem.n_cols, nd, _i32(offs) if nd else np.zeros(1, np.int32),
                       _f64(dia.ravel()) if nd else np.zeros(1), _i32(rem.row_ptr), _i32(rem.col) if rem.nnz else
                       np.zeros(1, np.int32), _f64(rem.val) if rem.nnz else np.zeros(1), _f64(x), out)
    return out
