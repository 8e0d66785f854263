"""Python classes over the C ABI (argument marshalling only).

Every product, conversion and gradient runs in the CUDA library; these
classes only allocate device memory with torch, keep the borrowed tensors
alive for as long as the C handles use them, and pass pointers and the
current torch stream.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

_DT = {torch.float64: L.F64, torch.float32: L.F32}


def _vp(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream: torch.cuda.Stream | None = None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return t.contiguous()


def _ld(t: torch.Tensor) -> int:
    return t.stride(0) if t.dim() == 2 else 1


class _Handle:
    """Owns one C handle; destroyed with the Python object."""

    def __init__(self):
        self._h = ctypes.c_void_p()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def __del__(self):
        try:
            if self._h:
                L.load().gbsp_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


class _Product(_Handle):
    n_rows: int
    n_cols: int
    dtype: torch.dtype

    def _vec_out(self, rows: int, k: int | None, like: torch.Tensor) -> torch.Tensor:
        shape = (rows,) if k is None else (rows, k)
        return torch.empty(shape, dtype=self.dtype, device=like.device)

    def spmm(self, X: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False,
             transpose: bool = False, basis: int = L.BASIS_PERMUTED, stream=None) -> torch.Tensor:
        """Y = op(A) X for row-major X (n x k); a 1-D X is a single vector.
        For k >= 8 a CRS handle is the faster format (its lanes cover one
        row's right-hand sides); JDS-family handles gather k values a row."""
        if not X.is_cuda or X.dtype != self.dtype:
            raise ValueError(f"X must be a CUDA tensor of dtype {self.dtype}")
        if X.dim() == 1 or X.stride(-1) != 1:
            X = X.contiguous()
        vec = X.dim() == 1
        k = 1 if vec else X.shape[1]
        rows_in, rows_out = (self.n_rows, self.n_cols) if transpose else (self.n_cols, self.n_rows)
        if X.shape[0] != rows_in:
            raise ValueError(f"x has {X.shape[0]} rows, expected {rows_in}")
        if out is None:
            out = (torch.zeros if accumulate else torch.empty)(
                (rows_out,) if vec else (rows_out, k), dtype=self.dtype, device=X.device)
        elif out.shape[0] != rows_out or out.dtype != self.dtype:
            raise ValueError("out has the wrong shape or dtype")
        L.check(L.load().gbsp_spmm(self._h, L.OP_T if transpose else L.OP_N, basis, k, _vp(X),
                                   _ld(X), _vp(out), _ld(out), int(accumulate), _stream(stream)),
                "gbsp_spmm")
        return out

    def spmv(self, x: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False,
             transpose: bool = False, basis: int = L.BASIS_PERMUTED, stream=None) -> torch.Tensor:
        """y = op(A) x (or y += op(A) x)."""
        if x.dim() != 1:
            raise ValueError("spmv takes a 1-D vector; use spmm for several")
        return self.spmm(x, out, accumulate, transpose, basis, stream)

    def host_stage(self, transpose: bool = False, device=None) -> tuple[torch.Tensor, torch.Tensor]:
        """Device stages (input, output) for spmv_host, reusable across calls."""
        dev = device if device is not None else self._device
        n_in, n_out = (self.n_rows, self.n_cols) if transpose else (self.n_cols, self.n_rows)
        return (torch.empty(n_in, dtype=self.dtype, device=dev), torch.empty(n_out, dtype=self.dtype, device=dev))

    def spmv_host(self, x: torch.Tensor, out: torch.Tensor | None = None, stage=None, accumulate: bool = False,
                  transpose: bool = False, basis: int = L.BASIS_PERMUTED, stream=None) -> torch.Tensor:
        """y = op(A) x with x and y in host memory: copy in, product, copy
        out, in order on the stream (gbsp_spmv_host).  `out` holds the result
        once the stream is synchronised; page-locked tensors move at the full
        speed of the host link."""
        n_in, n_out = (self.n_rows, self.n_cols) if transpose else (self.n_cols, self.n_rows)
        for t, n, name in ((x, n_in, "x"), (out, n_out, "out")):
            if t is None and name == "out":
                continue
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != self.dtype or t.dim() != 1 or t.numel() != n or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous host vector of {n} {self.dtype} elements")
        if out is None:
            out = (torch.zeros if accumulate else torch.empty)(n_out, dtype=self.dtype, pin_memory=True)
        dx, dy = stage if stage is not None else self.host_stage(transpose)
        if dx.numel() != n_in or dy.numel() != n_out or not (dx.is_cuda and dy.is_cuda):
            raise ValueError("stage vectors have the wrong size")
        L.check(L.load().gbsp_spmv_host(self._h, L.OP_T if transpose else L.OP_N, basis, int(accumulate),
                                        _vp(x), _vp(out), _vp(dx), _vp(dy), _stream(stream)),
                "gbsp_spmv_host")
        return out

    def spmv_symmetric(self, x: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False,
                       stream=None) -> torch.Tensor:
        """y = (S + S^T - diag S) x for the stored triangle S (FP64 atomics:
        reproducible within rounding only).  CRS or row-only SELL handles."""
        x = _need_cuda(x, "x", self.dtype)
        if out is None:
            out = torch.zeros(self.n_rows, dtype=self.dtype, device=x.device)
        L.check(L.load().gbsp_spmv_symmetric(self._h, _vp(x), _vp(out), int(accumulate), _stream(stream)),
                "gbsp_spmv_symmetric")
        return out

    def set_grid_limit(self, max_ctas: int = 0) -> None:
        """Cap the product kernel's grid at max_ctas CTAs (0: no cap); for
        throughput-against-CTAs measurements."""
        L.check(L.load().gbsp_set_grid_limit(self._h, int(max_ctas)), "gbsp_set_grid_limit")

    def set_kernel(self, kernel: str = "vector", lanes: int = 0, rows_per_warp: int = 0,
                   tile: int = 0, rhs_tile: int = 0, compensated: bool | None = None) -> None:
        o = L.KernelOpts()
        L.check(L.load().gbsp_get_kernel(self._h, ctypes.byref(o)), "gbsp_get_kernel")
        accum = o.accum if compensated is None else (L.ACC_COMPENSATED if compensated else L.ACC_PLAIN)
        o = L.KernelOpts(L.KERNELS[kernel], lanes, rows_per_warp, tile, rhs_tile, accum)
        L.check(L.load().gbsp_set_kernel(self._h, ctypes.byref(o)), "gbsp_set_kernel")

    def kernel_opts(self) -> dict:
        o = L.KernelOpts()
        L.check(L.load().gbsp_get_kernel(self._h, ctypes.byref(o)), "gbsp_get_kernel")
        return {f: getattr(o, f) for f, _ in L.KernelOpts._fields_}

    def autotune(self, k: int = 1, stream=None) -> tuple[dict, float]:
        """Time the candidate kernels on this matrix and keep the fastest."""
        dev = self._device
        X = torch.zeros((self.n_cols,) if k == 1 else (self.n_cols, k), dtype=self.dtype, device=dev)
        Y = torch.zeros((self.n_rows,) if k == 1 else (self.n_rows, k), dtype=self.dtype, device=dev)
        best = L.KernelOpts()
        ms = ctypes.c_float()
        L.check(L.load().gbsp_autotune(self._h, k, _vp(X), _vp(Y), _stream(stream),
                                       ctypes.byref(best), ctypes.byref(ms)), "gbsp_autotune")
        return {f: getattr(best, f) for f, _ in L.KernelOpts._fields_}, ms.value


class CRSMatrix(_Product):
    """A CRS matrix on the GPU (Sect. 2): row_ptr (int32, n_rows+1), col
    (int32, nnz), val (float64 or float32, nnz), all borrowed by the C
    handle and kept alive here."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n_cols: int):
        super().__init__()
        self.row_ptr = _need_cuda(row_ptr, "row_ptr", torch.int32)
        self.col = _need_cuda(col, "col", torch.int32)
        self.val = _need_cuda(val, "val")
        if self.val.dtype not in _DT:
            raise ValueError("val must be float64 or float32")
        self.dtype = self.val.dtype
        self.n_rows = self.row_ptr.numel() - 1
        self.n_cols = int(n_cols)
        self.nnz = self.col.numel()
        if self.val.numel() != self.nnz:
            raise ValueError("col and val lengths differ")
        self._device = self.row_ptr.device
        self._tile_table = None
        self._transpose = None
        L.check(L.load().gbsp_crs_create(self.n_rows, self.n_cols, self.nnz, _vp(self.row_ptr),
                                         _vp(self.col), _vp(self.val), _DT[self.dtype],
                                         ctypes.byref(self._h)), "gbsp_crs_create")

    @classmethod
    def from_host(cls, A, device="cuda", dtype=torch.float64) -> "CRSMatrix":
        """From any object with n_rows, n_cols, row_ptr, col, val (numpy)."""
        return cls(torch.as_tensor(A.row_ptr, dtype=torch.int32).to(device),
                   torch.as_tensor(A.col, dtype=torch.int32).to(device),
                   torch.as_tensor(A.val).to(device=device, dtype=dtype), A.n_cols)

    def set_values(self, val: torch.Tensor) -> None:
        """Point the handle at new values (same pattern and dtype); no copy."""
        val = _need_cuda(val, "val", self.dtype)
        if val.numel() != self.nnz:
            raise ValueError("val has the wrong length")
        L.check(L.load().gbsp_set_values(self._h, _vp(val)), "gbsp_set_values")
        self.val = val

    def validate(self, stream=None) -> int:
        """0 if the CRS arrays are well formed, else GBSP_ERR_MATRIX (-2)."""
        st = torch.empty(1, dtype=torch.int32, device=self._device)
        L.check(L.load().gbsp_crs_validate(self._h, _vp(st), _stream(stream)), "gbsp_crs_validate")
        out = ctypes.c_int32()
        L.check(L.load().gbsp_read_status(_vp(st), _stream(stream), ctypes.byref(out)),
                "gbsp_read_status")
        return out.value

    def prepare_tiled(self, tile: int = 2048, stream=None) -> None:
        """Build the tile table of the TILED kernel and select that kernel."""
        nb = ctypes.c_int64()
        L.check(L.load().gbsp_crs_tile_bytes(self._h, tile, ctypes.byref(nb)), "gbsp_crs_tile_bytes")
        self._tile_table = torch.empty(nb.value // 4, dtype=torch.int32, device=self._device)
        L.check(L.load().gbsp_crs_prepare(self._h, tile, _vp(self._tile_table), nb.value,
                                          _stream(stream)), "gbsp_crs_prepare")
        self.set_kernel("tiled")

    def to_jds(self, fmt: str = "JDS", perm: str = "symmetric", block: int = 256, unroll: int = 4,
               stream=None, value_map: bool = False, window: int = 1024) -> "JDSMatrix":
        """Convert on the GPU to a JDS-family format (JDS, NBJDS, NUJDS,
        RBJDS, SOJDS, JDS_LITERAL, or SELL with a sorting `window`)."""
        return JDSMatrix(self, fmt, perm, block, unroll, stream, value_map, window)

    def transpose(self, stream=None) -> "CRSMatrix":
        """Build the transposed structure (a CRS of A^T with its entry map)
        and attach it, so spmv(..., transpose=True) computes A^T g."""
        lib = L.load()
        dev = self._device
        ws = ctypes.c_int64()
        L.check(lib.gbsp_transpose_workspace(self._h, ctypes.byref(ws)), "gbsp_transpose_workspace")
        t_row_ptr = torch.empty(self.n_cols + 1, dtype=torch.int32, device=dev)
        t_col = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        t_val = torch.empty(self.nnz, dtype=self.dtype, device=dev)
        tmap = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        work = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        bufs = L.TransposeBuffers(_vp(t_row_ptr).value, _vp(t_col).value, _vp(t_val).value,
                                  _vp(tmap).value, _vp(work).value)
        T = CRSMatrix.__new__(CRSMatrix)
        _Handle.__init__(T)
        L.check(lib.gbsp_transpose_build(self._h, ctypes.byref(bufs), ws.value, _stream(stream),
                                         ctypes.byref(T._h)), "gbsp_transpose_build")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        del work
        T.row_ptr, T.col, T.val, T.tmap = t_row_ptr, t_col, t_val, tmap
        T.dtype, T.n_rows, T.n_cols, T.nnz = self.dtype, self.n_cols, self.n_rows, self.nnz
        T._device, T._tile_table, T._transpose = dev, None, None
        T._source = self
        self._transpose = T
        return T

    def upper(self, stream=None) -> "CRSMatrix":
        """CRS of the upper triangle (col >= row, CRS order kept) of this
        square matrix, for ``spmv_symmetric``."""
        lib = L.load()
        dev = self._device
        ws = ctypes.c_int64()
        L.check(lib.gbsp_upper_workspace(self.n_rows, ctypes.byref(ws)), "gbsp_upper_workspace")
        row_ptr_u = torch.empty(self.n_rows + 1, dtype=torch.int32, device=dev)
        work = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        nnz_u = ctypes.c_int64()
        L.check(lib.gbsp_upper_plan(self._h, _vp(row_ptr_u), _vp(work), ws.value, _stream(stream),
                                    ctypes.byref(nnz_u)), "gbsp_upper_plan")
        col_u = torch.empty(nnz_u.value, dtype=torch.int32, device=dev)
        val_u = torch.empty(nnz_u.value, dtype=self.dtype, device=dev)
        U = CRSMatrix.__new__(CRSMatrix)
        _Handle.__init__(U)
        L.check(lib.gbsp_upper_build(self._h, _vp(row_ptr_u), _vp(col_u), _vp(val_u), nnz_u.value,
                                     _stream(stream), ctypes.byref(U._h)), "gbsp_upper_build")
        U.row_ptr, U.col, U.val = row_ptr_u, col_u, val_u
        U.dtype, U.n_rows, U.n_cols, U.nnz = self.dtype, self.n_rows, self.n_cols, nnz_u.value
        U._device, U._tile_table, U._transpose = dev, None, None
        return U

    def attach_transpose(self, at: "_Product") -> None:
        L.check(L.load().gbsp_attach_transpose(self._h, at.handle), "gbsp_attach_transpose")
        self._transpose = at

    def refresh_transpose_values(self, stream=None) -> None:
        """Re-gather A^T's values after A's values changed in place."""
        L.check(L.load().gbsp_transpose_values(self._h, _stream(stream)), "gbsp_transpose_values")

    def dval(self, g: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None,
             accumulate: bool = False, stream=None) -> torch.Tensor:
        """dval_k = g[row_k] * x[col_k] (+= if accumulate)."""
        g = _need_cuda(g, "g", self.dtype)
        x = _need_cuda(x, "x", self.dtype)
        if out is None:
            out = (torch.zeros if accumulate else torch.empty)(self.nnz, dtype=self.dtype, device=g.device)
        L.check(L.load().gbsp_dval(self._h, _vp(g), _vp(x), _vp(out), int(accumulate),
                                   _stream(stream)), "gbsp_dval")
        return out

    def dval_multi(self, G: torch.Tensor, X: torch.Tensor, out: torch.Tensor | None = None,
                   accumulate: bool = False, stream=None) -> torch.Tensor:
        """dval_k = sum_t G[row_k, t] X[col_k, t], G and X 2-D in any
        layout (row-major, or columns that are contiguous vectors)."""
        for t, name in ((G, "G"), (X, "X")):  # no copy: the layout is passed as strides
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != self.dtype:
                raise ValueError(f"{name} must be a CUDA tensor of dtype {self.dtype}")
        if G.dim() != 2 or X.dim() != 2:
            raise ValueError("G and X must be 2-D")
        m = G.shape[1]
        if X.shape[1] != m:
            raise ValueError("G and X need the same number of columns")
        if G.shape[0] != self.n_rows or X.shape[0] != self.n_cols:
            raise ValueError("G needs n_rows rows and X n_cols rows")
        if out is None:
            out = (torch.zeros if accumulate else torch.empty)(self.nnz, dtype=self.dtype, device=G.device)
        if min(G.stride()) < 1 or min(X.stride()) < 1:
            G, X = G.contiguous(), X.contiguous()  # broadcast (stride 0) views
        (gr, gt), (xr, xt) = G.stride(), X.stride()
        L.check(L.load().gbsp_dval_multi_strided(self._h, m, _vp(G), gr, gt, _vp(X), xr, xt,
                                                 _vp(out), int(accumulate), _stream(stream)),
                "gbsp_dval_multi_strided")
        return out


class JDSMatrix(_Product):
    """A JDS-family matrix built on the GPU from a CRS matrix (Sect. 2).

    fmt: JDS, NBJDS, NUJDS, RBJDS, SOJDS or JDS_LITERAL; perm: 'symmetric'
    (rows and columns permuted, the paper's scheme) or 'row_only'."""

    def __init__(self, A: CRSMatrix, fmt="JDS", perm="symmetric", block=256, unroll=4, stream=None,
                 value_map: bool = False, window: int = 1024):
        super().__init__()
        lib = L.load()
        dev = A._device
        self.dtype, self.n_rows, self.n_cols, self.nnz = A.dtype, A.n_rows, A.n_cols, A.nnz
        self._device = dev
        opts = L.JdsOpts(L.FORMATS[fmt], L.PERM[perm], block, unroll, window)
        sizes = L.JdsSizes()
        scratch = torch.empty(16, dtype=torch.int32, device=dev)
        L.check(lib.gbsp_jds_plan(A.handle, ctypes.byref(opts), _vp(scratch), _stream(stream),
                                  ctypes.byref(sizes)), "gbsp_jds_plan")
        self.n_diag = sizes.n_diag
        self.n_blocks = sizes.n_blocks
        self.jd_ptr = torch.empty(sizes.n_diag + 1, dtype=torch.int32, device=dev)
        self.col = torch.empty(A.nnz, dtype=torch.int32, device=dev)
        self.val = torch.empty(A.nnz, dtype=A.dtype, device=dev)
        self.perm = torch.empty(A.n_rows, dtype=torch.int32, device=dev)
        self.iperm = torch.empty(A.n_rows, dtype=torch.int32, device=dev)
        self.blk_ptr = (torch.empty(sizes.n_blocks + 1, dtype=torch.int32, device=dev)
                        if fmt in ("RBJDS", "SOJDS", "SELL", "PSELL") else None)
        self.rlen = (torch.empty(A.n_rows, dtype=torch.int32, device=dev) if fmt in ("SELL", "PSELL")
                     else None)
        work = torch.empty(max(sizes.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        self.vmap = torch.empty(A.nnz, dtype=torch.int32, device=dev) if value_map else None
        bufs = L.JdsBuffers(_vp(self.jd_ptr).value, _vp(self.col).value, _vp(self.val).value,
                            _vp(self.perm).value, _vp(self.iperm).value, _vp(self.blk_ptr).value,
                            _vp(work).value, _vp(self.vmap).value, _vp(self.rlen).value)
        L.check(lib.gbsp_jds_build(A.handle, ctypes.byref(opts), ctypes.byref(bufs),
                                   ctypes.byref(sizes), _stream(stream), ctypes.byref(self._h)),
                "gbsp_jds_build")
        del work  # the build synchronised the stream
        self.fmt, self.perm_mode, self.block, self.unroll = fmt, perm, block, unroll
        self.window = window if fmt in ("SELL", "PSELL") else None
        self.symmetric = perm == "symmetric"

    def refresh_values(self, crs_val: torch.Tensor, stream=None) -> None:
        """Re-gather the stored values from CRS-ordered values (needs value_map)."""
        crs_val = _need_cuda(crs_val, "crs_val", self.dtype)
        L.check(L.load().gbsp_jds_values(self._h, _vp(crs_val), _stream(stream)), "gbsp_jds_values")

    def split(self, depth: int = 64, chunk: int = 128, stream=None) -> None:
        """Sum diagonals >= depth in chunks by a separate kernel (long rows
        spread over many threads); depth=0 removes the split."""
        lib = L.load()
        if depth == 0:
            L.check(lib.gbsp_jds_split(self._h, 0, 0, None, 0, _stream(stream)), "gbsp_jds_split")
            self._split_ws = None
            return
        nb = ctypes.c_int64()
        L.check(lib.gbsp_jds_split_bytes(self._h, depth, chunk, ctypes.byref(nb)), "gbsp_jds_split_bytes")
        self._split_ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self._device)
        L.check(lib.gbsp_jds_split(self._h, depth, chunk, _vp(self._split_ws), self._split_ws.numel(),
                                   _stream(stream)), "gbsp_jds_split")

    def set_format(self, fmt: str, block: int = 0, unroll: int = 0) -> None:
        L.check(L.load().gbsp_jds_set_format(self._h, L.FORMATS[fmt], block, unroll),
                "gbsp_jds_set_format")
        self.fmt = fmt
        self.block = block or self.block
        self.unroll = unroll or self.unroll

    def permute(self, v: torch.Tensor, back: bool = False, stream=None) -> torch.Tensor:
        """v -> P v (row order of the JDS basis), or back with back=True."""
        v = _need_cuda(v, "v", self.dtype)
        k = 1 if v.dim() == 1 else v.shape[1]
        out = torch.empty_like(v)
        L.check(L.load().gbsp_permute_vec(self._h, int(back), k, _vp(v), _ld(v), _vp(out), _ld(out),
                                          _stream(stream)), "gbsp_permute_vec")
        return out

    def stage_x(self, pages_per_group: int = 12, min_refs: int = 32, stream=None) -> None:
        """SELL only: stage the most referenced pages of x per 1024-row group
        in shared memory (0 removes it).  Products stay bit-identical."""
        lib = L.load()
        if pages_per_group == 0:
            L.check(lib.gbsp_sell_stage(self._h, 0, 1, None, None, None, 0, _stream(stream)), "gbsp_sell_stage")
            self._stage = None
            return
        cb, pb, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        L.check(lib.gbsp_sell_stage_bytes(self._h, pages_per_group, ctypes.byref(cb), ctypes.byref(pb),
                                          ctypes.byref(wb)), "gbsp_sell_stage_bytes")
        col_st = torch.empty(cb.value // 4, dtype=torch.int32, device=self._device)
        pages = torch.empty(max(pb.value // 4, 1), dtype=torch.int32, device=self._device)
        work = torch.empty(max(wb.value, 1), dtype=torch.uint8, device=self._device)
        L.check(lib.gbsp_sell_stage(self._h, pages_per_group, min_refs, _vp(col_st), _vp(pages), _vp(work),
                                    wb.value, _stream(stream)), "gbsp_sell_stage")
        self._stage = (col_st, pages)

    def spmv_original(self, x: torch.Tensor, out=None, accumulate=False, stream=None):
        return self.spmv(x, out, accumulate, basis=L.BASIS_ORIGINAL, stream=stream)


class DIAMatrix(_Product):
    """The DIA part of a hybrid matrix: selected secondary diagonals, one
    value per row (built by :class:`HybridMatrix`)."""


class HybridMatrix:
    """Dense secondary diagonals in DIA form plus the remainder (Sect. 4.2's
    suggested hybrid): ``y = DIA x`` then the remainder's product added to
    it.  The remainder is kept in CRS or converted to SELL-32-sigma with the
    row-only permutation (vectors stay in the original basis)."""

    def __init__(self, A: CRSMatrix, max_diags: int = 16, min_fill: float = 2.0 / 3.0,
                 remainder: str = "SELL", window: int = 128, unroll: int = 4, stream=None):
        lib = L.load()
        dev = A._device
        ws = ctypes.c_int64()
        L.check(lib.gbsp_dia_plan_workspace(A.handle, ctypes.byref(ws)), "gbsp_dia_plan_workspace")
        work = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        row_ptr_rem = torch.empty(A.n_rows + 1, dtype=torch.int32, device=dev)
        sz = L.DiaSizes()
        L.check(lib.gbsp_dia_plan(A.handle, max_diags, float(min_fill), _vp(row_ptr_rem), _vp(work), ws.value,
                                  _stream(stream), ctypes.byref(sz)), "gbsp_dia_plan")
        del work
        nd = sz.n_diags
        self.offsets_host = [int(sz.offsets[k]) for k in range(nd)]
        self.nnz_dia, self.nnz_rem = int(sz.nnz_dia), int(sz.nnz_rem)
        self.dia = torch.empty((nd, A.n_rows), dtype=A.dtype, device=dev)
        self.offsets = torch.empty(max(nd, 1), dtype=torch.int32, device=dev)
        col_rem = torch.empty(self.nnz_rem, dtype=torch.int32, device=dev)
        val_rem = torch.empty(self.nnz_rem, dtype=A.dtype, device=dev)
        D = DIAMatrix.__new__(DIAMatrix)
        _Handle.__init__(D)
        R = CRSMatrix.__new__(CRSMatrix)
        _Handle.__init__(R)
        L.check(lib.gbsp_dia_build(A.handle, ctypes.byref(sz), _vp(self.dia), _vp(self.offsets), _vp(row_ptr_rem),
                                   _vp(col_rem), _vp(val_rem), _stream(stream), ctypes.byref(D._h),
                                   ctypes.byref(R._h)), "gbsp_dia_build")
        D.n_rows, D.n_cols, D.dtype, D._device = A.n_rows, A.n_cols, A.dtype, dev
        D._dia, D._offsets = self.dia, self.offsets
        R.row_ptr, R.col, R.val = row_ptr_rem, col_rem, val_rem
        R.dtype, R.n_rows, R.n_cols, R.nnz = A.dtype, A.n_rows, A.n_cols, self.nnz_rem
        R._device, R._tile_table, R._transpose = dev, None, None
        self.dia_part, self.remainder = D, R
        self.n_rows, self.n_cols, self.dtype = A.n_rows, A.n_cols, A.dtype
        # the remainder sums like the source handle (plain or compensated FP32)
        R.set_kernel("vector", compensated=A.kernel_opts()["accum"] == L.ACC_COMPENSATED)
        self.rem_op = None
        if self.nnz_rem > 0:
            self.rem_op = R.to_jds("SELL", "row_only", window=window, unroll=unroll) if remainder == "SELL" else R

    def spmv(self, x: torch.Tensor, out: torch.Tensor | None = None, accumulate: bool = False,
             stream=None) -> torch.Tensor:
        out = self.dia_part.spmv(x, out=out, accumulate=accumulate, stream=stream)
        if self.rem_op is not None:
            if isinstance(self.rem_op, JDSMatrix):
                self.rem_op.spmv_original(x, out=out, accumulate=True, stream=stream)
            else:
                self.rem_op.spmv(x, out=out, accumulate=True, stream=stream)
        return out
