"""Differentiable sparse products (argument marshalling over the C ABI).

``spmv(pattern, val, x)`` is y = A x with A's values ``val`` (CRS entry
order) and x both differentiable; the backward pass runs the library's
kernels: dx = A^T g on the transposed structure (a CRS of A^T, or a JDS of
A^T -- the "transposed JDS" form), and dval_k = g[row_k] x[col_k].

``power_apply(pattern, val, x, m, checkpoint)`` is A^m x for iterated
products as in the eigensolvers the paper is about (Sect. 1): the forward
pass stores x_t only every `checkpoint` steps; the backward pass recomputes
each segment from its checkpoint, runs g_{t-1} = A^T g_t down the segment
and adds the segment's value gradient sum_t g_t[row] x_{t-1}[col] with ONE
fused pass over the entries (gbsp_dval_multi_strided).  The fused kernel adds the
terms for t = m, m-1, ..., 1 in that order into one running sum, so the
gradients are bit-identical for every checkpoint interval.
"""
from __future__ import annotations

import torch

from .sparse import CRSMatrix


class Pattern:
    """Sparsity pattern (row_ptr, col on the GPU) plus the kernels' set-up.

    The value gradient always runs on the CRS handle (dval is in CRS entry
    order).  The products can run elsewhere:
      forward: "crs" -- the CRS handle; "jds" -- a JDS of A (row-only
               permutation, NUJDS walk) whose values are re-gathered when they
               change; "sell" -- SELL-32-sigma of A (row-only, window 128),
               likewise; "auto" -- whichever of the three the autotuner times
               fastest.
      adjoint: "crs" -- the CRS of A^T (transposed structure); "jds" / "sell"
               -- a JDS / SELL of A^T (the transposed-JDS form); "auto" -- the
               fastest of the three.
    """

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, n_cols: int, dtype=torch.float64,
                 adjoint: str = "crs", forward: str = "crs", tiled: bool = False):
        self.row_ptr = row_ptr.contiguous()
        self.col = col.contiguous()
        self.n_rows = self.row_ptr.numel() - 1
        self.n_cols = int(n_cols)
        self.nnz = self.col.numel()
        self.dtype = dtype
        self.adjoint = adjoint
        self.forward = forward
        dummy = torch.zeros(max(self.nnz, 1), dtype=dtype, device=self.row_ptr.device)[: self.nnz]
        self.A = CRSMatrix(self.row_ptr, self.col, dummy, self.n_cols)
        if tiled:
            self.A.prepare_tiled(1024)
        self.F = None
        self._fkey = None
        self.ST = None
        self.AT = None
        self.JT = None
        self._adj = None
        self._akey = None

    @classmethod
    def from_host(cls, A, device="cuda", dtype=torch.float64, **kw) -> "Pattern":
        return cls(torch.as_tensor(A.row_ptr, dtype=torch.int32).to(device),
                   torch.as_tensor(A.col, dtype=torch.int32).to(device), A.n_cols, dtype, **kw)

    def bind(self, val: torch.Tensor) -> CRSMatrix:
        """Point the CRS handle at `val`."""
        if val.dtype != self.dtype or val.numel() != self.nnz:
            raise ValueError("values do not match the pattern")
        self.A.set_values(val.detach())
        return self.A

    def forward_op(self, val: torch.Tensor):
        A = self.bind(val)
        if self.forward == "crs":
            return A
        if self.F is None:
            cands = []
            if self.forward in ("jds", "auto"):
                cands.append(A.to_jds("NUJDS", "row_only", unroll=4, value_map=True))
            if self.forward in ("sell", "auto"):
                cands.append(A.to_jds("SELL", "row_only", window=128, unroll=4, value_map=True))
            for J in cands:
                J.refresh_values(val.detach())
            if self.forward == "auto":
                timed = [(A.autotune(1)[1], 0, A)] + [(J.autotune(1)[1], i + 1, J) for i, J in enumerate(cands)]
                self.F = min(timed, key=lambda t: (t[0], t[1]))[2]
            else:
                self.F = cands[0]
            self._fkey = None
        if self.F is not A:
            key = (val.data_ptr(), val._version)
            if self._fkey != key:
                self.F.refresh_values(val.detach())
                self._fkey = key
        return self.F

    def apply(self, val: torch.Tensor, x: torch.Tensor, out=None) -> torch.Tensor:
        """A x for 1-D x or an (n, 1) column view (with `out` likewise)."""
        return self.forward_op(val).spmm(x, out=out, basis=1)

    def adjoint_op(self, val: torch.Tensor):
        """Handle computing A^T g for the bound values (built on first use,
        values re-gathered whenever `val` changed)."""
        self.bind(val)
        if self.AT is None:
            self.AT = self.A.transpose()
            if self.adjoint in ("jds", "auto"):
                self.JT = self.AT.to_jds("NUJDS", "row_only", unroll=4, value_map=True)
                self.JT.refresh_values(self.AT.val)
            if self.adjoint in ("sell", "auto"):
                self.ST = self.AT.to_jds("SELL", "row_only", window=128, unroll=4, value_map=True)
                self.ST.refresh_values(self.AT.val)
            self._adj = {"jds": self.JT, "sell": self.ST}.get(self.adjoint, self.AT)
            if self.adjoint == "auto":
                timed = [(H.autotune(1)[1], i, H) for i, H in enumerate((self.AT, self.JT, self.ST))]
                self._adj = min(timed, key=lambda t: (t[0], t[1]))[2]
            self._akey = None
        key = (val.data_ptr(), val._version)
        if self._akey != key:
            self.A.refresh_transpose_values()
            if self._adj is not self.AT:
                self._adj.refresh_values(self.AT.val)
            self._akey = key
        return self._adj

    def apply_t(self, val: torch.Tensor, g: torch.Tensor, out=None) -> torch.Tensor:
        """A^T g for 1-D g or an (n, 1) column view (with `out` likewise)."""
        return self.adjoint_op(val).spmm(g, out=out, basis=1)


class SpMVFunction(torch.autograd.Function):
    """y = A(val) x; gradients for val (per stored entry) and x."""

    @staticmethod
    def forward(ctx, val, x, pattern: Pattern):
        ctx.pattern = pattern
        ctx.save_for_backward(val, x)
        return pattern.apply(val, x.detach().contiguous())

    @staticmethod
    def backward(ctx, gy):
        val, x = ctx.saved_tensors
        p = ctx.pattern
        gy = gy.contiguous()
        dval = dx = None
        if ctx.needs_input_grad[0]:
            dval = p.bind(val).dval(gy, x.detach().contiguous())
        if ctx.needs_input_grad[1]:
            dx = p.apply_t(val, gy)
        return dval, dx, None


def spmv(pattern: Pattern, val: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    return SpMVFunction.apply(val, x, pattern)


class PowerFunction(torch.autograd.Function):
    """x_m = A^m x with checkpointed recomputation in the backward pass."""

    @staticmethod
    def forward(ctx, val, x, pattern: Pattern, m: int, c: int):
        cur = x.detach().contiguous()
        ckpts = [cur]
        for t in range(1, m + 1):
            cur = pattern.apply(val, cur)
            if t % c == 0 and t < m:
                ckpts.append(cur)
        ctx.pattern, ctx.m, ctx.c = pattern, m, c
        ctx.save_for_backward(val, *ckpts)
        return cur

    @staticmethod
    def backward(ctx, gm):
        val, *ckpts = ctx.saved_tensors
        p, m, c = ctx.pattern, ctx.m, ctx.c
        n = p.n_rows
        dev, dt = gm.device, gm.dtype
        dval = torch.zeros(p.nnz, dtype=dt, device=dev) if ctx.needs_input_grad[0] else None
        g = gm.contiguous()
        for seg in range((m - 1) // c, -1, -1):
            t0 = seg * c
            w = min(t0 + c, m) - t0
            # X[:, i] = x_{t1-1-i}: recomputed from the checkpoint x_{t0}.
            # Columns are contiguous vectors (column-major n x w), so every
            # product reads and writes with unit stride; the fused dval takes
            # the layout as strides.
            X = torch.empty((w, n), dtype=dt, device=dev).t()
            X[:, w - 1] = ckpts[seg]
            for j in range(1, w):
                p.apply(val, X[:, w - j:w - j + 1], out=X[:, w - 1 - j:w - j])
            # G[:, i] = g_{t1-i}, i.e. g_{t-1} = A^T g_t down the segment
            G = torch.empty((w, n), dtype=dt, device=dev).t()
            G[:, 0] = g
            for i in range(1, w):
                p.apply_t(val, G[:, i - 1:i], out=G[:, i:i + 1])
            if dval is not None:
                # terms g_t[row] x_{t-1}[col] for t = t1, t1-1, ..., t0+1
                p.bind(val).dval_multi(G, X, out=dval, accumulate=True)
            g = p.apply_t(val, G[:, w - 1:w]).reshape(n)
        return dval, (g if ctx.needs_input_grad[1] else None), None, None, None


def power_apply(pattern: Pattern, val: torch.Tensor, x: torch.Tensor, m: int,
                checkpoint: int = 1) -> torch.Tensor:
    """A^m x, differentiable in val and x, with x_t stored every
    `checkpoint` steps."""
    if m < 1 or checkpoint < 1:
        raise ValueError("m and checkpoint must be >= 1")
    return PowerFunction.apply(val, x, pattern, int(m), int(checkpoint))
