"""Batched products in one persistent launch, optionally replayed from a
CUDA graph (argument marshalling over gbsp_batch_*).

Each item is (matrix handle, X, Y): Y = A X with k = X.shape[1] right-hand
sides (a 1-D X is k = 1).  JDS-family items work in their permuted basis.
``Batch.autotuned`` picks, per matrix, the storage scheme and kernel options
with the library's autotuner.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .sparse import CRSMatrix, _stream, _vp


def _ld(t: torch.Tensor) -> int:
    return t.stride(0) if t.dim() == 2 else 1


class Batch:
    def __init__(self, items, chunk: int = 4096, ready: torch.Tensor | None = None, stream=None):
        lib = L.load()
        self.items = list(items)
        self.ready = ready
        arr = (L.BatchItem * len(self.items))()
        for i, (A, X, Y) in enumerate(self.items):
            if X.dim() == 2 and X.stride(-1) != 1 or Y.dim() == 2 and Y.stride(-1) != 1:
                raise ValueError("X and Y must be row-major")
            k = 1 if X.dim() == 1 else X.shape[1]
            arr[i] = L.BatchItem(A.handle.value, k, X.data_ptr(), _ld(X), Y.data_ptr(), _ld(Y))
        self._arr = arr
        nb = ctypes.c_int64()
        L.check(lib.gbsp_batch_plan(len(self.items), arr, chunk, ctypes.byref(nb)), "gbsp_batch_plan")
        dev = self.items[0][1].device if self.items else torch.device("cuda")
        self.table = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=dev)
        self._h = ctypes.c_void_p()
        L.check(lib.gbsp_batch_create(len(self.items), arr, chunk, _vp(self.table), self.table.numel(),
                                      _vp(ready), _stream(stream), ctypes.byref(self._h)),
                "gbsp_batch_create")

    def run(self, status: torch.Tensor | None = None, stream=None) -> None:
        L.check(L.load().gbsp_batch_run(self._h, _vp(status), _stream(stream)), "gbsp_batch_run")

    def info(self) -> tuple[int, int]:
        nw, grid = ctypes.c_int64(), ctypes.c_int32()
        L.check(L.load().gbsp_batch_info(self._h, ctypes.byref(nw), ctypes.byref(grid)), "gbsp_batch_info")
        return nw.value, grid.value

    def graph(self, status: torch.Tensor | None = None) -> torch.cuda.CUDAGraph:
        """Capture one run (counter reset + persistent kernel) in a CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(status, stream=s)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(status)
        return g

    def __del__(self):
        try:
            if self._h:
                L.load().gbsp_batch_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass

    @staticmethod
    def autotuned(mats, ks, dtype=torch.float64, device="cuda", formats=("CRS", "JDS", "SELL"),
                  compensated: bool = True, chunk: int = 4096, window: int = 1024,
                  sell_for_k1: bool = True):
        """Build a batch over host CRS matrices `mats` with k_b right-hand
        sides: for every matrix, tune the CRS kernel and (if asked) the JDS
        walks and SELL-32-sigma (row-only permutation, `window` rows), and
        keep the fastest scheme.  With `sell_for_k1`, matrices with k = 1
        take SELL without timing: inside one persistent launch its
        thread-per-row walk spends far fewer FP64 instructions per entry
        than the lanes-per-row CRS walk, which stand-alone timings of small,
        launch-bound matrices do not show (on the 256-matrix batch of the
        benchmark: 421 us all-SELL against 676 us with per-matrix timing).
        Returns (batch, handles, X, Y) with X, Y in the basis of the chosen
        handle (the JDS permuted basis for JDS items; for SELL items x in the
        original basis and y in the window-permuted one), filled with zeros."""
        handles, Xs, Ys = [], [], []
        for A, k in zip(mats, ks):
            M = CRSMatrix.from_host(A, device=device, dtype=dtype)
            if dtype == torch.float32:
                M.set_kernel("vector", compensated=compensated)
            if sell_for_k1 and k == 1 and "SELL" in formats:
                G = M.to_jds("SELL", "row_only", window=window, unroll=4)
                if dtype == torch.float32:
                    G.set_kernel("vector", compensated=compensated)
                handles.append(G)
                Xs.append(torch.zeros(A.n_cols, dtype=dtype, device=device))
                Ys.append(torch.zeros(A.n_rows, dtype=dtype, device=device))
                continue
            best, best_ms = M.autotune(k)
            choice = M
            if "JDS" in formats and A.n_rows == A.n_cols:
                J = M.to_jds("JDS", "symmetric")
                if dtype == torch.float32:
                    J.set_kernel("vector", compensated=compensated)
                _, jms = J.autotune(k)
                if jms < best_ms:
                    choice, best_ms = J, jms
            if "SELL" in formats:
                G = M.to_jds("SELL", "row_only", window=window, unroll=4)
                if dtype == torch.float32:
                    G.set_kernel("vector", compensated=compensated)
                _, gms = G.autotune(k)
                if gms < best_ms:
                    choice, best_ms = G, gms
            handles.append(choice)
            shape_x = (A.n_cols,) if k == 1 else (A.n_cols, k)
            shape_y = (A.n_rows,) if k == 1 else (A.n_rows, k)
            Xs.append(torch.zeros(shape_x, dtype=dtype, device=device))
            Ys.append(torch.zeros(shape_y, dtype=dtype, device=device))
        b = Batch(list(zip(handles, Xs, Ys)), chunk=chunk)
        return b, handles, Xs, Ys
