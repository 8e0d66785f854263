"""The basic sparse vector operations of Sect. 4.1 (ADD / SCP over packed
dense, constant-stride and indirect access) on the device: argument
marshalling over ``gbsp_gather_sum``."""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .sparse import _need_cuda, _stream, _vp

OPS = {"ADD": 0, "SCP": 1}
ACCESS = {"PD": 0, "CS": 1, "IND": 2, "IND_TMA": 3}


def partials_needed(n: int) -> int:
    c = ctypes.c_int32()
    L.check(L.load().gbsp_gather_partials(n, ctypes.byref(c)), "gbsp_gather_partials")
    return int(c.value)


class GatherSum:
    """One configured gather sum with its scratch, for repeated launches:
    ``s = GatherSum("SCP", "IND", n, b, a=a, ind=ind); s(); s.out``."""

    def __init__(self, op: str, access: str, n: int, b: torch.Tensor, a: torch.Tensor | None = None,
                 k: int = 1, ind: torch.Tensor | None = None, status: torch.Tensor | None = None):
        if op not in OPS or access not in ACCESS:
            raise ValueError(f"unknown op {op!r} or access {access!r}")
        self.b = _need_cuda(b, "b", torch.float64)
        self.a = _need_cuda(a, "a", torch.float64) if op == "SCP" else None
        self.ind = _need_cuda(ind, "ind", torch.int32) if access in ("IND", "IND_TMA") else None
        if self.a is not None and self.a.numel() < n:
            raise ValueError("a shorter than n")
        if self.ind is not None and self.ind.numel() < n:
            raise ValueError("ind shorter than n")
        self.op, self.access, self.n, self.k = OPS[op], ACCESS[access], int(n), int(k)
        dev = self.b.device
        self.n_partials = partials_needed(self.n)
        self.partials = torch.empty(self.n_partials, dtype=torch.float64, device=dev)
        self.out = torch.zeros(1, dtype=torch.float64, device=dev)
        if status is not None:
            status = _need_cuda(status, "status", torch.int32)
            if status.numel() < 1:
                raise ValueError("status must hold one int32")
        self.status = status

    def __call__(self, stream=None) -> torch.Tensor:
        L.check(L.load().gbsp_gather_sum(self.op, self.access, self.n, self.k, _vp(self.a), _vp(self.b),
                                         self.b.numel(), _vp(self.ind), _vp(self.partials), self.n_partials,
                                         _vp(self.out), _vp(self.status), _stream(stream)),
                "gbsp_gather_sum")
        return self.out


def gather_sum(op: str, access: str, n: int, b: torch.Tensor, a: torch.Tensor | None = None, k: int = 1,
               ind: torch.Tensor | None = None, status: torch.Tensor | None = None) -> torch.Tensor:
    """s = sum_i B(idx(i)) (ADD) or sum_i A(i) B(idx(i)) (SCP), idx(i) = i
    (PD), k i (CS) or ind(i) (IND), as a 1-element FP64 device tensor."""
    return GatherSum(op, access, n, b, a, k, ind, status)()


class FmaChain:
    """The FP64 issue-rate launch (``gbsp_fma_chain``): n_threads threads,
    each running 8 independent chains x <- fma(x, a, b) for `iters` steps;
    lanes >= active_lanes of each warp skip the chains.  ``flops`` counts
    the arithmetic of the active lanes only."""

    def __init__(self, n_threads: int, active_lanes: int = 32, iters: int = 4096, x0: float = 1.0,
                 a: float = 0.5, b: float = 1.0, device="cuda"):
        self.n, self.active, self.iters = int(n_threads), int(active_lanes), int(iters)
        self.inp = torch.tensor([x0, a, b], dtype=torch.float64, device=device)
        self.out = torch.empty(max(self.n, 1), dtype=torch.float64, device=device)
        full, rest = divmod(self.n, 32)
        self.active_threads = full * self.active + min(rest, self.active)
        self.flops = 16.0 * self.iters * self.active_threads

    def __call__(self, stream=None) -> torch.Tensor:
        L.check(L.load().gbsp_fma_chain(self.n, self.active, self.iters, _vp(self.inp), _vp(self.out),
                                        _stream(stream)), "gbsp_fma_chain")
        return self.out


def stage_sweep(b: torch.Tensor, out: torch.Tensor | None = None, status: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Every SM reads all of ``b`` through shared memory once
    (``gbsp_stage_sweep``): the floor of a column-panel gather for
    uniformly random indices.  Returns, per SM, the sum of the first double
    of every 32 KB chunk."""
    b = _need_cuda(b, "b", torch.float64)
    sms = torch.cuda.get_device_properties(b.device).multi_processor_count
    if out is None:
        out = torch.empty(sms, dtype=torch.float64, device=b.device)
    L.check(L.load().gbsp_stage_sweep(_vp(b), b.numel(), _vp(out), out.numel(), _vp(status), _stream(stream)),
            "gbsp_stage_sweep")
    return out
