"""Access-pattern analysis of the x gather (argument marshalling over
``gbsp_stride_hist`` and ``gbsp_warp_sectors``): the stride distribution of
Sect. 4.2 (Fig. 4a) and the sectors touched per warp-wide gather."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from .sparse import _need_cuda, _stream, _vp


def stride_hist(col: torch.Tensor, stream=None) -> tuple[np.ndarray, np.ndarray]:
    """(forward[33], backward[33]) counts of col[i+1] - col[i] in storage
    order; bin 0 = no jump, bin b = 2^(b-1) <= |jump| < 2^b."""
    col = _need_cuda(col, "col", torch.int32)
    h = torch.empty(66, dtype=torch.int64, device=col.device)
    L.check(L.load().gbsp_stride_hist(_vp(col), col.numel(), _vp(h), _stream(stream)), "gbsp_stride_hist")
    out = h.cpu().numpy()
    return out[:33], out[33:]


def warp_sectors(M, lanes: int = 32, elem_bytes: int | None = None, stream=None) -> np.ndarray:
    """hist[c] = warp-wide x loads of M's product kernel that touch c
    distinct 32-byte sectors (CRS: `lanes` lanes per row)."""
    eb = elem_bytes if elem_bytes is not None else (8 if M.dtype == torch.float64 else 4)
    h = torch.empty(33, dtype=torch.int64, device=M._device)
    L.check(L.load().gbsp_warp_sectors(M._h, lanes, eb, _vp(h), _stream(stream)), "gbsp_warp_sectors")
    return h.cpu().numpy()


def summary(fwd: np.ndarray, bwd: np.ndarray, elem_bytes: int = 8) -> dict:
    """Shares of the jumps as the paper reads Fig. 4a: backward jumps, and
    forward jumps below 64 bytes of x."""
    total = int(fwd.sum() + bwd.sum())
    if total == 0:
        return {"jumps": 0}
    b64 = 1 + int(np.log2(64 // elem_bytes))  # bins 0..b64-1 are below 64 bytes
    return {"jumps": total, "backward_share": round(float(bwd.sum()) / total, 4),
            "below_64B_share": round(float(fwd[:b64].sum() + bwd[:b64].sum()) / total, 4)}


def mean_sectors(hist: np.ndarray) -> float:
    n = hist.sum()
    return float((np.arange(33) * hist).sum() / n) if n else 0.0
