"""Helpers shared by the GPU parity tests (test infrastructure)."""
from __future__ import annotations

import functools

import numpy as np
import torch

from paper_0910_4836_gb300 import synth as S

# FP64 acceptance per entry: |y - y_ref| <= 1e-14 * sum_j |a_ij||x_j|
TOL64 = 1e-14
U32 = 2.0 ** -24


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def crs(A, dtype=torch.float64):
    from paper_0910_4836_gb300 import CRSMatrix
    return CRSMatrix.from_host(A, device="cuda", dtype=dtype)


def assert_close64(y, ref, s, what="", tol=TOL64):
    err = np.abs(np.asarray(y, np.float64) - ref)
    bound = tol * s
    bad = err > bound
    if bad.any():
        i = int(np.argmax(err - bound))
        raise AssertionError(f"{what}: {int(bad.sum())} of {len(ref)} entries out of tolerance; "
                             f"worst row {i}: got {y[i]!r}, ref {ref[i]!r}, sum|a||x| {s[i]!r}")


def dot2_bound(ref, s, lens):
    """Dot2 error bound in float (Ogita, Rump & Oishi 2005, Prop. 4.2 type):
    u|y| + gamma_n^2 sum|a||x|, gamma_n = n u / (1 - n u), plus one u|y|
    for the final rounding to float and n u^2 for the lane-combination."""
    n = np.maximum(lens, 1).astype(np.float64) + 6.0
    g = n * U32 / (1 - n * U32)
    return 2 * U32 * np.abs(ref) + (g * g + n * U32 * U32) * s


@functools.lru_cache(maxsize=None)
def full_config(i):
    return S.config(i)


def adversarial_matrices():
    """Edge cases: empty rows, one row, no entries, one long row, warp
    boundaries, rectangular shapes."""
    out = []
    out.append(S.CRS(1, 1, np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0), "empty_1x1"))
    out.append(S.CRS(7, 5, np.zeros(8, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty_7x5"))
    out.append(S.from_coo(1, 1, [0], [0], [3.0], name="one"))
    out.append(S.from_coo(3, 5000, [1] * 5000, np.arange(5000),
                          S.uniform(5, 1, np.arange(5000), -1, 1), name="long_row_5000"))
    # rows of length 31, 32, 33 and neighbours, straddling warp boundaries
    rows, cols = [], []
    for i, l in enumerate([31, 32, 33, 1, 0, 64, 63, 65, 2, 33, 31, 0, 97]):
        rows += [i] * l
        cols += list(range(l))
    out.append(S.from_coo(13, 100, rows, cols, S.uniform(6, 1, np.arange(len(rows)), -1, 1),
                          name="warp_edges"))
    out.append(S.small_random(300, 77, 7, density=0.1, empty_rows=0.3))
    out.append(S.small_random(64, 300, 8, density=0.05, empty_rows=0.1))
    out.append(S.zipf_rows(20000, 9, lmax=3000))
    # lengths on both sides of the kernels' long-row thresholds (64 for
    # RUNS, 512 for VECTOR) in random order: long rows at every position of
    # a lane group, several in one warp, next to empty rows
    pick = np.array([0, 1, 5, 63, 64, 65, 100, 511, 512, 513, 800])
    lens = pick[S.randint(10, 1, np.arange(3000), 0, len(pick) - 1)]
    rows = np.repeat(np.arange(3000), lens)
    t = np.arange(rows.size)
    pos = t - np.repeat(np.cumsum(lens) - lens, lens)  # position in the row
    cols = (rows * 37 + pos * 13) % 4000                # distinct within a row
    out.append(S.from_coo(3000, 4000, rows, cols, S.uniform(10, 3, t, -1, 1), name="long_row_thresholds"))
    return out
