"""Seeded synthetic sparse matrices and vectors.

This module only *builds inputs*; it holds none of the SpMVM arithmetic, so
both the CPU oracle tests and the CUDA path consume the very same arrays.

Randomness comes from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``t`` of stream ``s`` is ``mix(key(seed, s) + (t+1)*GAMMA)``.
Every draw is addressed by an integer counter, so the arrays are identical on
every machine and numpy version, and any single entry can be regenerated.

Matrices are returned as 0-based CRS (``row_ptr`` int32 of length n_rows+1,
``col`` int32, ``val`` float64) with column indices sorted inside each row.

Workload recipes (the paper's Holstein-Hubbard matrix, Sect. 4.2, is not
available, so these stand in for it):

* ``laplace2d``     2D 5-point Laplacian, Dirichlet, 4 on the diagonal.
* ``hh_like``       symmetric banded-plus-scattered matrix shaped like the
                    paper's electron-phonon Hamiltonian (Sect. 4.2: dense
                    secondary diagonals, scattered entries, ~14 nnz/row).
* ``zipf_rows``     irregular rows, lengths truncated Zipf(2) on [1, 5000],
                    uniform random columns.
* ``stencil7`` / ``stencil27``  3D stencils.
* ``random_rows``   U{lo..hi} entries per row, uniform random columns.
* ``batch_set``     256 uneven matrices, half 7-point stencils, half random.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function (Steele et al. 2014)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D)
                         & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix(base)[0]


def bits(seed: int, stream: int, counter) -> np.ndarray:
    """64 random bits for each counter value (array-like of non-negative ints)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(_stream_key(seed, stream) + (c + np.uint64(1)) * _GAMMA)


def uniform01(seed: int, stream: int, counter) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits scaled by 2^-53."""
    return (bits(seed, stream, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, stream: int, counter, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, counter)


def randint(seed: int, stream: int, counter, lo, hi) -> np.ndarray:
    """Integers in [lo, hi] (inclusive; lo/hi may be arrays)."""
    lo = np.asarray(lo, dtype=np.int64)
    span = np.asarray(hi, dtype=np.int64) - lo + 1
    u = uniform01(seed, stream, counter)
    r = np.floor(u * span).astype(np.int64)
    return lo + np.minimum(r, span - 1)


def normal(seed: int, stream: int, counter) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = 1.0 - uniform01(seed, stream, counter)          # (0, 1]
    u2 = uniform01(seed, stream + 7919, counter)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class CRS:
    """A 0-based CRS matrix held in host numpy arrays."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray   # int32 [n_rows + 1]
    col: np.ndarray       # int32 [nnz]
    val: np.ndarray       # float64 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def row_ids(self) -> np.ndarray:
        """Row index of every stored entry, in storage order."""
        return np.repeat(np.arange(self.n_rows, dtype=np.int32), self.row_lengths())

    def astype(self, dtype) -> "CRS":
        return CRS(self.n_rows, self.n_cols, self.row_ptr, self.col,
                   self.val.astype(dtype), self.name)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n_rows, self.n_cols), dtype=self.val.dtype)
        d[self.row_ids(), self.col] = self.val
        return d


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    """Sorted distinct values (a plain sort plus an adjacent-difference mask)."""
    key = np.sort(key)
    if key.size:
        keep = np.empty(key.size, dtype=bool)
        keep[0] = True
        np.not_equal(key[1:], key[:-1], out=keep[1:])
        key = key[keep]
    return key


def from_coo(n_rows: int, n_cols: int, rows, cols, vals=None, *, dedupe: bool = True,
             name: str = "") -> CRS:
    """Sort coordinates by (row, col) into CRS; duplicates keep the first value."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(n_cols) + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    if dedupe and key.size:
        keep = np.empty(key.size, dtype=bool)
        keep[0] = True
        np.not_equal(key[1:], key[:-1], out=keep[1:])
        key, order = key[keep], order[keep]
    r = key // n_cols
    c = key - r * n_cols
    counts = np.bincount(r, minlength=n_rows)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 indices")
    v = (np.zeros(len(key)) if vals is None else np.asarray(vals)[order]).astype(np.float64)
    return CRS(n_rows, n_cols, row_ptr.astype(np.int32), c.astype(np.int32), v, name)


def vector(n: int, seed: int, stream: int = 101, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """A dense vector with entries uniform in [lo, hi)."""
    return uniform(seed, stream, np.arange(n), lo, hi)


def int_vector(n: int, seed: int, bound: int, stream: int = 103) -> np.ndarray:
    """Integer-valued float64 vector with entries in [-bound, bound]."""
    return randint(seed, stream, np.arange(n), -bound, bound).astype(np.float64)


# --------------------------------------------------------------------------
# Index arrays for the basic gather operations (Sect. 4.1: dense, constant
# stride, indirect with constant or random stride)
# --------------------------------------------------------------------------

def stride_indices(n: int, k: int) -> np.ndarray:
    """ind(i) = k*i for i < n (the IS case), int32."""
    if n > 0 and k * (n - 1) >= 2 ** 31:
        raise ValueError("stride_indices: k*(n-1) exceeds int32")
    return (np.arange(n, dtype=np.int64) * k).astype(np.int32)


def bernoulli_indices(length: int, p: float, seed: int, stream: int = 211) -> np.ndarray:
    """The IR index array as Sect. 4.1 draws it: every position j < length
    of the gathered vector is taken when a uniform draw is below p = 1/k."""
    j = np.arange(length, dtype=np.int64)
    return j[uniform01(seed, stream, j) < p].astype(np.int32)


def geometric_indices(n: int, p: float, seed: int, stream: int = 213) -> np.ndarray:
    """n indices with the gap law of ``bernoulli_indices`` (gaps Geometric(p)
    on {1, 2, ...}: mean 1/p, variance (1-p)/p^2), drawn gap by gap by
    inversion, so that long index arrays need no draw per skipped position.
    The first index is the first gap minus one."""
    if p >= 1.0:
        gaps = np.ones(n, dtype=np.int64)
    else:
        u = 1.0 - uniform01(seed, stream, np.arange(n))      # (0, 1]
        gaps = 1 + np.floor(np.log(u) / np.log1p(-p)).astype(np.int64)
    ind = np.cumsum(gaps) - 1
    if n > 0 and ind[-1] >= 2 ** 31:
        raise ValueError("geometric_indices: indices exceed int32")
    return ind.astype(np.int32)


def uniform_indices(n: int, length: int, seed: int, stream: int = 219) -> np.ndarray:
    """n indices uniform on [0, length), int32: the x gathers of a matrix
    with uniformly random columns (the Zipf-rows workload), as an index
    array for the basic gather sums."""
    if length > 2 ** 31:
        raise ValueError("uniform_indices: length exceeds int32")
    u = uniform01(seed, stream, np.arange(n))
    return np.minimum((u * length).astype(np.int64), length - 1).astype(np.int32)


def gaussian_indices(n: int, mean: float, var: float, length: int, seed: int,
                     stream: int = 217) -> np.ndarray:
    """Indices whose strides are normal(mean, var) rounded to integers, so
    that backward jumps occur once the variance is large enough (the
    mean/variance plane of Sect. 4.1).  ind(0) = 0 and every step wraps
    modulo `length`, which keeps the walk inside the vector."""
    z = normal(seed, stream, np.arange(1, n))
    steps = np.rint(mean + np.sqrt(var) * z).astype(np.int64)
    ind = np.concatenate([[0], np.cumsum(steps)]) % length
    return ind.astype(np.int32)


# --------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------

def laplace2d(nx: int = 64, ny: int = 64) -> CRS:
    """2D 5-point Laplacian on an nx*ny grid, Dirichlet boundary: 4 on the
    diagonal, -1 for each in-grid neighbour.  64x64 gives N=4096, nnz=20,224."""
    n = nx * ny
    i = np.arange(n, dtype=np.int64)
    gx, gy = i % nx, i // nx
    rows, cols, vals = [i], [i], [np.full(n, 4.0)]
    for dx, dy in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (gx + dx >= 0) & (gx + dx < nx) & (gy + dy >= 0) & (gy + dy < ny)
        rows.append(i[ok])
        cols.append(i[ok] + dx + dy * nx)
        vals.append(np.full(int(ok.sum()), -1.0))
    return from_coo(n, n, np.concatenate(rows), np.concatenate(cols),
                    np.concatenate(vals), dedupe=False, name=f"laplace2d_{nx}x{ny}")


HH_BAND_OFFSETS = (1, 256, 512, 768, 1024, 65536, 131072, 196608, 262144)


def hh_like(n: int = 6_000_000, seed: int = 1) -> CRS:
    """Symmetric banded-plus-scattered matrix shaped like a Holstein-Hubbard
    Hamiltonian (Sect. 4.2).

    Row i draws m_i ~ U{3..10} upper-triangle neighbours.  Each neighbour is,
    with probability 0.8, at a band offset drawn uniformly from
    {1, 256k, 65536k : k=1..4} (offsets >= 256 jittered by U{-2..2}), else a
    uniform column in (i, n).  Columns >= n are dropped, duplicates removed,
    the pattern mirrored with equal values normal(0,1), and a normal(0,1)
    diagonal added.  Mean row length is about 14, as the paper's test matrix.
    """
    rows_m = randint(seed, 1, np.arange(n), 3, 10)
    i = np.repeat(np.arange(n, dtype=np.int64), rows_m)
    t = np.arange(i.size, dtype=np.int64)
    band = uniform01(seed, 2, t) < 0.8
    offs = np.asarray(HH_BAND_OFFSETS, dtype=np.int64)[randint(seed, 3, t, 0, len(HH_BAND_OFFSETS) - 1)]
    jit = np.where(offs >= 256, randint(seed, 4, t, -2, 2), 0)
    j_band = i + offs + jit
    j_rand = randint(seed, 5, t, i + 1, max(n - 1, 1))
    j = np.where(band, j_band, j_rand)
    keep = (j > i) & (j < n)
    i, j = i[keep], j[keep]
    upper = _sorted_unique(i * n + j)
    del i, j, keep, t, band, offs, jit, j_band, j_rand
    ui, uj = upper // n, upper % n
    diag = np.arange(n, dtype=np.int64)
    key = np.concatenate([upper, uj * n + ui, diag * n + diag])
    del ui, uj
    key.sort()
    r = key // n
    c = key - r * n
    lo = np.minimum(r, c)
    hi = np.maximum(r, c)
    val = np.where(r == c, normal(seed, 7, r), normal(seed, 6, lo * n + hi))
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CRS(n, n, row_ptr.astype(np.int32), c.astype(np.int32), val, f"hh_like_{n}")


HH_OUTER_OFFSETS = tuple(65536 * k for k in range(1, 7))


def hh_diagonals(n: int = 6_000_000, seed: int = 5, fill: float = 0.8, band: int = 400) -> CRS:
    """Symmetric stand-in that follows Sect. 4.2's description of the
    Holstein-Hubbard matrix literally: some 60% of the entries on 12 outer
    secondary diagonals, the rest spread evenly over a band a few hundred
    diagonals wide.

    Six upper offsets 65536k (k = 1..6) each hold an entry in row i with
    probability `fill`; row i also draws U{1..4} upper entries at offsets
    uniform in [1, band].  Columns >= n are dropped, duplicates removed, the
    pattern mirrored with equal values normal(0,1), and a normal(0,1)
    diagonal added: at n = 6e6 about 15 entries a row, 60% of them on the
    twelve outer diagonals."""
    i_all = np.arange(n, dtype=np.int64)
    parts_i, parts_j = [], []
    for k, o in enumerate(HH_OUTER_OFFSETS):
        keep = (uniform01(seed, 20 + k, i_all) < fill) & (i_all + o < n)
        parts_i.append(i_all[keep])
        parts_j.append(i_all[keep] + o)
    m = randint(seed, 30, i_all, 1, 4)
    i = np.repeat(i_all, m)
    t = np.arange(i.size, dtype=np.int64)
    j = i + randint(seed, 31, t, 1, band)
    keep = j < n
    parts_i.append(i[keep])
    parts_j.append(j[keep])
    i = np.concatenate(parts_i)
    j = np.concatenate(parts_j)
    upper = _sorted_unique(i * n + j)
    del i, j, keep, t, parts_i, parts_j
    ui, uj = upper // n, upper % n
    key = np.concatenate([upper, uj * n + ui, i_all * n + i_all])
    del ui, uj
    key.sort()
    r = key // n
    c = key - r * n
    lo = np.minimum(r, c)
    hi = np.maximum(r, c)
    val = np.where(r == c, normal(seed, 33, r), normal(seed, 32, lo * n + hi))
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CRS(n, n, row_ptr.astype(np.int32), c.astype(np.int32), val, f"hh_diagonals_{n}")


def zipf_lengths(n: int, seed: int, s: float = 2.0, lmin: int = 1, lmax: int = 5000,
                 stream: int = 11) -> np.ndarray:
    """Row lengths from Zipf(s) truncated (renormalised) to [lmin, lmax]."""
    k = np.arange(lmin, lmax + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-s))
    cdf /= cdf[-1]
    u = uniform01(seed, stream, np.arange(n))
    return lmin + np.minimum(np.searchsorted(cdf, u, side="right"), lmax - lmin)


def zipf_rows(n: int = 4_000_000, seed: int = 2, lmax: int = 5000) -> CRS:
    """Irregular matrix: row lengths truncated Zipf(2) on [1, lmax], uniform
    random columns (deduplicated, so a row may come out slightly shorter),
    values uniform in [-1, 1)."""
    lens = zipf_lengths(n, seed, lmax=lmax)
    i = np.repeat(np.arange(n, dtype=np.int64), lens)
    c = randint(seed, 12, np.arange(i.size), 0, n - 1)
    key = _sorted_unique(i * n + c)
    del i, c
    r = key // n
    c = key - r * n
    val = uniform(seed, 13, key, -1.0, 1.0)
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CRS(n, n, row_ptr.astype(np.int32), c.astype(np.int32), val, f"zipf_rows_{n}")


def _stencil(dims, offsets, seed: int, values: str, name: str) -> CRS:
    nx, ny, nz = dims
    n = nx * ny * nz
    p = np.arange(n, dtype=np.int64)
    x, y, z = p % nx, (p // nx) % ny, p // (nx * ny)
    rows, cols = [], []
    for dx, dy, dz in offsets:
        ok = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
              & (z + dz >= 0) & (z + dz < nz))
        rows.append(p[ok])
        cols.append(p[ok] + dx + dy * nx + dz * nx * ny)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    key = rows * n + cols
    key.sort()
    r = key // n
    c = key - r * n
    if values == "laplace":
        val = np.where(r == c, float(len(offsets) - 1), -1.0)
    elif values == "contractive":
        val = np.where(r == c, 0.5, uniform(seed, 21, key, -1.0, 1.0) / 52.0)
    elif values == "contractive_sym":
        lo, hi = np.minimum(r, c), np.maximum(r, c)
        val = np.where(r == c, 0.5, uniform(seed, 21, lo * n + hi, -1.0, 1.0) / 52.0)
    else:
        raise ValueError(values)
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CRS(n, n, row_ptr.astype(np.int32), c.astype(np.int32), val.astype(np.float64), name)


def stencil7(nx: int, ny: int, nz: int) -> CRS:
    """3D 7-point stencil, 6 on the diagonal, -1 off it."""
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return _stencil((nx, ny, nz), offs, 0, "laplace", f"stencil7_{nx}x{ny}x{nz}")


def stencil27(m: int = 100, seed: int = 4, symmetric_values: bool = False) -> CRS:
    """3D 27-point stencil on an m^3 grid with a_ii = 1/2 and off-diagonal
    values uniform in [-1, 1)/52, so every absolute row sum is below 1 and
    A^20 x neither overflows nor underflows.  ``symmetric_values`` draws each
    off-diagonal pair from one counter so that A is symmetric."""
    offs = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)]
    kind = "contractive_sym" if symmetric_values else "contractive"
    return _stencil((m, m, m), offs, seed, kind, f"stencil27_{m}^3" + ("_sym" if symmetric_values else ""))


def random_rows(n: int, seed: int, lo: int = 5, hi: int = 30, n_cols: int | None = None,
                stream: int = 31) -> CRS:
    """Each row draws U{lo..hi} uniform random columns (deduplicated); values
    uniform in [-1, 1)."""
    n_cols = n if n_cols is None else n_cols
    lens = randint(seed, stream, np.arange(n), lo, hi)
    i = np.repeat(np.arange(n, dtype=np.int64), lens)
    c = randint(seed, stream + 1, np.arange(i.size), 0, n_cols - 1)
    key = _sorted_unique(i * n_cols + c)
    r = key // n_cols
    c = key - r * n_cols
    val = uniform(seed, stream + 2, key, -1.0, 1.0)
    counts = np.bincount(r, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CRS(n, n_cols, row_ptr.astype(np.int32), c.astype(np.int32), val,
               f"random_rows_{n}x{n_cols}")


def batch_sizes(count: int = 256, seed: int = 3, lo: float = 1e3, hi: float = 2e5) -> np.ndarray:
    """Matrix dimensions log-uniform in [lo, hi]."""
    u = uniform01(seed, 41, np.arange(count))
    return np.round(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batch_set(count: int = 256, seed: int = 3, lo: float = 1e3, hi: float = 2e5) -> list[CRS]:
    """Uneven matrices: even indices are 7-point stencils on an a*a*c grid
    (a = floor(N^(1/3)), c = round(N/a^2), so the realised N is a*a*c), odd
    indices random with U{5..30} entries per row."""
    out = []
    for b, n in enumerate(batch_sizes(count, seed, lo, hi)):
        if b % 2 == 0:
            a = max(int(math.floor(n ** (1.0 / 3.0) + 1e-9)), 1)
            c = max(int(round(n / (a * a))), 1)
            out.append(stencil7(a, a, c))
        else:
            out.append(random_rows(int(n), seed * 1000 + b, 5, 30))
    return out


def batch_k(count: int, mode: str) -> list[int]:
    """Right-hand-side counts: uniform 1, 4 or 16, or mixed {1,4,16}[b mod 3]."""
    if mode == "mixed":
        return [(1, 4, 16)[b % 3] for b in range(count)]
    return [int(mode)] * count


def integer_values(a: CRS, seed: int, bound: int, stream: int = 51) -> CRS:
    """Same pattern with integer values in [-bound, bound] (zeros kept as
    stored entries), for exact-arithmetic checks."""
    v = randint(seed, stream, np.arange(a.nnz), -bound, bound).astype(np.float64)
    return CRS(a.n_rows, a.n_cols, a.row_ptr, a.col, v, a.name + "_int")


def small_random(n_rows: int, n_cols: int, seed: int, density: float = 0.05,
                 empty_rows: float = 0.0) -> CRS:
    """Tiny random matrix for exhaustive checks; ``empty_rows`` is the
    fraction of rows forced empty."""
    r, c = np.meshgrid(np.arange(n_rows), np.arange(n_cols), indexing="ij")
    r, c = r.ravel(), c.ravel()
    t = np.arange(r.size)
    keep = uniform01(seed, 61, t) < density
    if empty_rows > 0:
        dead = uniform01(seed, 62, np.arange(n_rows)) < empty_rows
        keep &= ~dead[r]
    vals = uniform(seed, 63, t, -1.0, 1.0)
    return from_coo(n_rows, n_cols, r[keep], c[keep], vals[keep], name=f"small_{n_rows}x{n_cols}")


def long_rows(n: int, long_lengths, seed: int, short_max: int = 6) -> CRS:
    """``n`` rows of U{0..short_max} entries plus, at rows spread through the
    matrix, rows of the given (long) lengths; uniform random columns.  Rows
    longer than 2^17 entries with more than 2^15 windows push the windowed
    length sort of SELL past a 32-bit key."""
    lens = randint(seed, 71, np.arange(n), 0, short_max).astype(np.int64)
    at = [(k + 1) * n // (len(long_lengths) + 1) for k in range(len(long_lengths))]
    for r, l in zip(at, long_lengths):
        lens[r] = min(int(l), n)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    t = np.arange(rows.size)
    cols = randint(seed, 72, t, 0, n - 1).astype(np.int64)
    for r, l in zip(at, long_lengths):  # the long rows: distinct columns
        sel = rows == r
        cols[sel] = (r + np.arange(sel.sum(), dtype=np.int64) * 7) % n
    vals = uniform(seed, 73, t, -1.0, 1.0)
    return from_coo(n, n, rows, cols, vals, name=f"long_rows_{n}")


# ----------------------------------------------------- index-limit matrix --
# The largest matrix whose CRS fits the int32 index arrays the library takes:
# nnz = 2^31 - 2^16 - 1 (the library keeps 2^16 entries of headroom), on
# 2^24 rows of ragged length 7..248.  Entries are closed-form functions of
# (row, position in row), so any row can be regenerated on the host, and the
# whole matrix on the device, from the same expressions.  The functions take
# int64 numpy arrays or int64 torch tensors alike.
LIMIT_NNZ = 2 ** 31 - 2 ** 16 - 1
LIMIT_ROWS = 2 ** 24


def limit_lengths(i):
    """Row lengths: pairs (2p, 2p+1) get 128 +/- h(p), h in [-120, 120], so
    each pair holds 256 entries; the first 2^16 + 1 rows lose one entry."""
    h = ((i // 2) * 2654435761) % 241 - 120
    return 128 + (1 - 2 * (i % 2)) * h - (i < 2 ** 16 + 1) * 1


def limit_cols(i, j):
    """Column of entry j of row i: distinct within a row (131 is odd); rows
    whose columns wrap past the last column are not sorted, which CRS
    allows."""
    return (i * 7 + j * 131 + 1000) % LIMIT_ROWS


def limit_vals(i, j):
    """Integer values in [-3, 3]."""
    return (i + 3 * j) % 7 - 3


def limit_x(c):
    """Integer x in [-5, 5]; with the values above every row sum is an
    integer below 2^12, exact in any summation order."""
    return c % 11 - 5


def limit_rows_crs(rows) -> CRS:
    """Only the given rows of the index-limit matrix, as a CRS with one row
    per requested row and the full column range (host side)."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = limit_lengths(rows)
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    r = np.repeat(rows, lens)
    j = np.arange(rp[-1], dtype=np.int64) - np.repeat(rp[:-1], lens)
    return CRS(len(rows), LIMIT_ROWS, rp.astype(np.int32), limit_cols(r, j).astype(np.int32),
               limit_vals(r, j).astype(np.float64), "limit_rows")


def config(i: int) -> CRS:
    """The five workload matrices by index (0: Laplacian 64x64, 1: HH-like
    N=6e6, 2: Zipf rows N=4e6, 4: 27-point stencil 100^3).  Index 3 is the
    batch, see ``batch_set``."""
    if i == 0:
        return laplace2d(64, 64)
    if i == 1:
        return hh_like(6_000_000, 1)
    if i == 2:
        return zipf_rows(4_000_000, 2)
    if i == 4:
        return stencil27(100, 4)
    raise ValueError("config 3 is a batch: use batch_set()")
