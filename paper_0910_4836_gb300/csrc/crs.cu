// CRS products (Sect. 2, CRS kernel: y_i = sum over row i of val_j x[col_j]).
//
// VECTOR: a warp is cut into groups of L lanes; each group owns one row at a
// time and strides through its entries (lane l takes entries l, l+L, ...),
// so a warp-wide load covers 32/L adjacent rows' entries contiguously.  Each
// group keeps R rows in flight: the loads of all R rows are issued before
// any product is formed, which is what keeps enough bytes in flight to
// saturate HBM with short rows.  The partial sums are combined by a fixed
// butterfly of warp shuffles; when a group holds as many rows as it has
// lanes, by a reduce-scatter that leaves each lane one row's total (same
// tree, fewer FP64 additions: on GB300 each one is a full-rate-limited FP64
// instruction).  In a warp whose rows include one longer than kLongRow, the
// groups take their rows one at a time and the long rows are then summed by
// the whole warp.
//
// RUNS: as VECTOR, but a group's rows are consecutive and its lanes stride
// through their entries as one run (below).
//
// SpMM: lanes over right-hand sides -- a group of KT lanes owns one row and
// lane c accumulates column c of the RHS tile, so each entry (val, col) is
// read once per tile and X's row slice is read as one contiguous segment.
//
// All three run in CTAs of two warps, one CTA per two warps' worth of rows
// (row_grid below).
#include <algorithm>

#include "accum.cuh"
#include "internal.cuh"

namespace gbsp {

constexpr int kThreads = 256;
// Row length beyond which a row is summed by the whole warp instead of its
// lane group: VECTOR (lanes run to the group's longest row) and RUNS (whose
// groups share one run, so a long row would hold its whole group).
constexpr int kLongRow = 512;
constexpr int kRunsLongRow = 64;

// Flagged rows with the whole warp on each row in turn.  Every lane passes
// its group's mask (bit i: row first + i * step is long; only `leader`
// lanes' masks are read); lanes stride through a row four loads deep, then
// a full-warp sum.  Called only from the out-of-line long-row steps below,
// so it does not weigh on the common path's registers.
template <int VM>
__device__ __forceinline__ void crs_warp_long_rows(bool leader, unsigned mask, int64_t first, int64_t step,
                                                const int32_t *__restrict__ row_ptr,
                                                const int32_t *__restrict__ col,
                                                const typename ValT<VM>::T *__restrict__ val,
                                                const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                                                typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    typedef typename ValT<VM>::T T;
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, leader && mask != 0);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        unsigned m = __shfl_sync(0xffffffffu, mask, src);
        const int64_t f = __shfl_sync(0xffffffffu, first, src);
        while (m) {
            const int64_t r = f + (int64_t)(__ffs(m) - 1) * step;
            m &= m - 1;
            const int s0 = __ldg(row_ptr + r), s1 = __ldg(row_ptr + r + 1);
            Acc<VM> a;
            a.init();
            for (int j = s0 + lane; j < s1; j += 4 * 32) {
                int c[4];
                T v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool ok = j + 32 * u < s1;
                    c[u] = ok ? __ldg(col + j + 32 * u) : -1;
                    v[u] = ok ? __ldg(val + j + 32 * u) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c[u] >= 0) a.add(v[u], ld_vec(x + (int64_t)c[u] * ldx));
            }
            group_reduce<32, VM>(a);
            if (lane == 0) {
                if (accumulate) a.add_value(y[r * ldy]);
                y[r * ldy] = a.result();
            }
        }
    }
}

// The step of a warp that holds a very long row (heavy-tailed row lengths),
// for VECTOR and RUNS alike: group g's rows are first_g + i step, i < R.
// Rows up to `thr` entries are summed one at a time by their group's L lanes
// (four loads in flight per lane, then the group's butterfly); longer rows,
// which would keep their group busy long after the rest of the warp is done,
// are then summed by the whole warp.  Out of line, and light on registers,
// so that the common step keeps its own.
template <int VM, int L>
__device__ __noinline__ void crs_step_with_long_rows(int R, int64_t first, int64_t step, int thr, int64_t n_rows,
                                                     const int32_t *__restrict__ row_ptr,
                                                     const int32_t *__restrict__ col,
                                                     const typename ValT<VM>::T *__restrict__ val,
                                                     const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                                                     typename ValT<VM>::T *__restrict__ y, int64_t ldy,
                                                     int accumulate) {
    typedef typename ValT<VM>::T T;
    const int gl = (threadIdx.x & 31) % L;
    unsigned lmask = 0;
#pragma unroll 1
    for (int i = 0; i < R; ++i) {
        const int64_t r = first + i * step;
        int s0 = 0, s1 = 0;
        if (r < n_rows) {
            s0 = __ldg(row_ptr + r);
            s1 = __ldg(row_ptr + r + 1);
        }
        if (s1 - s0 > thr) {
            lmask |= 1u << i;
            s1 = s0;
        }
        Acc<VM> a;
        a.init();
        for (int j = s0 + gl; j < s1; j += 4 * L) {
            int c[4];
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = j + L * u < s1;
                c[u] = ok ? __ldg(col + j + L * u) : -1;
                v[u] = ok ? __ldg(val + j + L * u) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c[u] >= 0) a.add(v[u], ld_vec(x + (int64_t)c[u] * ldx));
        }
        group_reduce<L, VM>(a);
        if (gl == 0 && r < n_rows && !((lmask >> i) & 1u)) {
            if (accumulate) a.add_value(y[r * ldy]);
            y[r * ldy] = a.result();
        }
    }
    crs_warp_long_rows<VM>(gl == 0, lmask, first, step, row_ptr, col, val, x, ldx, y, ldy, accumulate);
}

// The occupancy hint (stated for 256-thread CTAs; the kernel is launched in
// two-warp CTAs, see row_grid) holds the common step at the registers it
// needs on its own (48 for four rows a group, 40 for fewer): without it, the
// call to the long-row step raised some shapes to 60.
template <int VM, int L, int R>
__global__ void __launch_bounds__(kThreads, R == 4 ? 5 : 6)
crs_vector_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                  const int32_t *__restrict__ col, const typename ValT<VM>::T *__restrict__ val,
                  const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                  typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    typedef typename ValT<VM>::T T;
    constexpr int G = 32 / L;
    constexpr int RW = G * R;
    const int lane = threadIdx.x & 31;
    const int grp = lane / L, gl = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * RW; base < n_rows; base += nwarp * RW) {
        int k0[R], k1[R];
        int len = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int64_t r = base + i * G + grp;
            k0[i] = 0;
            k1[i] = 0;
            if (r < n_rows) {
                k0[i] = __ldg(row_ptr + r);
                k1[i] = __ldg(row_ptr + r + 1);
            }
            len = max(len, k1[i] - k0[i]);
        }
        if (__reduce_max_sync(0xffffffffu, (unsigned)len) > (unsigned)kLongRow) {
            crs_step_with_long_rows<VM, L>(R, base + grp, G, kLongRow, n_rows, row_ptr, col, val, x, ldx, y, ldy,
                                              accumulate);
            continue;
        }
        Acc<VM> acc[R];
#pragma unroll
        for (int i = 0; i < R; ++i) acc[i].init();
        for (int j = gl; j < len; j += L) {
            int c[R];
            T v[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int k = k0[i] + j;
                const bool ok = k < k1[i];
                // read-only path, not evict-first: a lane group touches a
                // sector in several iterations, so it must survive in L1/L2
                c[i] = ok ? __ldg(col + k) : -1;
                v[i] = ok ? __ldg(val + k) : T(0);
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (c[i] >= 0) acc[i].add(v[i], ld_vec(x + (int64_t)c[i] * ldx));
        }
        if (R == L && VM != VM_F32C) {
            // reduce-scatter: log2(L) steps, each lane trading half of its
            // partial sums with its partner, so lane gl ends with row gl's
            // total after L - 1 additions instead of R log2(L).  The tree per
            // row is the xor butterfly of group_reduce with some additions'
            // operands swapped, which plain sums do not notice: every row's
            // sum is bit-identical to it.  (The compensated merge is not
            // symmetric in its error terms, so FP32C keeps the butterfly.)
#pragma unroll
            for (int o = L / 2, h = R / 2; o > 0; o >>= 1, h >>= 1) {
                const bool up = (gl & o) != 0;
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    Acc<VM> send = up ? acc[k] : acc[k + h];
                    Acc<VM> keep = up ? acc[k + h] : acc[k];
                    keep.merge_shfl_xor(send, o);
                    acc[k] = keep;
                }
            }
            const int64_t r = base + gl * G + grp;
            if (r < n_rows) {
                if (accumulate) acc[0].add_value(y[r * ldy]);
                y[r * ldy] = acc[0].result();
            }
        } else {
#pragma unroll
            for (int i = 0; i < R; ++i) group_reduce<L, VM>(acc[i]);
            if (gl == 0) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int64_t r = base + i * G + grp;
                    if (r < n_rows) {
                        if (accumulate) acc[i].add_value(y[r * ldy]);
                        y[r * ldy] = acc[i].result();
                    }
                }
            }
        }
    }
}

// Park a lane's running sum in its row's slot.  Indices are compile-time
// after unrolling, so the slots stay in registers (selects, no FP64 work).
template <int VM, int R>
__device__ __forceinline__ void park(Acc<VM> (&part)[R], int cur, const Acc<VM> &acc) {
#pragma unroll
    for (int m = 0; m < R; ++m)
        if (m == cur) part[m] = acc;
}

// RUNS: the R rows of a lane group are consecutive, so CRS stores their
// entries as one contiguous run, and the group's L lanes stride through that
// whole run (lane l takes run entries l, l+L, ...) instead of through each
// row up to the longest row's length.  A lane keeps one running FMA chain
// and parks it in the row's slot when its next entry lies in a later row
// (each row is one stretch of the run, so a slot is written once; register
// selects, no FP64 work); the slots are then combined over the group by the
// reduce-scatter, after which lane l holds rows (R/L) l .. (R/L) l + R/L - 1.
// FP64 lane-slots per warp: 32 x the longest group run / L, plus R (1 - 1/L)
// additions per lane, where VECTOR pays R x 32 x the longest row / L.  U
// entries per lane are loaded and gathered before any product is formed (U
// gathers in flight).
constexpr int kRunsU = 4;

// Reduce-scatter of the R row slots over the group's L lanes, then the
// stores (rows flagged in lmask are not stored).
template <int VM, int L, int R>
__device__ __forceinline__ void runs_store(Acc<VM> (&part)[R], int64_t rg, unsigned lmask, int64_t n_rows,
                                           typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    const int gl = (threadIdx.x & 31) % L;
#pragma unroll
    for (int o = L / 2, h = R / 2; o > 0; o >>= 1, h >>= 1) {
        const bool up = (gl & o) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            Acc<VM> send = up ? part[k] : part[k + h];
            Acc<VM> keep = up ? part[k + h] : part[k];
            keep.merge_shfl_xor(send, o);
            part[k] = keep;
        }
    }
    constexpr int Q = R / L;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int64_t r = rg + (int64_t)Q * gl + q;
        if (r < n_rows && !((lmask >> (Q * gl + q)) & 1u)) {
            if (accumulate) part[q].add_value(y[r * ldy]);
            y[r * ldy] = part[q].result();
        }
    }
}

// A RUNS step whose warp holds a row longer than kRunsLongRow: such rows are
// cut out of their group's run (its index skips them: run index j of row i
// sits at entry j + b_i - p_i, p_i the run length before row i) and summed
// afterwards by the whole warp.  Out of line, so that the common step keeps
// its code.
template <int VM, int L, int R>
__device__ __noinline__ void runs_step_cut(int64_t rg, int64_t n_rows, const int32_t *__restrict__ row_ptr,
                                           const int32_t *__restrict__ col,
                                           const typename ValT<VM>::T *__restrict__ val,
                                           const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                                           typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    typedef typename ValT<VM>::T T;
    constexpr int U = kRunsU;
    const int gl = (threadIdx.x & 31) % L;
    int b[R + 1], p[R];  // row pointers; run index of each row's start
#pragma unroll
    for (int i = 0; i <= R; ++i) b[i] = __ldg(row_ptr + min(rg + i, n_rows));
    unsigned lmask = 0;
    int n = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        p[i] = n;
        const int li = b[i + 1] - b[i];
        if (li > kRunsLongRow) lmask |= 1u << i;
        else n += li;
    }
    Acc<VM> part[R];
#pragma unroll
    for (int i = 0; i < R; ++i) part[i].init();
    Acc<VM> acc;
    acc.init();
    int cur = 0;
    for (int j = gl; j < n; j += U * L) {
        int c[U], row[U];
        T v[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int jj = j + u * L;
            // the last row starting at or before jj (a cut-out or empty row
            // starts where the next one does, which then wins)
            int i = 0, k = jj + b[0];
#pragma unroll
            for (int m = 1; m < R; ++m)
                if (jj >= p[m]) {
                    i = m;
                    k = jj + b[m] - p[m];
                }
            row[u] = i;
            const bool ok = jj < n;
            c[u] = ok ? __ldg(col + k) : -1;
            v[u] = ok ? __ldg(val + k) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? ld_vec(x + (int64_t)c[u] * ldx) : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (c[u] >= 0) {
                if (row[u] != cur) {
                    park<VM, R>(part, cur, acc);
                    acc.init();
                    cur = row[u];
                }
                acc.add(v[u], xv[u]);
            }
        }
    }
    park<VM, R>(part, cur, acc);
    runs_store<VM, L, R>(part, rg, lmask, n_rows, y, ldy, accumulate);
    crs_warp_long_rows<VM>(gl == 0, lmask, rg, 1, row_ptr, col, val, x, ldx, y, ldy, accumulate);
}

template <int VM, int L, int R>
__global__ void __launch_bounds__(kThreads, R == 4 ? 5 : 4)
crs_runs_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col, const typename ValT<VM>::T *__restrict__ val,
                const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    typedef typename ValT<VM>::T T;
    static_assert(R >= L && R % L == 0, "a group's rows must divide over its lanes");
    constexpr int G = 32 / L;
    constexpr int RW = G * R;
    constexpr int U = kRunsU;
    const int lane = threadIdx.x & 31;
    const int grp = lane / L, gl = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * RW; base < n_rows; base += nwarp * RW) {
        const int64_t rg = base + (int64_t)grp * R;
        int b[R + 1];
#pragma unroll
        for (int i = 0; i <= R; ++i) b[i] = __ldg(row_ptr + min(rg + i, n_rows));
        int longest = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) longest = max(longest, b[i + 1] - b[i]);
        if (__reduce_max_sync(0xffffffffu, (unsigned)longest) > (unsigned)kRunsLongRow) {
            runs_step_cut<VM, L, R>(rg, n_rows, row_ptr, col, val, x, ldx, y, ldy, accumulate);
            continue;
        }
        Acc<VM> part[R];
#pragma unroll
        for (int i = 0; i < R; ++i) part[i].init();
        Acc<VM> acc;
        acc.init();
        int cur = 0;
        const int k0 = b[0], n = b[R] - b[0];
        for (int j = gl; j < n; j += U * L) {
            int c[U];
            T v[U], xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = j + u * L < n;
                c[u] = ok ? __ldg(col + k0 + j + u * L) : -1;
                v[u] = ok ? __ldg(val + k0 + j + u * L) : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? ld_vec(x + (int64_t)c[u] * ldx) : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (c[u] >= 0) {
                    const int k = k0 + j + u * L;
                    int i = 0;
#pragma unroll
                    for (int m = 1; m < R; ++m) i += k >= b[m] ? 1 : 0;
                    if (i != cur) {
                        park<VM, R>(part, cur, acc);
                        acc.init();
                        cur = i;
                    }
                    acc.add(v[u], xv[u]);
                }
            }
        }
        park<VM, R>(part, cur, acc);
        runs_store<VM, L, R>(part, rg, 0u, n_rows, y, ldy, accumulate);
    }
}

template <int VM, int KT>
__global__ void __launch_bounds__(kThreads)
crs_spmm_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col, const typename ValT<VM>::T *__restrict__ val,
                const typename ValT<VM>::T *__restrict__ X, int64_t ldx,
                typename ValT<VM>::T *__restrict__ Y, int64_t ldy, int k, int c0, int accumulate) {
    typedef typename ValT<VM>::T T;
    constexpr int G = 32 / KT;
    const int lane = threadIdx.x & 31;
    const int grp = lane / KT, c = lane % KT;
    const int cc = c0 + c;
    const bool active = cc < k;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp * G + grp; r - grp < n_rows; r += nwarp * G) {
        if (r >= n_rows) continue;
        const int k0 = __ldg(row_ptr + r), k1 = __ldg(row_ptr + r + 1);
        Acc<VM> acc;
        acc.init();
        int j = k0;
        for (; j + 4 <= k1; j += 4) {
            int ci[4];
            T vi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ci[u] = __ldg(col + j + u);
                vi[u] = __ldg(val + j + u);
            }
            if (active) {
#pragma unroll
                for (int u = 0; u < 4; ++u) acc.add(vi[u], ld_vec(X + (int64_t)ci[u] * ldx + cc));
            }
        }
        for (; j < k1; ++j) {
            const int ci = __ldg(col + j);
            const T vi = __ldg(val + j);
            if (active) acc.add(vi, ld_vec(X + (int64_t)ci * ldx + cc));
        }
        if (active) {
            T *yp = Y + r * ldy + cc;
            if (accumulate) acc.add_value(*yp);
            *yp = acc.result();
        }
    }
}

// The row (0..31, of a warp's 32 rows) of entry cb + lane, for a warp that
// holds its rows' starts (rs) and ends (re) one per lane; every lane takes
// part.  An entry belongs to the last nonempty row starting at or before
// it.  Row i marks position max(start_i - cb, 0) of the 32-entry chunk at
// cb when it is nonempty there (the row holding entry cb marks 0; rows
// ending by cb, empty rows and rows starting past the chunk mark nothing),
// so each marked position has exactly one row.  B: the marked positions,
// from one warp-wide OR; C: the marking rows, from one ballot.  Both are in
// increasing order, so the lane's row is the k-th set bit of C, k the
// number of marks at or below its position, less one: the first marking row
// plus k when they are consecutive (no empty rows among them), else a
// popcount halving.  No shuffles: they share the L1TEX data pipe with the
// loads.  Lanes past the warp's last entry get an unspecified row.
__device__ __forceinline__ int chunk_row(int32_t rs, int32_t re, int32_t cb, int lane) {
    const int32_t ds = max(rs - cb, 0), de = max(re - cb, 0);
    const bool mark = ds < 32 && de > ds;
    const unsigned B = __reduce_or_sync(0xffffffffu, mark ? 1u << ds : 0u);
    const unsigned C = __ballot_sync(0xffffffffu, mark);
    int k = __popc(B & (0xffffffffu >> (31 - lane))) - 1;
    int r = C ? __ffs(C) - 1 : 0;  // no marks: a chunk past the warp's entries
    if (!((C >> r) & ((C >> r) + 1))) return r + k;
    unsigned m = C;
    r = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int n = __popc(m & ((1u << w) - 1u));
        if (n <= k) {
            k -= n;
            m >>= w;
            r += w;
        }
    }
    return r;
}

// dval_k: d = (accumulate ? dval_k : 0), then d = fma(G[row_k, t], X[col_k, t], d)
// for t = 0, 1, ..., m-1 (m = 1: g[row] x[col]).  One running sum in a fixed
// order, so splitting the t range over several calls changes nothing.
// Both kernels give a warp 32 consecutive rows and walk their entries in
// chunks of 32: lane l takes entry c + l of chunk c, so every col load and
// dval store is one contiguous warp-wide access.
//   m = 1 (crs_dval_kernel): kDvalU chunks in flight together (their
//     gathers are what the kernel waits for); the warp's 32 row starts and
//     ends sit one per lane, and a lane finds its entry's row from one
//     warp-wide OR of the rows' start positions in the chunk and one ballot
//     (no shuffles: a five-step shuffle search per chunk took 42% of the
//     L1TEX data-pipe wavefronts); dval is written evict-first (it is not
//     read again here), which leaves L2 to the gathered vectors.
//   m > 1 (crs_dval_multi_kernel): one chunk at a time, rows found by
//     stepping forward through the row pointers in shared memory.  With
//     the loop over t inside, several chunks in flight took 72 registers
//     and ran slower (27-point stencil, m = 5: 287 us against 249 us); so did
//     the shuffle-free row lookup with one or two chunks in flight and one or
//     two steps loaded together (294-490 us against 259 us).
constexpr int kDvalWarps = kThreads / 32;
constexpr int kDvalU = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads)
crs_dval_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col, int m, const T *__restrict__ G, int64_t g_row,
                int64_t g_t, const T *__restrict__ X, int64_t x_row, int64_t x_t, T *__restrict__ dval,
                int accumulate) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 32; r0 < n_rows; r0 += nwarp * 32) {
        // lane i: start of row r0 + i (rows past the end start at nnz)
        const int32_t rpl = __ldg(row_ptr + min(r0 + lane, n_rows));
        const int32_t e1 = __ldg(row_ptr + min(r0 + 32, n_rows));
        const int32_t eb = __shfl_sync(0xffffffffu, rpl, 0);
        const T *Gw = G + r0 * g_row;
        // lane i: end of row r0 + i
        const int32_t rpn = __ldg(row_ptr + min(r0 + lane + 1, n_rows));
        for (int32_t c = eb; c < e1; c += 32 * kDvalU) {
            int32_t cj[kDvalU], rl[kDvalU];
            T d[kDvalU];
#pragma unroll
            for (int u = 0; u < kDvalU; ++u) {
                const int32_t cb = c + 32 * u;
                const int32_t e = cb + lane;
                rl[u] = chunk_row(rpl, rpn, cb, lane);
                cj[u] = e < e1 ? ld_stream(col + e) : -1;
            }
#pragma unroll
            for (int u = 0; u < kDvalU; ++u) {
                const int32_t e = c + 32 * u + lane;
                d[u] = cj[u] >= 0 ? fma(__ldg(Gw + rl[u] * g_row), __ldg(X + (int64_t)cj[u] * x_row),
                                        accumulate ? dval[e] : T(0))
                                  : T(0);
            }
#pragma unroll
            for (int u = 0; u < kDvalU; ++u)
                if (cj[u] >= 0) __stcs(dval + c + 32 * u + lane, d[u]);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
crs_dval_multi_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                const int32_t *__restrict__ col, int m, const T *__restrict__ G, int64_t g_row,
                int64_t g_t, const T *__restrict__ X, int64_t x_row, int64_t x_t, T *__restrict__ dval,
                int accumulate) {
    __shared__ int32_t srp[kDvalWarps][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *rp = srp[wid];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 32; r0 < n_rows; r0 += nwarp * 32) {
        __syncwarp();  // the previous range's row pointers are no longer read
        rp[lane] = __ldg(row_ptr + min(r0 + lane, n_rows));
        if (lane == 0) rp[32] = __ldg(row_ptr + min(r0 + 32, n_rows));
        __syncwarp();
        const int32_t e1 = rp[32];
        int r = 0;  // local row of this lane's current entry
        for (int32_t e = rp[0] + lane; e < e1; e += 32) {
            while (rp[r + 1] <= e) ++r;  // stops at r <= 31, since e < rp[32]
            const int64_t row = r0 + r;
            const int64_t cj = ld_stream(col + e);
            T d = accumulate ? dval[e] : T(0);
            for (int t = 0; t < m; ++t)
                d = fma(__ldg(G + row * g_row + t * g_t), __ldg(X + cj * x_row + t * x_t), d);
            dval[e] = d;
        }
    }
}

__global__ void crs_validate_kernel(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                    const int32_t *__restrict__ row_ptr,
                                    const int32_t *__restrict__ col, int32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (tid == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n_rows] != nnz)) bad = true;
    for (int64_t i = tid; i < n_rows; i += stride)
        if (row_ptr[i + 1] < row_ptr[i]) bad = true;
    for (int64_t k = tid; k < nnz; k += stride) {
        const int32_t c = col[k];
        if (c < 0 || (int64_t)c >= n_cols) bad = true;
    }
    if (bad) *status = (int32_t)GBSP_ERR_MATRIX;
}

// ------------------------------------------------------------------ host --

static int grid_for(int64_t warps_needed) {
    const int64_t blocks = ceil_div(warps_needed, kThreads / 32);
    const int64_t cap = (int64_t)num_sms() * 8 * 4;  // four waves of full occupancy
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

// The row kernels (VECTOR, RUNS, SpMM) run in CTAs of two warps, one CTA per
// two warps' worth of rows: a CTA's slot frees as soon as its two warps are
// done, instead of when the slowest of eight is, so the block scheduler
// keeps the SMs full of warps with work left.  HH-like 6M, CRS vector 4 x 4:
// 289 us against 305 us with 256-thread CTAs on a four-wave grid; Zipf
// rows 515 against 584 us; SpMM k = 16 2489 against 2680 us.
constexpr int kRowCta = 64;
static int row_grid(int64_t warps_needed) {
    return (int)std::max<int64_t>(1, ceil_div(warps_needed, kRowCta / 32));
}

template <int VM, int L>
static void launch_vector_R(const Mat &A, const VecArgs &v, int R, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    const int64_t rw = (32 / L) * R;
    const int grid = (int)limit_grid(row_grid(ceil_div(A.n_rows, rw)), A.grid_limit);
    auto *val = static_cast<const T *>(A.val);
    auto *x = static_cast<const T *>(v.x);
    auto *y = static_cast<T *>(v.y);
    switch (R) {
        case 1:
            crs_vector_kernel<VM, L, 1><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, x,
                                                                  v.ldx, y, v.ldy, v.accumulate);
            break;
        case 2:
            crs_vector_kernel<VM, L, 2><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, x,
                                                                  v.ldx, y, v.ldy, v.accumulate);
            break;
        default:
            crs_vector_kernel<VM, L, 4><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, x,
                                                                  v.ldx, y, v.ldy, v.accumulate);
            break;
    }
}

template <int VM>
static void launch_vector(const Mat &A, const VecArgs &v, cudaStream_t s) {
    const int R = A.kopt.rows_per_warp;
    switch (A.kopt.lanes) {
        case 1: launch_vector_R<VM, 1>(A, v, R, s); break;
        case 2: launch_vector_R<VM, 2>(A, v, R, s); break;
        case 4: launch_vector_R<VM, 4>(A, v, R, s); break;
        case 8: launch_vector_R<VM, 8>(A, v, R, s); break;
        case 16: launch_vector_R<VM, 16>(A, v, R, s); break;
        default: launch_vector_R<VM, 32>(A, v, R, s); break;
    }
}

template <int VM, int L, int R>
static void launch_runs_LR(const Mat &A, const VecArgs &v, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    const int grid = (int)limit_grid(row_grid(ceil_div(A.n_rows, (32 / L) * R)), A.grid_limit);
    crs_runs_kernel<VM, L, R><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, static_cast<const T *>(A.val),
                                                        static_cast<const T *>(v.x), v.ldx,
                                                        static_cast<T *>(v.y), v.ldy, v.accumulate);
}

// (lanes, rows) pairs of RUNS; gbsp_set_kernel admits exactly these.
template <int VM>
static void launch_runs(const Mat &A, const VecArgs &v, cudaStream_t s) {
    const int L = A.kopt.lanes, R = A.kopt.rows_per_warp;
    if (L == 1 && R == 4) launch_runs_LR<VM, 1, 4>(A, v, s);
    else if (L == 1) launch_runs_LR<VM, 1, 8>(A, v, s);
    else if (L == 2 && R == 4) launch_runs_LR<VM, 2, 4>(A, v, s);
    else if (L == 2) launch_runs_LR<VM, 2, 8>(A, v, s);
    else if (L == 4 && R == 4) launch_runs_LR<VM, 4, 4>(A, v, s);
    else if (L == 4) launch_runs_LR<VM, 4, 8>(A, v, s);
    else launch_runs_LR<VM, 8, 8>(A, v, s);
}

template <int VM>
static void launch_spmm(const Mat &A, const VecArgs &v, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    int kt = A.kopt.rhs_tile > 0 ? A.kopt.rhs_tile : 16;
    kt = std::min(kt, 32);
    // lanes per row: the power of two covering min(k, tile)
    int cols = std::min<int>(v.k, kt);
    int KT = 2;
    while (KT < cols) KT <<= 1;
    auto *val = static_cast<const T *>(A.val);
    auto *X = static_cast<const T *>(v.x);
    auto *Y = static_cast<T *>(v.y);
    const int grid = row_grid(ceil_div(A.n_rows, 32 / KT));
    for (int c0 = 0; c0 < v.k; c0 += KT) {
        switch (KT) {
            case 2:
                crs_spmm_kernel<VM, 2><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, X,
                                                                 v.ldx, Y, v.ldy, v.k, c0, v.accumulate);
                break;
            case 4:
                crs_spmm_kernel<VM, 4><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, X,
                                                                 v.ldx, Y, v.ldy, v.k, c0, v.accumulate);
                break;
            case 8:
                crs_spmm_kernel<VM, 8><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, X,
                                                                 v.ldx, Y, v.ldy, v.k, c0, v.accumulate);
                break;
            case 16:
                crs_spmm_kernel<VM, 16><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, X,
                                                                  v.ldx, Y, v.ldy, v.k, c0, v.accumulate);
                break;
            default:
                crs_spmm_kernel<VM, 32><<<grid, kRowCta, 0, s>>>(A.n_rows, A.row_ptr, A.col, val, X,
                                                                  v.ldx, Y, v.ldy, v.k, c0, v.accumulate);
                break;
        }
    }
}

// Default VECTOR shape.  FP64: three to six entries per lane.  On GB300
// every step of a lane group's shuffle reduction is a full FP64 instruction
// and idle lanes issue their FMAs anyway, so few lanes per row win: on the
// HH-like matrix (13 entries a row) 4 lanes ran at 362 us, 8 at 555 us and
// 16 at 1091 us.  FP32 arithmetic is cheap, and the compensated sums are
// long dependent chains, so FP32 rows get about one lane per entry.
void crs_default_opts(Mat &A) {
    const double mean = A.n_rows > 0 ? (double)A.nnz / (double)A.n_rows : 0.0;
    int lanes = 1;
    if (A.dtype == GBSP_F64) {
        while (lanes < 32 && 3.0 * (2 * lanes) <= mean) lanes <<= 1;
    } else {
        while (lanes < 32 && lanes < mean) lanes <<= 1;
        if (lanes > 1 && lanes >= 2 * mean) lanes >>= 1;
    }
    A.kopt.kernel = GBSP_KERNEL_VECTOR;
    A.kopt.lanes = lanes;
    A.kopt.rows_per_warp = lanes >= 16 ? 2 : 4;
    A.kopt.tile = 2048;
    A.kopt.rhs_tile = 16;
    A.kopt.accum = A.dtype == GBSP_F32 ? GBSP_ACC_COMPENSATED : GBSP_ACC_PLAIN;
}

gbsp_status crs_tiled_launch(const Mat &A, const VecArgs &v, cudaStream_t s);

gbsp_status crs_launch(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (A.n_rows == 0) return GBSP_OK;
    const int vm = A.dtype == GBSP_F64 ? VM_F64
                   : (A.kopt.accum == GBSP_ACC_COMPENSATED ? VM_F32C : VM_F32);
    if (v.k == 1 && A.kopt.kernel == GBSP_KERNEL_TILED && A.tile_rows != nullptr)
        return crs_tiled_launch(A, v, s);
    if (v.k == 1 && A.kopt.kernel == GBSP_KERNEL_RUNS) {
        if (vm == VM_F64) launch_runs<VM_F64>(A, v, s);
        else if (vm == VM_F32) launch_runs<VM_F32>(A, v, s);
        else launch_runs<VM_F32C>(A, v, s);
    } else if (v.k == 1) {
        if (vm == VM_F64) launch_vector<VM_F64>(A, v, s);
        else if (vm == VM_F32) launch_vector<VM_F32>(A, v, s);
        else launch_vector<VM_F32C>(A, v, s);
    } else {
        if (vm == VM_F64) launch_spmm<VM_F64>(A, v, s);
        else if (vm == VM_F32) launch_spmm<VM_F32>(A, v, s);
        else launch_spmm<VM_F32C>(A, v, s);
    }
    GBSP_LAUNCH_CHECK("crs product kernel");
    return GBSP_OK;
}

gbsp_status crs_validate_launch(const Mat &A, int32_t *d_status, cudaStream_t s) {
    GBSP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s));
    const int64_t work = std::max(A.n_rows, A.nnz);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, kThreads),
                                                                 (int64_t)num_sms() * 8));
    crs_validate_kernel<<<grid, kThreads, 0, s>>>(A.n_rows, A.n_cols, A.nnz, A.row_ptr, A.col,
                                                  d_status);
    GBSP_LAUNCH_CHECK("crs_validate_kernel");
    return GBSP_OK;
}

template <typename T>
static void launch_dval(const Mat &A, int32_t m, const void *G, int64_t g_row, int64_t g_t,
                        const void *X, int64_t x_row, int64_t x_t, void *dval, int32_t accumulate,
                        cudaStream_t s) {
    const int grid = grid_for(ceil_div(A.n_rows, 32));
    if (m == 1)
        crs_dval_kernel<T><<<grid, kThreads, 0, s>>>(A.n_rows, A.row_ptr, A.col, m, static_cast<const T *>(G), g_row,
                                                     g_t, static_cast<const T *>(X), x_row, x_t,
                                                     static_cast<T *>(dval), accumulate);
    else
        crs_dval_multi_kernel<T><<<grid, kThreads, 0, s>>>(A.n_rows, A.row_ptr, A.col, m, static_cast<const T *>(G),
                                                           g_row, g_t, static_cast<const T *>(X), x_row, x_t,
                                                           static_cast<T *>(dval), accumulate);
}

gbsp_status crs_dval_launch(const Mat &A, int32_t m, const void *G, int64_t g_row, int64_t g_t,
                            const void *X, int64_t x_row, int64_t x_t, void *dval, int32_t accumulate,
                            cudaStream_t s) {
    if (A.n_rows == 0 || A.nnz == 0) return GBSP_OK;
    if (A.dtype == GBSP_F64) launch_dval<double>(A, m, G, g_row, g_t, X, x_row, x_t, dval, accumulate, s);
    else launch_dval<float>(A, m, G, g_row, g_t, X, x_row, x_t, dval, accumulate, s);
    GBSP_LAUNCH_CHECK("crs_dval_kernel");
    return GBSP_OK;
}

}  // namespace gbsp
