// JDS-family products (Sect. 2, JDS kernel and its refinements).
//
// Storage: jagged diagonal d holds permuted rows 0 .. diagLen(d)-1 at
// positions jd_ptr[d] + r, so a warp of consecutive rows reads each diagonal
// as one contiguous segment.  Every kernel below gives each thread whole
// rows and adds a row's entries in slot order d = 0, 1, ... with an FMA
// chain starting from zero, so all JDS-family kernels return bit-identical
// results for the same storage pattern.
//
//   JDS_LITERAL  one launch per jagged diagonal; resvec makes a round trip
//                through memory per diagonal, as the paper's loop does.
//   JDS          one thread per row walks the diagonals; resvec stays in a
//                register (written once).
//   NUJDS        the same walk, u diagonals per step: the u loads of a step
//                are issued together (outer-loop unrolling, Sect. 2).
//   NBJDS        a CTA owns a block of `block` rows and walks only the
//                diagonals that have entries in it, each thread holding R
//                rows' sums in registers (blocking, Sect. 2).
//   RBJDS/SOJDS  like NBJDS, but the block's entries are stored
//                consecutively (diagonal-major inside the block), so a CTA
//                streams one contiguous chunk.
#include <algorithm>
#include <atomic>
#include <climits>
#include <vector>

#include "accum.cuh"
#include "internal.cuh"

namespace gbsp {

struct JdsArgs {
    int64_t n_rows, n_diag;
    const int32_t *jd_ptr, *col, *blk_ptr;
    const void *val;
    const void *x;
    void *y;
    int64_t ldx, ldy;
    int32_t k, c0;
    int32_t accumulate;
    int32_t block;
    const int32_t *x_perm;  // x index = x_perm[col] (ORIGINAL basis, symmetric storage)
    const int32_t *y_perm;  // y row = y_perm[r]      (ORIGINAL basis)
    const int32_t *rlen;    // SELL: permuted row lengths
    // deep-diagonal split (JDS / NUJDS): the walk stops at d_limit and adds
    // the chunk partial sums of rows that go deeper
    int64_t d_limit;
    int32_t split_k;
    const int4 *split_table;
    const int32_t *split_items;
    const void *split_part;
    void *split_shallow;   // walk sums of the rows that go deeper than d_limit
    int64_t split_rows;    // those rows: [0, split_rows)
    int64_t n_cols;
    int32_t grid_limit;    // 0 = none
    int32_t y_evict_first; // y too large to stay in L2 until its next use: write it evict-first
};

__device__ __forceinline__ int64_t xidx(const int32_t *x_perm, int32_t c) {
    return x_perm ? (int64_t)__ldg(x_perm + c) : (int64_t)c;
}

template <int VM>
__device__ __forceinline__ void store_row(const JdsArgs &a, int64_t r, int c, Acc<VM> &acc) {
    typedef typename ValT<VM>::T T;
    const int64_t row = a.y_perm ? (int64_t)__ldg(a.y_perm + r) : r;
    T *yp = static_cast<T *>(a.y) + row * a.ldy + c;
    if (a.accumulate) acc.add_value(*yp);
    *yp = acc.result();
}

// store_row for the SELL walks.  A y larger than a quarter of L2 is written
// evict-first: it cannot survive the next product's matrix stream anyway,
// and keeping it out of L2 leaves room for the gathered x (SELL step,
// HH-like 6M: about 1%).  A smaller y stays cached for the next product
// that reads it, as in a power iteration.  (The SELL kernels have a fixed
// register budget; in the JDS row walk the extra branch cost 6 registers
// and a quarter of its occupancy, so the other walks store plainly.)
template <int VM>
__device__ __forceinline__ void store_row_sell(const JdsArgs &a, int64_t r, int c, Acc<VM> &acc) {
    typedef typename ValT<VM>::T T;
    const int64_t row = a.y_perm ? (int64_t)__ldg(a.y_perm + r) : r;
    T *yp = static_cast<T *>(a.y) + row * a.ldy + c;
    if (a.accumulate) acc.add_value(*yp);
    if (a.y_evict_first) __stcs(yp, acc.result());
    else *yp = acc.result();
}

// JDS (U = 1) and NUJDS (U > 1): one thread per permuted row, U diagonals
// per step.  With R > 1 a warp owns 32*R consecutive rows and each thread R
// of them (rows base + 32 i + lane): the loads of all R rows and U diagonals
// are issued together, while each warp-wide load still covers 32
// consecutive entries of one diagonal.
// PLAIN: one vector read directly (no x permutation, unit stride).
template <int VM, int U, int R, bool PLAIN>
__global__ void __launch_bounds__(256) jds_row_kernel(JdsArgs a) {
    typedef typename ValT<VM>::T T;
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 32 * R; base < a.n_rows; base += nwarp * 32 * R) {
        int64_t rr[R];
#pragma unroll
        for (int i = 0; i < R; ++i) rr[i] = base + 32 * i + lane;
        if (rr[0] >= a.n_rows) continue;
        Acc<VM> acc[R];
#pragma unroll
        for (int i = 0; i < R; ++i) acc[i].init();
        // offsets of step 0 and its loads; each step then fetches the next
        // step's offsets before forming its own products, so the small
        // jd_ptr loads overlap the gathers instead of preceding them
        int32_t e[U + 1];
        e[0] = __ldg(a.jd_ptr);
#pragma unroll
        for (int j = 0; j < U; ++j) e[j + 1] = (j < a.d_limit) ? __ldg(a.jd_ptr + j + 1) : e[j];
        int c[R][U];
        T v[R][U];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = e[j + 1] - e[j] > rr[i];
                c[i][j] = ok ? ld_stream(a.col + e[j] + rr[i]) : -1;
                v[i][j] = ok ? ld_stream(val + e[j] + rr[i]) : T(0);
            }
        const int64_t dlim = a.d_limit;
        for (int64_t d0 = 0; d0 < dlim; d0 += U) {
            int32_t en[U + 1];
            en[0] = e[U];
#pragma unroll
            for (int j = 0; j < U; ++j)
                en[j + 1] = (d0 + U + j < dlim) ? __ldg(a.jd_ptr + d0 + U + j + 1) : en[j];
            // rr[0] is the thread's longest row (rows are sorted by length)
            const bool more = d0 + U < dlim && en[1] - en[0] > rr[0];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if (c[i][j] >= 0)
                        acc[i].add(v[i][j], ld_vec(PLAIN ? x + c[i][j] : x + xidx(a.x_perm, c[i][j]) * a.ldx));
            if (!more) break;
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const bool ok = en[j + 1] - en[j] > rr[i];
                    c[i][j] = ok ? ld_stream(a.col + en[j] + rr[i]) : -1;
                    v[i][j] = ok ? ld_stream(val + en[j] + rr[i]) : T(0);
                }
#pragma unroll
            for (int j = 0; j <= U; ++j) e[j] = en[j];
        }
        // rows that go deeper than the split depth: their walk sum waits in
        // the workspace for the merge with the chunk partial sums
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (rr[i] >= a.n_rows) continue;
            if (rr[i] < a.split_rows) static_cast<Acc<VM> *>(a.split_shallow)[rr[i]] = acc[i];
            else store_row<VM>(a, rr[i], 0, acc[i]);
        }
    }
}

// Deep part of a split JDS walk: CTA items are (chunk k, 256 rows); thread
// row r sums its entries in diagonals [d_begin, d_end) of chunk k, in slot
// order, into part[offset_k + r].
template <int VM>
__global__ void __launch_bounds__(256) jds_deep_kernel(JdsArgs a, int64_t n_items) {
    typedef typename ValT<VM>::T T;
    constexpr int W = 256;  // diagonals of jd_ptr staged in shared memory at a time
    constexpr int G = 8;    // diagonals whose loads are issued together
    __shared__ int32_t sj[W + 1];
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    Acc<VM> *part = static_cast<Acc<VM> *>(const_cast<void *>(a.split_part));
    // a CTA works on one item at a time, so its threads share the chunk and
    // its diagonal offsets; its items come in increasing order, so the chunk
    // index only moves forward
    int32_t k = 0;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        while (k + 1 < a.split_k && __ldg(a.split_items + k + 1) <= it) ++k;
        const int4 t = __ldg(a.split_table + k);
        const int64_t r = (it - __ldg(a.split_items + k)) * 256 + threadIdx.x;
        const bool live = r < t.z;
        Acc<VM> acc;
        acc.init();
        bool done = !live;
        for (int32_t w0 = t.x; w0 < t.y; w0 += W) {
            const int32_t wn = min(W, t.y - w0);
            __syncthreads();
            for (int i = threadIdx.x; i <= wn; i += blockDim.x) sj[i] = __ldg(a.jd_ptr + w0 + i);
            __syncthreads();
            if (done) continue;
            for (int32_t d = 0; d < wn; d += G) {
                int c[G];
                T v[G];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    // diagonal lengths fall with d: once row r is past one, it is past the rest
                    const bool ok = d + j < wn && sj[d + j + 1] - sj[d + j] > r;
                    c[j] = ok ? ld_stream(a.col + sj[d + j] + r) : -1;
                    v[j] = ok ? ld_stream(val + sj[d + j] + r) : T(0);
                }
#pragma unroll
                for (int j = 0; j < G; ++j)
                    if (c[j] >= 0) acc.add(v[j], ld_vec(x + xidx(a.x_perm, c[j]) * a.ldx));
                if (c[G - 1] < 0) {
                    done = true;
                    break;
                }
            }
        }
        if (live) part[(int64_t)t.w + r] = acc;
    }
}

// Last step of a split walk: row r (a row deeper than the split depth)
// takes its walk sum and adds its chunk partial sums.  Rows with more than
// 8 chunks ([0, wide_rows)) get a warp: lane l sums chunks l, l+32, ... in
// order and a fixed shuffle tree combines the lanes.  The others get a
// thread that adds its (at most 8) chunks in chunk order, loads issued
// together.
template <int VM>
__global__ void __launch_bounds__(256) jds_split_merge_kernel(JdsArgs a, int64_t wide_rows) {
    const Acc<VM> *part = static_cast<const Acc<VM> *>(a.split_part);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < wide_rows; r += nwarps) {
        Acc<VM> s;
        s.init();
        for (int32_t k0 = lane; k0 < a.split_k; k0 += 32 * 4) {
            Acc<VM> p[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int32_t k = k0 + 32 * j;
                const int4 t = k < a.split_k ? __ldg(a.split_table + k) : make_int4(0, 0, 0, 0);
                ok[j] = k < a.split_k && r < t.z;
                if (ok[j]) p[j] = part[(int64_t)t.w + r];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j]) s.merge(p[j]);
            if (!ok[3]) break;
        }
        group_reduce<32>(s);
        if (lane == 0) {
            Acc<VM> acc = static_cast<const Acc<VM> *>(a.split_shallow)[r];
            acc.merge(s);
            store_row<VM>(a, r, 0, acc);
        }
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = wide_rows + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.split_rows; r += stride) {
        Acc<VM> acc = static_cast<const Acc<VM> *>(a.split_shallow)[r];
        for (int32_t k0 = 0; k0 < a.split_k; k0 += 8) {
            Acc<VM> p[8];
            bool ok[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int4 t = k0 + j < a.split_k ? __ldg(a.split_table + k0 + j) : make_int4(0, 0, 0, 0);
                ok[j] = k0 + j < a.split_k && r < t.z;  // rows of chunk k are [0, t.z)
                if (ok[j]) p[j] = part[(int64_t)t.w + r];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (ok[j]) acc.merge(p[j]);
            if (!ok[7]) break;
        }
        store_row<VM>(a, r, 0, acc);
    }
}

// NBJDS (CONTIG = false) and RBJDS / SOJDS (CONTIG = true): a CTA per row
// block, R rows per thread in flight; KT > 1 gives KT right-hand sides per
// thread (SpMM, then R = 1).
template <int VM, bool CONTIG, int R, int KT>
__global__ void __launch_bounds__(256) jds_block_kernel(JdsArgs a) {
    typedef typename ValT<VM>::T T;
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    const int64_t n_blocks = ceil_div_dev(a.n_rows, a.block);
    for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
        const int64_t b0 = blk * a.block;
        const int64_t b1 = min(b0 + (int64_t)a.block, a.n_rows);
        const int64_t cbase = CONTIG ? (int64_t)__ldg(a.blk_ptr + blk) : 0;
        for (int64_t c0 = b0; c0 < b1; c0 += (int64_t)blockDim.x * R) {
            int64_t rr[R];
#pragma unroll
            for (int i = 0; i < R; ++i) rr[i] = c0 + threadIdx.x + (int64_t)i * blockDim.x;
            Acc<VM> acc[R][KT];
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int q = 0; q < KT; ++q) acc[i][q].init();
            int32_t st = __ldg(a.jd_ptr);
            int64_t off = cbase;
            for (int64_t d = 0; d < a.n_diag; ++d) {
                const int32_t en = __ldg(a.jd_ptr + d + 1);
                const int64_t dl = en - st;
                if (dl <= b0) break;  // no entries of this block in diagonal d
                int c[R];
                T v[R];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const bool ok = rr[i] < b1 && rr[i] < dl;
                    const int64_t kk = CONTIG ? off + (rr[i] - b0) : (int64_t)st + rr[i];
                    c[i] = ok ? ld_stream(a.col + kk) : -1;
                    v[i] = ok ? ld_stream(val + kk) : T(0);
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    if (c[i] < 0) continue;
                    const T *xr = x + xidx(a.x_perm, c[i]) * a.ldx + a.c0;
#pragma unroll
                    for (int q = 0; q < KT; ++q)
                        if (KT == 1 || a.c0 + q < a.k) acc[i][q].add(v[i], ld_vec(xr + q));
                }
                if (CONTIG) off += min(b1, dl) - b0;
                st = en;
            }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (rr[i] >= b1) continue;
#pragma unroll
                for (int q = 0; q < KT; ++q)
                    if (KT == 1 || a.c0 + q < a.k) store_row<VM>(a, rr[i], a.c0 + q, acc[i][q]);
            }
        }
    }
}

// SELL-32-sigma: one warp per block of 32 permuted rows, lane = row.  Slot
// d of the block holds the rows with length > d, which are its first
// popc(ballot(len > d)) rows, so lane l's entry of slot d sits at
// (start of slot d) + l: every warp-wide load is one contiguous segment.
// A CTA's warps take consecutive blocks, so a 1024-thread CTA works on one
// 1024-row window at a time and its gathers of x stay local.  U slots per
// step; KT right-hand sides per thread (SpMM).  Row entries are added in
// slot order, as in every JDS-family kernel.
template <int VM, int U, int KT, bool PLAIN>
__device__ __forceinline__ void sell_walk(const JdsArgs &a) {
    typedef typename ValT<VM>::T T;
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t nb = ceil_div_dev(a.n_rows, 32);
    const int wpc = blockDim.x >> 5;  // warps per CTA
    const int wid = threadIdx.x >> 5;
    const int64_t ngroups = ceil_div_dev(nb, wpc);
    // A CTA takes wpc consecutive blocks (a group) per iteration.  Blocks are
    // sorted by length inside their window, so the warp's pick among them
    // rotates by 7 from one iteration to the next: otherwise warp 0 would
    // always get the longest rows and warp wpc-1 the shortest.
    // The group a CTA takes also rotates (by one per iteration): with a
    // window longer than a group, a fixed stride of gridDim.x groups would
    // hand every CTA the same position in every window.  Both rotations are
    // kept as running 32-bit counters (no division in the loop).
    uint32_t rot = blockIdx.x;  // (blockIdx.x + iteration) mod gridDim.x
    int pick = wid;             // (wid + 7 iteration) mod wpc
    for (int64_t g0 = 0; g0 < ngroups; g0 += gridDim.x) {
        const int64_t g = g0 + rot;
        const int64_t b = g * wpc + pick;
        rot = rot + 1 == gridDim.x ? 0u : rot + 1;
        pick += 7;
        while (pick >= wpc) pick -= wpc;
        if (g >= ngroups || b >= nb) continue;
        const int64_t r = b * 32 + lane;
        // row lengths are read once: streamed like val / col (evict-first)
        const int32_t len = r < a.n_rows ? ld_stream(a.rlen + r) : 0;
        const int32_t width = __shfl_sync(0xffffffffu, len, 0);  // lane 0 holds the longest row
        // entry offsets fit int32 (nnz < 2^31)
        int32_t off = __ldg(a.blk_ptr + b);
        Acc<VM> acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q].init();
        // step 0 loads; each step then issues the next step's loads after
        // forming its own products
        int c[U];
        T v[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const bool ok = len > j;
            c[j] = ok ? ld_stream(a.col + (off + lane)) : -1;
            v[j] = ok ? ld_stream(val + (off + lane)) : T(0);
            off += __popc(__ballot_sync(0xffffffffu, ok));
        }
        for (int32_t d0 = 0; d0 < width; d0 += U) {
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (c[j] < 0) continue;
                if (PLAIN) {
                    acc[0].add(v[j], ld_vec(x + c[j]));
                } else {
                    const T *xr = x + xidx(a.x_perm, c[j]) * a.ldx + a.c0;
#pragma unroll
                    for (int q = 0; q < KT; ++q)
                        if (KT == 1 || a.c0 + q < a.k) acc[q].add(v[j], ld_vec(xr + q));
                }
            }
            if (d0 + U >= width) break;
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = len > d0 + U + j;
                c[j] = ok ? ld_stream(a.col + (off + lane)) : -1;
                v[j] = ok ? ld_stream(val + (off + lane)) : T(0);
                off += __popc(__ballot_sync(0xffffffffu, ok));
            }
        }
        if (r < a.n_rows) {
#pragma unroll
            for (int q = 0; q < KT; ++q)
                if (KT == 1 || a.c0 + q < a.k) store_row_sell<VM>(a, r, a.c0 + q, acc[q]);
        }
    }
}


template <int VM, int U, int KT, bool PLAIN>
__global__ void __launch_bounds__(1024) sell_kernel(JdsArgs a) {
    sell_walk<VM, U, KT, PLAIN>(a);
}

// The plain one-vector FP64 walk compiled for two CTAs per SM: at the same
// 32 registers this schedules it 1.4% faster than the unhinted kernel.  The
// other instances keep the kernel above: under the hint the SpMM ones would
// spill and the FP32 ones ran 3% slower, and a hint of one CTA per SM gives
// them 48 registers.
template <int U>
__global__ void __launch_bounds__(1024, 2) sell_kernel_f64(JdsArgs a) {
    sell_walk<VM_F64, U, 1, true>(a);
}

// SELL with the banded part of x staged in shared memory.  A CTA of 32 warps
// takes a group of 32 consecutive blocks (1024 rows) at a time, as the SELL
// kernel does; before walking them it copies the group's chosen x pages
// (1024 entries each, the pages its rows reference most) into shared memory
// with coalesced loads.  A staged entry's column is stored as
// ~(slot * 1024 + col % 1024) and read from shared memory; the rest are
// gathered from global memory as before.  The arithmetic is the SELL
// kernel's, entry for entry, so the results are bit-identical; only where
// each x value is read from changes.  Two CTAs per SM, so one stages while
// the other walks.
constexpr int kStagePage = 1024;
constexpr int kMaxDevices = 64;

template <int VM, int U>
__global__ void __launch_bounds__(1024, 2) sell_staged_kernel(JdsArgs a, const int32_t *__restrict__ col_st,
                                                               const int32_t *__restrict__ pages, int P) {
    typedef typename ValT<VM>::T T;
    extern __shared__ __align__(16) unsigned char stage_smem[];
    T *xs = reinterpret_cast<T *>(stage_smem);
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    const int lane = threadIdx.x & 31;
    const int64_t nb = ceil_div_dev(a.n_rows, 32);
    const int wpc = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5;
    const int64_t ngroups = ceil_div_dev(nb, wpc);
    // the SELL walk's rotations, as running 32-bit counters
    uint32_t rot = blockIdx.x;
    int pick = wid;
    for (int64_t g0 = 0; g0 < ngroups; g0 += gridDim.x) {
        const int64_t g = g0 + rot;
        const int64_t b = g * wpc + pick;
        rot = rot + 1 == gridDim.x ? 0u : rot + 1;
        pick += 7;
        while (pick >= wpc) pick -= wpc;
        __syncthreads();  // the previous group's staged x is no longer read
        if (g < ngroups) {
            for (int q = threadIdx.x; q < P * kStagePage; q += blockDim.x) {
                const int32_t pg = __ldg(pages + g * P + q / kStagePage);
                const int64_t idx = (int64_t)pg * kStagePage + (q % kStagePage);
                xs[q] = (pg >= 0 && idx < a.n_cols) ? ld_vec(x + idx) : T(0);
            }
        }
        __syncthreads();
        if (g >= ngroups || b >= nb) continue;
        const int64_t r = b * 32 + lane;
        const int32_t len = r < a.n_rows ? ld_stream(a.rlen + r) : 0;
        const int32_t width = __shfl_sync(0xffffffffu, len, 0);
        int64_t off = __ldg(a.blk_ptr + b);
        Acc<VM> acc;
        acc.init();
        constexpr int NONE = INT_MIN;
        int c[U];
        T v[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const bool ok = len > j;
            c[j] = ok ? ld_stream(col_st + off + lane) : NONE;
            v[j] = ok ? ld_stream(val + off + lane) : T(0);
            off += __popc(__ballot_sync(0xffffffffu, len > j));
        }
        for (int32_t d0 = 0; d0 < width; d0 += U) {
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (c[j] == NONE) continue;
                acc.add(v[j], c[j] >= 0 ? ld_vec(x + c[j]) : xs[~c[j]]);
            }
            if (d0 + U >= width) break;
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = len > d0 + U + j;
                c[j] = ok ? ld_stream(col_st + off + lane) : NONE;
                v[j] = ok ? ld_stream(val + off + lane) : T(0);
                off += __popc(__ballot_sync(0xffffffffu, len > d0 + U + j));
            }
        }
        if (r < a.n_rows) store_row<VM>(a, r, 0, acc);
    }
}

// Paired SELL: one warp per block of 64 permuted rows, lane p walks row
// 64g+p and then, if present, row 64g+L+p (the short partner of its window,
// L = lanes of the block).  Slot t holds the lanes whose two rows have more
// than t entries, so lane p's entry sits at (start of slot t) + (active
// lanes below p).  When a lane reaches the end of its first row it sets that
// row's sum aside and restarts; both rows are stored at the end.  Entries of
// every row are added in order.
template <int VM, int U, int KT, bool PLAIN>
__global__ void __launch_bounds__(1024, (KT == 1 ? 2 : 1)) psell_kernel(JdsArgs a) {
    typedef typename ValT<VM>::T T;
    const T *__restrict__ val = static_cast<const T *>(a.val);
    const T *__restrict__ x = static_cast<const T *>(a.x);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nb = ceil_div_dev(a.n_rows, 64);
    const int wpc = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5;
    // same rotation of blocks over warps and groups over CTAs as SELL
    const int64_t ngroups = ceil_div_dev(nb, wpc);
    uint32_t rot = blockIdx.x;
    int pick = wid;
    for (int64_t g0 = 0; g0 < ngroups; g0 += gridDim.x) {
        const int64_t g = g0 + rot;
        const int64_t b = g * wpc + pick;
        rot = rot + 1 == gridDim.x ? 0u : rot + 1;
        pick += 7;
        while (pick >= wpc) pick -= wpc;
        if (g >= ngroups || b >= nb) continue;
        const int R = (int)min((int64_t)64, a.n_rows - 64 * b), L = (R + 1) / 2;
        const bool lane_ok = lane < L, has_b = lane_ok && L + lane < R;
        const int32_t la = lane_ok ? ld_stream(a.rlen + 64 * b + lane) : 0;
        const int32_t lb = has_b ? ld_stream(a.rlen + 64 * b + L + lane) : 0;
        const int32_t total = la + lb;
        const int32_t width = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)total);
        int32_t off = __ldg(a.blk_ptr + b);  // entries fit int32 (CRS row_ptr is int32)
        Acc<VM> acc[KT], first[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            acc[q].init();
            first[q].init();
        }
        int c[U];
        T v[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const bool ok = total > j;
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            const int32_t pos = off + __popc(m & lt);
            c[j] = ok ? ld_stream(a.col + pos) : -1;
            v[j] = ok ? ld_stream(val + pos) : T(0);
            off += __popc(m);
        }
        for (int32_t d0 = 0; d0 < width; d0 += U) {
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (c[j] < 0) continue;
                if (d0 + j == la) {  // first row done: set it aside, start the second
#pragma unroll
                    for (int q = 0; q < KT; ++q) {
                        first[q] = acc[q];
                        acc[q].init();
                    }
                }
                if (PLAIN) {
                    acc[0].add(v[j], ld_vec(x + c[j]));
                } else {
                    const T *xr = x + xidx(a.x_perm, c[j]) * a.ldx + a.c0;
#pragma unroll
                    for (int q = 0; q < KT; ++q)
                        if (KT == 1 || a.c0 + q < a.k) acc[q].add(v[j], ld_vec(xr + q));
                }
            }
            if (d0 + U >= width) break;
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = total > d0 + U + j;
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                const int32_t pos = off + __popc(m & lt);
                c[j] = ok ? ld_stream(a.col + pos) : -1;
                v[j] = ok ? ld_stream(val + pos) : T(0);
                off += __popc(m);
            }
        }
        if (lane_ok) {
            // lb > 0: `first` holds row a and `acc` row b; else `acc` holds
            // row a and row b (if any) is empty, its sum the zero in `first`
            const int64_t ra = 64 * b + lane, rb = 64 * b + L + lane;
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                if (KT > 1 && a.c0 + q >= a.k) continue;
                store_row<VM>(a, ra, a.c0 + q, lb > 0 ? first[q] : acc[q]);
                if (has_b) store_row<VM>(a, rb, a.c0 + q, lb > 0 ? acc[q] : first[q]);
            }
        }
    }
}

// JDS_LITERAL: the paper's loop, one launch per diagonal d:
//   resvec(i) = resvec(i) + val(off+i) * invec(col_idx(off+i)), i < diagLen(d).
template <typename T>
__global__ void jds_literal_kernel(int64_t len, int32_t off, const int32_t *__restrict__ col,
                                   const T *__restrict__ val, const T *__restrict__ x, int64_t ldx,
                                   T *__restrict__ y, int64_t ldy, const int32_t *x_perm,
                                   const int32_t *y_perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int64_t row = y_perm ? (int64_t)__ldg(y_perm + i) : i;
    T *yp = y + row * ldy;
    *yp = fma(ld_stream(val + off + i), ld_vec(x + xidx(x_perm, ld_stream(col + off + i)) * ldx), *yp);
}

template <typename T>
__global__ void zero_rows_kernel(int64_t n, T *y, int64_t ldy, int k) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * k) return;
    y[(i / k) * ldy + (i % k)] = T(0);
}

// Basis change: dir 0 out[r] = in[perm[r]], dir 1 out[perm[r]] = in[r].
template <typename T>
__global__ void permute_kernel(int64_t n, int k, const int32_t *__restrict__ perm, int dir,
                               const T *__restrict__ in, int64_t ld_in, T *__restrict__ out,
                               int64_t ld_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * k) return;
    const int64_t r = i / k, c = i % k;
    const int64_t p = __ldg(perm + r);
    if (dir == 0) out[r * ld_out + c] = in[p * ld_in + c];
    else out[p * ld_out + c] = in[r * ld_in + c];
}

// ------------------------------------------------------------------ host --

// Thread-per-row kernels: a grid of 64 CTAs per SM, each thread taking
// about two rows (measured best on GB300 for the HH-like workload).
static int row_grid(int64_t rows) {
    const int64_t blocks = ceil_div(rows, 256);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 64));
}

template <int VM, int U>
static void launch_row(const JdsArgs &a, int R, cudaStream_t s) {
    const unsigned g4 = (unsigned)limit_grid(row_grid(ceil_div(a.n_rows, 4)), a.grid_limit);
    const unsigned g2 = (unsigned)limit_grid(row_grid(ceil_div(a.n_rows, 2)), a.grid_limit);
    const unsigned g1 = (unsigned)limit_grid(row_grid(a.n_rows), a.grid_limit);
    if (!a.x_perm && a.ldx == 1) {
        if (R >= 4) jds_row_kernel<VM, U, 4, true><<<g4, 256, 0, s>>>(a);
        else if (R >= 2) jds_row_kernel<VM, U, 2, true><<<g2, 256, 0, s>>>(a);
        else jds_row_kernel<VM, U, 1, true><<<g1, 256, 0, s>>>(a);
    } else {
        if (R >= 4) jds_row_kernel<VM, U, 4, false><<<g4, 256, 0, s>>>(a);
        else if (R >= 2) jds_row_kernel<VM, U, 2, false><<<g2, 256, 0, s>>>(a);
        else jds_row_kernel<VM, U, 1, false><<<g1, 256, 0, s>>>(a);
    }
}

template <int VM, bool CONTIG>
static void launch_block(const JdsArgs &a, int KT, cudaStream_t s) {
    const int64_t nb = ceil_div(a.n_rows, a.block);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)num_sms() * 8 * 16));
    // CTA width: the block size rounded up to a warp, at most 256 threads
    const int threads = (int)std::min<int64_t>(256, std::max<int64_t>(32, ceil_div(a.block, 32) * 32));
    if (KT > 1) {
        switch (KT) {
            case 2: jds_block_kernel<VM, CONTIG, 1, 2><<<grid, threads, 0, s>>>(a); break;
            case 4: jds_block_kernel<VM, CONTIG, 1, 4><<<grid, threads, 0, s>>>(a); break;
            case 8: jds_block_kernel<VM, CONTIG, 1, 8><<<grid, threads, 0, s>>>(a); break;
            default: jds_block_kernel<VM, CONTIG, 1, 16><<<grid, threads, 0, s>>>(a); break;
        }
        return;
    }
    const int64_t R = std::min<int64_t>(8, ceil_div(a.block, threads));
    if (R <= 1) jds_block_kernel<VM, CONTIG, 1, 1><<<grid, threads, 0, s>>>(a);
    else if (R <= 2) jds_block_kernel<VM, CONTIG, 2, 1><<<grid, threads, 0, s>>>(a);
    else if (R <= 4) jds_block_kernel<VM, CONTIG, 4, 1><<<grid, threads, 0, s>>>(a);
    else jds_block_kernel<VM, CONTIG, 8, 1><<<grid, threads, 0, s>>>(a);
}

template <int VM, int U>
static void launch_sell_U(JdsArgs a, int KT, cudaStream_t s) {
    const int64_t nb = ceil_div(a.n_rows, 32);
    const int threads = 1024;
    const int64_t grid = limit_grid(
        std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb * 32, threads), (int64_t)num_sms() * 2)), a.grid_limit);
    // one vector, read directly (no x permutation, unit stride): the plain
    // walk, without the SpMM index arithmetic
    const bool plain = KT == 1 && !a.x_perm && a.ldx == 1 && a.c0 == 0;
    switch (KT) {
        case 1:
            if (plain && VM == VM_F64) sell_kernel_f64<U><<<(unsigned)grid, threads, 0, s>>>(a);
            else if (plain) sell_kernel<VM, U, 1, true><<<(unsigned)grid, threads, 0, s>>>(a);
            else sell_kernel<VM, U, 1, false><<<(unsigned)grid, threads, 0, s>>>(a);
            break;
        case 2: sell_kernel<VM, U, 2, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        case 4: sell_kernel<VM, U, 4, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        case 8: sell_kernel<VM, U, 8, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        default: sell_kernel<VM, U, 16, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
    }
}

template <int VM, int U>
static void launch_psell_U(JdsArgs a, int KT, cudaStream_t s) {
    const int64_t nb = ceil_div(a.n_rows, 64);
    const int threads = 1024;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb * 32, threads), (int64_t)num_sms() * 2));
    const bool plain = KT == 1 && !a.x_perm && a.ldx == 1 && a.c0 == 0;
    switch (KT) {
        case 1:
            if (plain) psell_kernel<VM, U, 1, true><<<(unsigned)grid, threads, 0, s>>>(a);
            else psell_kernel<VM, U, 1, false><<<(unsigned)grid, threads, 0, s>>>(a);
            break;
        case 2: psell_kernel<VM, U, 2, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        case 4: psell_kernel<VM, U, 4, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        case 8: psell_kernel<VM, U, 8, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
        default: psell_kernel<VM, U, 16, false><<<(unsigned)grid, threads, 0, s>>>(a); break;
    }
}

template <int VM>
static void launch_psell(const Mat &A, JdsArgs a, cudaStream_t s) {
    int KT = 1;
    if (a.k > 1) {
        const int tile = A.kopt.rhs_tile > 0 ? std::min(A.kopt.rhs_tile, 16) : 16;
        const int cols = std::min(a.k, tile);
        KT = 2;
        while (KT < cols) KT <<= 1;
    }
    for (int c0 = 0; c0 < a.k; c0 += KT) {
        a.c0 = c0;
        if (KT > 1 || A.unroll <= 1) launch_psell_U<VM, 1>(a, KT, s);
        else if (A.unroll <= 2) launch_psell_U<VM, 2>(a, KT, s);
        else launch_psell_U<VM, 4>(a, KT, s);
    }
}

template <int VM, int U>
static gbsp_status launch_sell_staged_U(const Mat &A, JdsArgs a, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    const int P = A.stage_pages_per_group;
    const int smem = P * kStagePage * (int)sizeof(T);
    // largest dynamic shared memory set so far for this kernel, per device
    static std::atomic<int> configured[kMaxDevices];
    int dev = 0;
    GBSP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices || smem > configured[dev].load()) {
        GBSP_CUDA(cudaFuncSetAttribute(sell_staged_kernel<VM, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GBSP_CUDA(cudaFuncSetAttribute(sell_staged_kernel<VM, U>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       100));
        if (dev >= 0 && dev < kMaxDevices) {
            int cur = configured[dev].load();
            while (cur < smem && !configured[dev].compare_exchange_weak(cur, smem)) {
            }
        }
    }
    const int64_t ngroups = ceil_div(ceil_div(a.n_rows, 32), 32);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ngroups, (int64_t)num_sms() * 2));
    sell_staged_kernel<VM, U><<<(unsigned)grid, 1024, smem, s>>>(a, A.stage_col, A.stage_pages, P);
    return GBSP_OK;
}

template <int VM>
static void launch_sell(const Mat &A, JdsArgs a, cudaStream_t s) {
    int KT = 1;
    if (a.k > 1) {
        const int tile = A.kopt.rhs_tile > 0 ? std::min(A.kopt.rhs_tile, 16) : 16;
        const int cols = std::min(a.k, tile);
        KT = 2;
        while (KT < cols) KT <<= 1;
    }
    for (int c0 = 0; c0 < a.k; c0 += KT) {
        a.c0 = c0;
        if (KT > 1 || A.unroll <= 1) launch_sell_U<VM, 1>(a, KT, s);
        else if (A.unroll <= 2) launch_sell_U<VM, 2>(a, KT, s);
        else launch_sell_U<VM, 4>(a, KT, s);
    }
}

template <int VM>
static gbsp_status launch_family(const Mat &A, JdsArgs a, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    const int fmt = A.format;
    if (fmt == GBSP_SELL && A.stage_col && a.k == 1 && !a.x_perm) {
        if (A.unroll <= 1) return launch_sell_staged_U<VM, 1>(A, a, s);
        if (A.unroll <= 2) return launch_sell_staged_U<VM, 2>(A, a, s);
        return launch_sell_staged_U<VM, 4>(A, a, s);
    }
    if (fmt == GBSP_SELL) {
        launch_sell<VM>(A, a, s);
        return GBSP_OK;
    }
    if (fmt == GBSP_PSELL) {
        launch_psell<VM>(A, a, s);
        return GBSP_OK;
    }
    if (a.k > 1 || fmt == GBSP_NBJDS || fmt == GBSP_RBJDS || fmt == GBSP_SOJDS) {
        const bool contig = fmt == GBSP_RBJDS || fmt == GBSP_SOJDS;
        if (!contig && fmt != GBSP_NBJDS) a.block = 256;  // JDS / NUJDS walked per 256-row block
        int KT = 1;
        if (a.k > 1) {
            const int tile = A.kopt.rhs_tile > 0 ? std::min(A.kopt.rhs_tile, 16) : 16;
            const int cols = std::min(a.k, tile);
            KT = 2;
            while (KT < cols) KT <<= 1;
        }
        for (int c0 = 0; c0 < a.k; c0 += KT) {
            a.c0 = c0;
            if (contig) launch_block<VM, true>(a, KT, s);
            else launch_block<VM, false>(a, KT, s);
        }
        return GBSP_OK;
    }
    if (fmt == GBSP_JDS_LITERAL) {
        if (!a.accumulate) {
            // resvec starts at zero; rows are written through y_perm's image,
            // which is every row, so zero the whole output
            const int64_t n = a.n_rows;
            zero_rows_kernel<T><<<(unsigned)ceil_div(std::max<int64_t>(n, 1), 256), 256, 0, s>>>(
                n, static_cast<T *>(a.y), a.ldy, 1);
        }
        for (int64_t d = 0; d < A.n_diag; ++d) {
            const int64_t len = A.h_jd_ptr[d + 1] - A.h_jd_ptr[d];
            if (len <= 0) break;
            jds_literal_kernel<T><<<(unsigned)ceil_div(len, 256), 256, 0, s>>>(
                len, A.h_jd_ptr[d], a.col, static_cast<const T *>(a.val), static_cast<const T *>(a.x),
                a.ldx, static_cast<T *>(a.y), a.ldy, a.x_perm, a.y_perm);
        }
        return GBSP_OK;
    }
    const int u = fmt == GBSP_NUJDS ? A.unroll : 1;
    const int R = A.kopt.rows_per_warp > 1 ? A.kopt.rows_per_warp : 1;  // rows per thread
    if (A.split_k > 0) {
        // deep diagonals (chunk partial sums), the walk that stops at the
        // split depth, then the merge of the two for the deep rows
        a.d_limit = A.split_depth;
        a.split_k = A.split_k;
        a.split_table = A.split_table;
        a.split_items = A.split_items;
        a.split_part = A.split_part;
        a.split_shallow = A.split_shallow;
        a.split_rows = A.split_rows;
        // fork: the deep kernel on the side stream, overlapping the walk
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(A.split_items_total, (int64_t)num_sms() * 16));
        GBSP_CUDA(cudaEventRecord(A.split_fork, s));
        GBSP_CUDA(cudaStreamWaitEvent(A.split_side, A.split_fork, 0));
        jds_deep_kernel<VM><<<(unsigned)grid, 256, 0, A.split_side>>>(a, A.split_items_total);
        GBSP_CUDA(cudaEventRecord(A.split_join, A.split_side));
    }
    if (u <= 1) launch_row<VM, 1>(a, R, s);
    else if (u <= 2) launch_row<VM, 2>(a, R, s);
    else if (u <= 4) launch_row<VM, 4>(a, R, s);
    else if (u <= 8) launch_row<VM, 8>(a, std::min(R, 2), s);
    else launch_row<VM, 16>(a, 1, s);
    if (A.split_k > 0) {
        GBSP_CUDA(cudaStreamWaitEvent(s, A.split_join, 0));  // join
        const int64_t work = std::max<int64_t>(A.split_wide_rows * 32, A.split_rows - A.split_wide_rows);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)num_sms() * 8));
        jds_split_merge_kernel<VM><<<(unsigned)grid, 256, 0, s>>>(a, A.split_wide_rows);
    }
    return GBSP_OK;
}

gbsp_status jds_launch(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (A.n_rows == 0) return GBSP_OK;
    JdsArgs a{};
    a.n_rows = A.n_rows;
    a.n_diag = A.n_diag;
    a.jd_ptr = A.jd_ptr;
    a.col = A.col;
    a.blk_ptr = A.blk_ptr;
    a.val = A.val;
    a.x = v.x;
    a.y = v.y;
    a.ldx = v.ldx;
    a.ldy = v.ldy;
    a.k = v.k;
    a.c0 = 0;
    a.accumulate = v.accumulate;
    a.block = A.format == GBSP_RBJDS || A.format == GBSP_SOJDS ? A.built_block
                                                                 : std::max(A.block, 1);
    a.x_perm = v.x_perm;
    a.y_perm = v.y_perm;
    a.rlen = A.rlen;
    a.d_limit = A.n_diag;
    a.split_k = 0;
    a.split_rows = 0;
    a.split_shallow = nullptr;
    a.n_cols = A.n_cols;
    a.grid_limit = A.grid_limit;
    {
        const int64_t ybytes = A.n_rows * std::max<int64_t>(v.ldy, v.k) * (A.dtype == GBSP_F64 ? 8 : 4);
        a.y_evict_first = ybytes > (int64_t(32) << 20) ? 1 : 0;
    }
    gbsp_status st;
    if (A.dtype == GBSP_F64) st = launch_family<VM_F64>(A, a, s);
    else if (A.kopt.accum == GBSP_ACC_COMPENSATED) st = launch_family<VM_F32C>(A, a, s);
    else st = launch_family<VM_F32>(A, a, s);
    if (st != GBSP_OK) return st;
    GBSP_LAUNCH_CHECK("jds product kernel");
    return GBSP_OK;
}

// Split set-up: chunks of `chunk` diagonals from `depth` on; chunk k holds
// the rows [0, diagLen(d_begin)).  Workspace: the chunk table, the per-chunk
// first CTA item, then the ragged partial sums (one accumulator per row and
// chunk), then the walk sums of the rows of chunk 0.
static int64_t acc_bytes(int dtype, int accum) {
    return dtype == GBSP_F64 ? 8 : (accum == GBSP_ACC_COMPENSATED ? 8 : 4);
}

static void split_plan(const Mat &A, int32_t depth, int32_t chunk, std::vector<int4> *table,
                       std::vector<int32_t> *items, int64_t *parts) {
    table->clear();
    items->clear();
    int64_t off = 0, it = 0;
    for (int64_t d0 = depth; d0 < A.n_diag; d0 += chunk) {
        const int64_t d1 = std::min<int64_t>(d0 + chunk, A.n_diag);
        const int64_t rows = A.h_jd_ptr[d0 + 1] - A.h_jd_ptr[d0];
        if (rows <= 0) break;
        table->push_back(make_int4((int)d0, (int)d1, (int)rows, (int)off));
        items->push_back((int32_t)it);
        off += rows;
        it += ceil_div(rows, 256);
    }
    items->push_back((int32_t)it);
    *parts = off;
}

gbsp_status jds_split_bytes_impl(const Mat &A, int32_t depth, int32_t chunk, int64_t *bytes) {
    std::vector<int4> t;
    std::vector<int32_t> it;
    int64_t parts = 0;
    split_plan(A, depth, chunk, &t, &it, &parts);
    const int64_t rows = t.empty() ? 0 : t[0].z;  // rows deeper than the split depth
    *bytes = 256 + 16 * (int64_t)t.size() + 4 * (int64_t)it.size() + 16 +
             (parts + rows) * acc_bytes(A.dtype, GBSP_ACC_COMPENSATED);
    return GBSP_OK;
}

gbsp_status jds_split_impl(Mat &A, int32_t depth, int32_t chunk, void *ws, int64_t bytes, cudaStream_t s) {
    if (depth <= 0 || depth >= A.n_diag) {
        A.split_k = 0;
        A.split_depth = 0;
        return GBSP_OK;
    }
    std::vector<int4> t;
    std::vector<int32_t> it;
    int64_t parts = 0;
    split_plan(A, depth, chunk, &t, &it, &parts);
    int64_t need = 0;
    jds_split_bytes_impl(A, depth, chunk, &need);
    if (bytes < need) {
        set_error("gbsp_jds_split: workspace needs %lld bytes", (long long)need);
        return GBSP_ERR_NOMEM;
    }
    char *p = static_cast<char *>(ws);
    int4 *dt = reinterpret_cast<int4 *>(p);
    int32_t *di = reinterpret_cast<int32_t *>(p + 16 * t.size());
    const int64_t po = ((16 * (int64_t)t.size() + 4 * (int64_t)it.size()) + 255) & ~int64_t(255);
    if (!A.split_side) {
        GBSP_CUDA(cudaStreamCreateWithFlags(&A.split_side, cudaStreamNonBlocking));
        GBSP_CUDA(cudaEventCreateWithFlags(&A.split_fork, cudaEventDisableTiming));
        GBSP_CUDA(cudaEventCreateWithFlags(&A.split_join, cudaEventDisableTiming));
    }
    GBSP_CUDA(cudaMemcpyAsync(dt, t.data(), 16 * t.size(), cudaMemcpyHostToDevice, s));
    GBSP_CUDA(cudaMemcpyAsync(di, it.data(), 4 * it.size(), cudaMemcpyHostToDevice, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    A.split_depth = depth;
    A.split_chunk = chunk;
    A.split_k = (int32_t)t.size();
    A.split_table = dt;
    A.split_items = di;
    A.split_items_total = it.back();
    A.split_part = p + po;
    A.split_rows = t.empty() ? 0 : t[0].z;
    A.split_wide_rows = t.size() > 8 ? t[8].z : 0;  // rows with more than 8 chunks
    A.split_shallow = p + po + parts * acc_bytes(A.dtype, GBSP_ACC_COMPENSATED);
    return GBSP_OK;
}

gbsp_status permute_launch(const Mat &A, int32_t dir, int32_t k, const void *in, int64_t ld_in,
                           void *out, int64_t ld_out, cudaStream_t s) {
    const int64_t n = A.n_rows * (int64_t)k;
    if (n == 0) return GBSP_OK;
    const unsigned grid = (unsigned)ceil_div(n, 256);
    if (A.dtype == GBSP_F64)
        permute_kernel<double><<<grid, 256, 0, s>>>(A.n_rows, k, A.perm, dir,
                                                    static_cast<const double *>(in), ld_in,
                                                    static_cast<double *>(out), ld_out);
    else
        permute_kernel<float><<<grid, 256, 0, s>>>(A.n_rows, k, A.perm, dir,
                                                   static_cast<const float *>(in), ld_in,
                                                   static_cast<float *>(out), ld_out);
    GBSP_LAUNCH_CHECK("permute_kernel");
    return GBSP_OK;
}

}  // namespace gbsp
