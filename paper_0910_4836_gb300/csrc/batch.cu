// Batched products in one persistent launch.
//
// Many matrices of uneven sizes, each with its own k right-hand sides,
// storage scheme and kernel options, are cut into work items of about
// `chunk` stored entries (a contiguous range of rows of one matrix).  The
// work table lives in caller memory; CTAs of one persistent grid take items
// through a device counter (reset by a memset on the stream before every
// launch, so the pair can be captured in a CUDA graph and replayed).  Each
// item runs the same per-row arithmetic as the stand-alone kernel of its
// format and options, so a matrix's batched result is bit-identical to the
// result of gbsp_spmm on it alone.
#include <algorithm>
#include <new>
#include <vector>

#include "accum.cuh"
#include "internal.cuh"
#include "sm100.cuh"

namespace gbsp {

struct BatchMat {
    int32_t kind;      // KIND_CRS / KIND_JDS
    int32_t format;    // gbsp_format
    int32_t vm;        // ValMode
    int32_t k;         // right-hand sides
    int32_t lanes, rows, rhs_tile, unroll;
    int32_t block;     // RBJDS / SOJDS block
    int32_t pad;
    int64_t n_rows, n_diag;
    const int32_t *row_ptr, *col, *jd_ptr, *blk_ptr, *rlen;
    const void *val;
    const void *x;
    void *y;
    int64_t ldx, ldy;
};

struct BatchWork {
    int32_t mat;
    int32_t pad;
    int64_t rb, re;  // rows [rb, re) of matrix `mat`
};

constexpr int kBatchThreads = 256;
constexpr uint64_t kReadyLimitNs = 1000000000ull;  // 1 s bound on the ready-flag wait

// CRS rows [rb, re), k = 1, L lanes per row (same arithmetic as crs_vector_kernel).
template <int VM, int L>
__device__ void batch_crs_rows(const BatchMat &m, int64_t rb, int64_t re) {
    typedef typename ValT<VM>::T T;
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31, grp = lane / L, gl = lane % L, wid = threadIdx.x >> 5;
    const T *val = static_cast<const T *>(m.val);
    const T *x = static_cast<const T *>(m.x);
    T *y = static_cast<T *>(m.y);
    for (int64_t base = rb + (int64_t)wid * G; base < re; base += (int64_t)(kBatchThreads / 32) * G) {
        const int64_t r = base + grp;
        int k0 = 0, k1 = 0;
        if (r < re) {
            k0 = __ldg(m.row_ptr + r);
            k1 = __ldg(m.row_ptr + r + 1);
        }
        Acc<VM> acc;
        acc.init();
        for (int j = k0 + gl; j < k1; j += L) acc.add(__ldg(val + j), ld_vec(x + (int64_t)__ldg(m.col + j) * m.ldx));
        group_reduce<L, VM>(acc);
        if (gl == 0 && r < re) y[r * m.ldy] = acc.result();
    }
}

// CRS rows with k > 1: lanes over right-hand sides (same as crs_spmm_kernel).
template <int VM, int KT>
__device__ void batch_crs_spmm_rows(const BatchMat &m, int64_t rb, int64_t re, int c0) {
    typedef typename ValT<VM>::T T;
    constexpr int G = 32 / KT;
    const int lane = threadIdx.x & 31, grp = lane / KT, c = lane % KT, wid = threadIdx.x >> 5;
    const int cc = c0 + c;
    const bool active = cc < m.k;
    const T *val = static_cast<const T *>(m.val);
    const T *X = static_cast<const T *>(m.x);
    T *Y = static_cast<T *>(m.y);
    for (int64_t r = rb + (int64_t)wid * G + grp; r < re; r += (int64_t)(kBatchThreads / 32) * G) {
        const int k0 = __ldg(m.row_ptr + r), k1 = __ldg(m.row_ptr + r + 1);
        Acc<VM> acc;
        acc.init();
        for (int j = k0; j < k1; ++j) {
            const int ci = __ldg(m.col + j);
            const T vi = __ldg(val + j);
            if (active) acc.add(vi, ld_vec(X + (int64_t)ci * m.ldx + cc));
        }
        if (active) Y[r * m.ldy + cc] = acc.result();
    }
}

// JDS-family rows [rb, re): one thread per row, every right-hand side of the
// tile per thread, row entries in slot order (same arithmetic as the JDS
// kernels).  RBJDS / SOJDS work items are whole blocks.
template <int VM, int KT>
__device__ void batch_jds_rows(const BatchMat &m, int64_t rb, int64_t re, int c0) {
    typedef typename ValT<VM>::T T;
    const T *val = static_cast<const T *>(m.val);
    const T *x = static_cast<const T *>(m.x);
    T *y = static_cast<T *>(m.y);
    const bool contig = m.format == GBSP_RBJDS || m.format == GBSP_SOJDS;
    for (int64_t r = rb + threadIdx.x; r < re; r += kBatchThreads) {
        Acc<VM> acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q].init();
        int64_t b0 = 0, b1 = 0, off = 0;
        if (contig) {
            const int64_t blk = r / m.block;
            b0 = blk * m.block;
            b1 = min(b0 + (int64_t)m.block, m.n_rows);
            off = __ldg(m.blk_ptr + blk);
        }
        int32_t st = __ldg(m.jd_ptr);
        for (int64_t d = 0; d < m.n_diag; ++d) {
            const int32_t en = __ldg(m.jd_ptr + d + 1);
            const int64_t dl = en - st;
            if (dl <= r) break;
            const int64_t kk = contig ? off + (r - b0) : (int64_t)st + r;
            const int ci = ld_stream(m.col + kk);
            const T vi = ld_stream(val + kk);
            const T *xr = x + (int64_t)ci * m.ldx + c0;
#pragma unroll
            for (int q = 0; q < KT; ++q)
                if (c0 + q < m.k) acc[q].add(vi, ld_vec(xr + q));
            if (contig) off += min(b1, dl) - b0;
            st = en;
        }
#pragma unroll
        for (int q = 0; q < KT; ++q)
            if (c0 + q < m.k) y[r * m.ldy + c0 + q] = acc[q].result();
    }
}

// SELL rows [rb, re) (whole 32-row blocks): one warp per block, lane = row
// (same arithmetic as sell_kernel).  PLAIN: one vector read directly.
template <int VM, int KT, bool PLAIN>
__device__ void batch_sell_rows(const BatchMat &m, int64_t rb, int64_t re, int c0) {
    typedef typename ValT<VM>::T T;
    constexpr int U = 4;  // slots whose loads are in flight together
    const T *val = static_cast<const T *>(m.val);
    const T *x = static_cast<const T *>(m.x);
    T *y = static_cast<T *>(m.y);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b = rb / 32 + wid; b * 32 < re; b += kBatchThreads / 32) {
        const int64_t r = b * 32 + lane;
        const int32_t len = r < m.n_rows ? __ldg(m.rlen + r) : 0;
        const int32_t width = __shfl_sync(0xffffffffu, len, 0);
        int32_t off = __ldg(m.blk_ptr + b);  // entry offsets fit int32
        Acc<VM> acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q].init();
        // U slots loaded together, then their products (the SELL kernel's walk)
        int c[U];
        T v[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const bool ok = len > j;
            c[j] = ok ? ld_stream(m.col + (off + lane)) : -1;
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
                    const T *xr = x + (int64_t)c[j] * m.ldx + c0;
#pragma unroll
                    for (int q = 0; q < KT; ++q)
                        if (c0 + q < m.k) acc[q].add(v[j], ld_vec(xr + q));
                }
            }
            if (d0 + U >= width) break;
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = len > d0 + U + j;
                c[j] = ok ? ld_stream(m.col + (off + lane)) : -1;
                v[j] = ok ? ld_stream(val + (off + lane)) : T(0);
                off += __popc(__ballot_sync(0xffffffffu, ok));
            }
        }
        if (r < m.n_rows) {
#pragma unroll
            for (int q = 0; q < KT; ++q)
                if (c0 + q < m.k) y[r * m.ldy + c0 + q] = acc[q].result();
        }
    }
}

// Right-hand-side tiles are clamped to KTMAX, the widest tile the kernel
// instance carries (a batch whose matrices all have k = 1 runs an instance
// without the wide-tile code and its registers; k = 16 runs as two 8-wide
// tiles at twice the occupancy of a 16-wide one).  The tile width never
// changes a result: every right-hand side is summed on its own, in the same
// entry order.
template <int KTMAX>
__device__ __forceinline__ int clamp_tile(int kt) { return kt < KTMAX ? kt : KTMAX; }

template <int VM, int KTMAX>
__device__ void batch_item(const BatchMat &m, int64_t rb, int64_t re) {
    if (m.kind == KIND_JDS && m.format == GBSP_SELL) {
        int KT = 1;
        if (m.k > 1) {
            KT = 2;
            while (KT < min(m.k, m.rhs_tile > 0 ? min(m.rhs_tile, 16) : 16)) KT <<= 1;
            KT = clamp_tile<KTMAX>(KT);
        }
        for (int c0 = 0; c0 < m.k; c0 += KT) {
            if (KT == 1) {  // k = 1, so c0 = 0
                if (m.ldx == 1) batch_sell_rows<VM, 1, true>(m, rb, re, c0);
                else batch_sell_rows<VM, 1, false>(m, rb, re, c0);
            }
            if constexpr (KTMAX >= 2) if (KT == 2) batch_sell_rows<VM, 2, false>(m, rb, re, c0);
            if constexpr (KTMAX >= 4) if (KT == 4) batch_sell_rows<VM, 4, false>(m, rb, re, c0);
            if constexpr (KTMAX >= 8) if (KT == 8) batch_sell_rows<VM, 8, false>(m, rb, re, c0);
            if constexpr (KTMAX >= 16) if (KT >= 16) batch_sell_rows<VM, 16, false>(m, rb, re, c0);
        }
        return;
    }
    if (m.kind == KIND_CRS) {
        if (m.k == 1) {
            switch (m.lanes) {
                case 1: batch_crs_rows<VM, 1>(m, rb, re); break;
                case 2: batch_crs_rows<VM, 2>(m, rb, re); break;
                case 4: batch_crs_rows<VM, 4>(m, rb, re); break;
                case 8: batch_crs_rows<VM, 8>(m, rb, re); break;
                case 16: batch_crs_rows<VM, 16>(m, rb, re); break;
                default: batch_crs_rows<VM, 32>(m, rb, re); break;
            }
        } else if constexpr (KTMAX >= 2) {
            int KT = 2;
            while (KT < min(m.k, m.rhs_tile > 0 ? min(m.rhs_tile, 32) : 16)) KT <<= 1;
            KT = clamp_tile<KTMAX>(KT);
            for (int c0 = 0; c0 < m.k; c0 += KT) {
                if (KT == 2) batch_crs_spmm_rows<VM, 2>(m, rb, re, c0);
                if constexpr (KTMAX >= 4) if (KT == 4) batch_crs_spmm_rows<VM, 4>(m, rb, re, c0);
                if constexpr (KTMAX >= 8) if (KT == 8) batch_crs_spmm_rows<VM, 8>(m, rb, re, c0);
                if constexpr (KTMAX >= 16) if (KT == 16) batch_crs_spmm_rows<VM, 16>(m, rb, re, c0);
                if constexpr (KTMAX >= 32) if (KT >= 32) batch_crs_spmm_rows<VM, 32>(m, rb, re, c0);
            }
        }
    } else {
        if (m.k == 1) {
            batch_jds_rows<VM, 1>(m, rb, re, 0);
        } else if constexpr (KTMAX >= 2) {
            int KT = 2;
            while (KT < min(m.k, m.rhs_tile > 0 ? min(m.rhs_tile, 16) : 16)) KT <<= 1;
            KT = clamp_tile<KTMAX>(KT);
            for (int c0 = 0; c0 < m.k; c0 += KT) {
                if (KT == 2) batch_jds_rows<VM, 2>(m, rb, re, c0);
                if constexpr (KTMAX >= 4) if (KT == 4) batch_jds_rows<VM, 4>(m, rb, re, c0);
                if constexpr (KTMAX >= 8) if (KT == 8) batch_jds_rows<VM, 8>(m, rb, re, c0);
                if constexpr (KTMAX >= 16) if (KT >= 16) batch_jds_rows<VM, 16>(m, rb, re, c0);
            }
        }
    }
}

template <int KTMAX>
__global__ void __launch_bounds__(kBatchThreads, KTMAX == 1 ? 5 : 4)
batch_kernel(const BatchMat *__restrict__ mats, const BatchWork *__restrict__ work, int64_t n_work,
             int32_t *counter, const volatile int32_t *ready, int32_t *status) {
    __shared__ int64_t next[2];
    __shared__ int32_t go;
    if (threadIdx.x == 0) {
        go = 1;
        if (ready) {
            // bounded wait for a flag set by the host or by work finished
            // earlier on the stream; never by a concurrently running kernel
            const uint64_t t0 = global_timer_ns();
            while (*ready == 0) {
                if (global_timer_ns() - t0 > kReadyLimitNs) {
                    go = 0;
                    if (status) atomicExch(status, (int32_t)GBSP_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(1000);
            }
        }
    }
    __syncthreads();
    if (!go) return;
    // Thread 0 claims the next item once its own share of the current one
    // is done, into the other of two shared slots, so one barrier per item
    // suffices.  Claiming only then (not ahead) keeps a CTA busy with an
    // expensive item from holding a cheap one at the tail of the queue.
    // Which CTA runs an item never changes its result.
    if (threadIdx.x == 0) next[0] = atomicAdd(counter, 1);
    __syncthreads();
    for (int i = 0;; i ^= 1) {
        const int64_t w = next[i];
        if (w >= n_work) break;
        const BatchWork wk = work[w];
        const BatchMat m = mats[wk.mat];
        if (m.vm == VM_F64) batch_item<VM_F64, KTMAX>(m, wk.rb, wk.re);
        else if (m.vm == VM_F32C) batch_item<VM_F32C, KTMAX>(m, wk.rb, wk.re);
        else batch_item<VM_F32, KTMAX>(m, wk.rb, wk.re);
        if (threadIdx.x == 0) next[i ^ 1] = atomicAdd(counter, 1);
        // every thread has read next[i]; next[i ^ 1] is written and visible
        __syncthreads();
    }
}

}  // namespace gbsp

using namespace gbsp;

struct gbsp_batch_s {
    int32_t n_mats = 0;
    int64_t n_work = 0;
    int32_t *counter = nullptr;
    const BatchMat *mats = nullptr;
    const BatchWork *work = nullptr;
    const int32_t *ready = nullptr;
    int grid = 0;
    int ktmax = 1;  // widest right-hand-side tile of the kernel instance: 1, 4 or 8
};

namespace {

constexpr int64_t kCounterBytes = 256;

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

// Host-side work list: contiguous row ranges of about `chunk` entries (whole
// blocks for RBJDS / SOJDS).  Needs the row pointers on the host, so it reads
// the CRS row_ptr (or JDS jd_ptr) back once.
gbsp_status make_work(int32_t n, const gbsp_batch_item *items, int32_t chunk, cudaStream_t s,
                      std::vector<BatchMat> *mats, std::vector<BatchWork> *work) {
    mats->clear();
    work->clear();
    for (int32_t b = 0; b < n; ++b) {
        const gbsp_batch_item &it = items[b];
        if (!it.A) return arg_error("gbsp_batch: NULL handle in item");
        const Mat &A = *it.A;
        if (A.kind == KIND_DIA) {
            set_error("gbsp_batch: DIA handles are not batched");
            return GBSP_ERR_UNSUPPORTED;
        }
        if (A.kind == KIND_JDS && A.format == GBSP_PSELL) {
            set_error("gbsp_batch: PSELL handles are not batched; use SELL");
            return GBSP_ERR_UNSUPPORTED;
        }
        if (it.k < 1 || it.ldx < it.k || it.ldy < it.k) return arg_error("gbsp_batch: bad k / leading dimension");
        if (A.n_rows > 0 && (!it.X || !it.Y)) return arg_error("gbsp_batch: NULL X or Y");
        BatchMat m{};
        m.kind = A.kind;
        m.format = A.kind == KIND_CRS ? GBSP_CRS : A.format;
        m.vm = A.dtype == GBSP_F64 ? VM_F64 : (A.kopt.accum == GBSP_ACC_COMPENSATED ? VM_F32C : VM_F32);
        m.k = it.k;
        m.lanes = A.kopt.lanes > 0 ? A.kopt.lanes : 4;
        m.rows = A.kopt.rows_per_warp;
        m.rhs_tile = A.kopt.rhs_tile;
        m.unroll = A.unroll;
        m.block = A.built_block > 0 ? A.built_block : 1;
        m.n_rows = A.n_rows;
        m.n_diag = A.n_diag;
        m.row_ptr = A.row_ptr;
        m.col = A.col;
        m.jd_ptr = A.jd_ptr;
        m.blk_ptr = A.blk_ptr;
        m.rlen = A.rlen;
        m.val = A.val;
        m.x = it.X;
        m.y = it.Y;
        m.ldx = it.ldx;
        m.ldy = it.ldy;
        if (m.format == GBSP_JDS_LITERAL) m.format = GBSP_JDS;  // same arithmetic row by row
        mats->push_back(m);
        if (A.n_rows == 0) continue;
        // row weights: entries per row, from the host copy of the structure
        std::vector<int64_t> start;  // cumulative entries before row r, sampled at chunk edges
        if (A.kind == KIND_CRS) {
            std::vector<int32_t> rp((size_t)A.n_rows + 1);
            GBSP_CUDA(cudaMemcpyAsync(rp.data(), A.row_ptr, 4 * (A.n_rows + 1), cudaMemcpyDeviceToHost, s));
            GBSP_CUDA(cudaStreamSynchronize(s));
            int64_t rb = 0;
            const int64_t minrows = 32;
            while (rb < A.n_rows) {
                int64_t re = rb + minrows;
                // extend while under the chunk (binary search on row_ptr)
                const int64_t target = (int64_t)rp[(size_t)rb] + chunk;
                int64_t lo = std::min(re, A.n_rows), hi = A.n_rows;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) / 2;
                    if (rp[(size_t)mid] <= target) lo = mid;
                    else hi = mid - 1;
                }
                re = std::max(std::min(re, A.n_rows), lo);
                work->push_back(BatchWork{b, 0, rb, re});
                rb = re;
            }
        } else if (A.format == GBSP_SELL) {
            // whole 32-row blocks of about `chunk` entries
            std::vector<int32_t> bp((size_t)A.n_blocks + 1);
            GBSP_CUDA(cudaMemcpyAsync(bp.data(), A.blk_ptr, 4 * (A.n_blocks + 1), cudaMemcpyDeviceToHost, s));
            GBSP_CUDA(cudaStreamSynchronize(s));
            int64_t b0 = 0;
            while (b0 < A.n_blocks) {
                int64_t b1 = b0 + 1;
                while (b1 < A.n_blocks && (int64_t)bp[(size_t)b1 + 1] - bp[(size_t)b0] <= chunk) ++b1;
                work->push_back(BatchWork{b, 0, b0 * 32, std::min(b1 * 32, A.n_rows)});
                b0 = b1;
            }
        } else {
            // JDS family: rows are sorted by decreasing length; entries of
            // rows [rb, re) = sum_d clamp(diagLen(d) - rb, 0, re - rb)
            const std::vector<int32_t> &jd = A.h_jd_ptr;
            const int64_t blk = (A.format == GBSP_RBJDS || A.format == GBSP_SOJDS) ? A.built_block : 32;
            auto entries = [&](int64_t rb, int64_t re) {
                int64_t e = 0;
                for (size_t d = 0; d + 1 < jd.size(); ++d) {
                    const int64_t dl = jd[d + 1] - jd[d];
                    if (dl <= rb) break;
                    e += std::min(dl, re) - rb;
                }
                return e;
            };
            int64_t rb = 0;
            while (rb < A.n_rows) {
                int64_t re = std::min(rb + blk, A.n_rows);
                while (re < A.n_rows && entries(rb, std::min(re + blk, A.n_rows)) <= chunk)
                    re = std::min(re + blk, A.n_rows);
                work->push_back(BatchWork{b, 0, rb, re});
                rb = re;
            }
        }
    }
    return GBSP_OK;
}

}  // namespace

extern "C" {

gbsp_status gbsp_batch_plan(int32_t n, const gbsp_batch_item *items, int32_t chunk, int64_t *table_bytes) {
    if (n < 0 || (n > 0 && !items) || !table_bytes) return arg_error("gbsp_batch_plan: bad arguments");
    if (chunk <= 0) chunk = 4096;
    std::vector<BatchMat> mats;
    std::vector<BatchWork> work;
    gbsp_status st = make_work(n, items, chunk, nullptr, &mats, &work);
    if (st != GBSP_OK) return st;
    *table_bytes = kCounterBytes + align256((int64_t)sizeof(BatchMat) * n) +
                   align256((int64_t)sizeof(BatchWork) * (int64_t)work.size());
    return GBSP_OK;
}

gbsp_status gbsp_batch_create(int32_t n, const gbsp_batch_item *items, int32_t chunk, void *d_table,
                              int64_t table_bytes, const int32_t *d_ready, void *stream, gbsp_batch *out) {
    if (!out) return arg_error("gbsp_batch_create: out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !items) || !d_table) return arg_error("gbsp_batch_create: bad arguments");
    if (reinterpret_cast<uintptr_t>(d_table) & 255) return arg_error("gbsp_batch_create: table must be 256-byte aligned");
    if (chunk <= 0) chunk = 4096;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<BatchMat> mats;
    std::vector<BatchWork> work;
    gbsp_status st = make_work(n, items, chunk, s, &mats, &work);
    if (st != GBSP_OK) return st;
    const int64_t need = kCounterBytes + align256((int64_t)sizeof(BatchMat) * n) +
                         align256((int64_t)sizeof(BatchWork) * (int64_t)work.size());
    if (table_bytes < need) {
        set_error("gbsp_batch_create: table needs %lld bytes", (long long)need);
        return GBSP_ERR_NOMEM;
    }
    char *p = static_cast<char *>(d_table);
    gbsp_batch b = new (std::nothrow) gbsp_batch_s();
    if (!b) return arg_error("gbsp_batch_create: out of host memory");
    b->n_mats = n;
    b->n_work = (int64_t)work.size();
    b->counter = reinterpret_cast<int32_t *>(p);
    b->mats = reinterpret_cast<const BatchMat *>(p + kCounterBytes);
    b->work = reinterpret_cast<const BatchWork *>(p + kCounterBytes + align256((int64_t)sizeof(BatchMat) * n));
    b->ready = d_ready;
    if (n > 0)
        GBSP_CUDA(cudaMemcpyAsync(const_cast<BatchMat *>(b->mats), mats.data(), sizeof(BatchMat) * n,
                                  cudaMemcpyHostToDevice, s));
    if (!work.empty())
        GBSP_CUDA(cudaMemcpyAsync(const_cast<BatchWork *>(b->work), work.data(), sizeof(BatchWork) * work.size(),
                                  cudaMemcpyHostToDevice, s));
    GBSP_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
    int kmax = 1;
    for (int32_t i = 0; i < n; ++i) kmax = std::max(kmax, (int)items[i].k);
    // the widest tile decides the registers, hence the CTAs per SM: 48
    // registers for 1 (5 CTAs of 256 threads), 64 for 4 and 8 (4 CTAs),
    // about 128 for 16 (2 CTAs); wider k runs as several 8-wide tiles
    b->ktmax = kmax == 1 ? 1 : (kmax <= 4 ? 4 : 8);
    int per_sm = 0;
    if (b->ktmax == 1)
        GBSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<1>, kBatchThreads, 0));
    else if (b->ktmax == 4)
        GBSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<4>, kBatchThreads, 0));
    else
        GBSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<8>, kBatchThreads, 0));
    b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->n_work, (int64_t)num_sms() * std::max(per_sm, 1)));
    *out = b;
    return GBSP_OK;
}

gbsp_status gbsp_batch_run(gbsp_batch b, int32_t *d_status, void *stream) {
    if (!b) return arg_error("gbsp_batch_run: NULL batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->n_work == 0) return GBSP_OK;
    GBSP_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int32_t), s));
    if (b->ktmax == 1)
        batch_kernel<1><<<b->grid, kBatchThreads, 0, s>>>(b->mats, b->work, b->n_work, b->counter, b->ready, d_status);
    else if (b->ktmax == 4)
        batch_kernel<4><<<b->grid, kBatchThreads, 0, s>>>(b->mats, b->work, b->n_work, b->counter, b->ready, d_status);
    else
        batch_kernel<8><<<b->grid, kBatchThreads, 0, s>>>(b->mats, b->work, b->n_work, b->counter, b->ready, d_status);
    GBSP_LAUNCH_CHECK("batch_kernel");
    return GBSP_OK;
}

gbsp_status gbsp_batch_info(gbsp_batch b, int64_t *n_work, int32_t *grid) {
    if (!b) return arg_error("gbsp_batch_info: NULL batch");
    if (n_work) *n_work = b->n_work;
    if (grid) *grid = b->grid;
    return GBSP_OK;
}

gbsp_status gbsp_batch_destroy(gbsp_batch b) {
    delete b;
    return GBSP_OK;
}

}  // extern "C"
