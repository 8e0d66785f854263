// Access-pattern analysis of the x gather.
//
// gbsp_stride_hist: the stride distribution of Sect. 4.2 (its Fig. 4a) -- the
// jumps between consecutive column indices in storage order, which is the
// order the paper's serial CRS, JDS, RBJDS and SOJDS loops read x.
// gbsp_warp_sectors: the GB300 counterpart -- for every warp-wide gather the
// product kernels issue, the number of distinct 32-byte sectors of x it
// touches (1 to 32; the L2 moves whole sectors, so this is the gather's cost
// in L2 traffic, the GPU analogue of the paper's count of cache lines loaded
// per entry).
//
// Both build a histogram in shared memory per CTA and add it to the caller's
// int64 array with integer atomics, so the counts are exact and the same on
// every run.
#include <algorithm>

#include "internal.cuh"
#include "accum.cuh"

namespace gbsp {

namespace {

constexpr int S_THREADS = 256;
constexpr int S_BINS = 33;

__device__ __forceinline__ int stride_bin(int64_t s) {
    const uint64_t a = (uint64_t)(s < 0 ? -s : s);
    return a == 0 ? 0 : 64 - __clzll((long long)a);
}

__global__ void __launch_bounds__(S_THREADS)
    stride_hist_kernel(const int32_t *__restrict__ col, int64_t nnz, unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long h[2 * S_BINS];
    for (int i = threadIdx.x; i < 2 * S_BINS; i += S_THREADS) h[i] = 0;
    __syncthreads();
    const int64_t T = (int64_t)gridDim.x * S_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * S_THREADS + threadIdx.x; i + 1 < nnz; i += T) {
        const int64_t s = (int64_t)__ldg(col + i + 1) - (int64_t)__ldg(col + i);
        atomicAdd(&h[(s < 0 ? S_BINS : 0) + stride_bin(s)], 1ull);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * S_BINS; i += S_THREADS)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// Distinct sectors among the active lanes of one warp-wide gather: inactive
// lanes carry a negative key of their own, so they match nobody; a lane
// counts when it is the lowest lane of its match group.
__device__ __forceinline__ int warp_distinct(bool active, int64_t col, int elem_bytes) {
    const int lane = threadIdx.x & 31;
    const long long key = active ? (long long)(col * elem_bytes / 32) : -1 - (long long)lane;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const bool leader = active && (__ffs(grp) - 1) == lane;
    return __popc(__ballot_sync(0xffffffffu, leader));
}

__device__ __forceinline__ void flush_bins(unsigned long long *h, unsigned long long *hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < S_BINS; i += S_THREADS)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// CRS with `lanes` lanes per row: a warp holds 32/lanes consecutive rows; at
// step t lane l of row group g reads entry row_ptr[r] + t*lanes + l.
__global__ void __launch_bounds__(S_THREADS)
    sectors_crs_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                       int lanes, int elem_bytes, unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long h[S_BINS];
    for (int i = threadIdx.x; i < S_BINS; i += S_THREADS) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int groups = 32 / lanes;
    const int g = lane / lanes, l = lane % lanes;
    const int64_t n_warps = ceil_div_dev(n_rows, groups);
    const int64_t warps_total = (int64_t)gridDim.x * (S_THREADS / 32);
    for (int64_t w = (int64_t)blockIdx.x * (S_THREADS / 32) + (threadIdx.x >> 5); w < n_warps; w += warps_total) {
        const int64_t r = w * groups + g;
        const int64_t e0 = r < n_rows ? __ldg(row_ptr + r) : 0;
        const int64_t e1 = r < n_rows ? __ldg(row_ptr + r + 1) : 0;
        const unsigned len = (unsigned)(e1 - e0);
        const unsigned maxlen = __reduce_max_sync(0xffffffffu, len);
        for (int64_t t = 0; t * lanes < (int64_t)maxlen; ++t) {
            const int64_t e = e0 + t * lanes + l;
            const bool active = e < e1;
            const int c = warp_distinct(active, active ? (int64_t)__ldg(col + e) : 0, elem_bytes);
            if (lane == 0 && c > 0) atomicAdd(&h[c], 1ull);
        }
    }
    flush_bins(h, hist);
}

// JDS storage, thread per permuted row: a warp holds rows r0..r0+31 and for
// diagonal d reads jd_ptr[d] + r for its rows below diagLen(d).
__global__ void __launch_bounds__(S_THREADS)
    sectors_jds_kernel(int64_t n_rows, int64_t n_diag, const int32_t *__restrict__ jd_ptr,
                       const int32_t *__restrict__ col, int elem_bytes, unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long h[S_BINS];
    for (int i = threadIdx.x; i < S_BINS; i += S_THREADS) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ceil_div_dev(n_rows, 32);
    const int64_t warps_total = (int64_t)gridDim.x * (S_THREADS / 32);
    for (int64_t w = (int64_t)blockIdx.x * (S_THREADS / 32) + (threadIdx.x >> 5); w < n_warps; w += warps_total) {
        const int64_t r0 = w * 32, r = r0 + lane;
        for (int64_t d = 0; d < n_diag; ++d) {
            const int64_t p0 = __ldg(jd_ptr + d), len = (int64_t)__ldg(jd_ptr + d + 1) - p0;
            if (len <= r0) break;
            const bool active = r < len;
            const int c = warp_distinct(active, active ? (int64_t)__ldg(col + p0 + r) : 0, elem_bytes);
            if (lane == 0) atomicAdd(&h[c], 1ull);
        }
    }
    flush_bins(h, hist);
}

// SELL-32: a warp holds one 32-row block; the rows reaching slot d are the
// first lanes (rows are sorted by length inside the block) and read
// consecutive storage.
__global__ void __launch_bounds__(S_THREADS)
    sectors_sell_kernel(int64_t n_rows, const int32_t *__restrict__ rlen, const int32_t *__restrict__ blk_ptr,
                        const int32_t *__restrict__ col, int elem_bytes, unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long h[S_BINS];
    for (int i = threadIdx.x; i < S_BINS; i += S_THREADS) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nb = ceil_div_dev(n_rows, 32);
    const int64_t warps_total = (int64_t)gridDim.x * (S_THREADS / 32);
    for (int64_t b = (int64_t)blockIdx.x * (S_THREADS / 32) + (threadIdx.x >> 5); b < nb; b += warps_total) {
        const int64_t r = b * 32 + lane;
        const int32_t len = r < n_rows ? __ldg(rlen + r) : 0;
        const int32_t width = __shfl_sync(0xffffffffu, len, 0);
        int64_t off = __ldg(blk_ptr + b);
        for (int32_t d = 0; d < width; ++d) {
            const bool active = len > d;
            const int c = warp_distinct(active, active ? (int64_t)__ldg(col + off + lane) : 0, elem_bytes);
            if (lane == 0) atomicAdd(&h[c], 1ull);
            off += __popc(__ballot_sync(0xffffffffu, active));
        }
    }
    flush_bins(h, hist);
}

unsigned grid_for(int64_t items_per_256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(items_per_256, (int64_t)num_sms() * 16));
}

}  // namespace

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_stride_hist(const int32_t *d_col, int64_t nnz, int64_t *d_hist, void *stream) {
    if (nnz < 0 || !d_hist || (nnz > 0 && !d_col)) return arg_error("gbsp_stride_hist: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GBSP_CUDA(cudaMemsetAsync(d_hist, 0, 2 * S_BINS * sizeof(int64_t), s));
    if (nnz > 1) {
        stride_hist_kernel<<<grid_for(ceil_div(nnz, S_THREADS)), S_THREADS, 0, s>>>(
            d_col, nnz, reinterpret_cast<unsigned long long *>(d_hist));
        GBSP_LAUNCH_CHECK("stride_hist_kernel");
    }
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_warp_sectors(gbsp_handle h, int32_t lanes, int32_t elem_bytes, int64_t *d_hist,
                                         void *stream) {
    if (!h || !d_hist) return arg_error("gbsp_warp_sectors: bad arguments");
    if (elem_bytes != 4 && elem_bytes != 8) return arg_error("gbsp_warp_sectors: elem_bytes must be 4 or 8");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(d_hist);
    const Mat &A = *h;
    if (A.kind == KIND_DIA) {
        set_error("gbsp_warp_sectors: a DIA handle reads x contiguously");
        return GBSP_ERR_UNSUPPORTED;
    }
    if (A.kind == KIND_CRS) {
        if (lanes < 1 || lanes > 32 || (lanes & (lanes - 1)))
            return arg_error("gbsp_warp_sectors: CRS lanes must be 1, 2, 4, 8, 16 or 32");
    } else if (A.format == GBSP_RBJDS || A.format == GBSP_SOJDS || A.format == GBSP_PSELL) {
        set_error("gbsp_warp_sectors: RBJDS / SOJDS / PSELL warp patterns are not modelled");
        return GBSP_ERR_UNSUPPORTED;
    }
    GBSP_CUDA(cudaMemsetAsync(d_hist, 0, S_BINS * sizeof(int64_t), s));
    if (A.n_rows == 0) return GBSP_OK;
    if (A.kind == KIND_CRS) {
        const int64_t warps = ceil_div(A.n_rows, 32 / lanes);
        sectors_crs_kernel<<<grid_for(ceil_div(warps, S_THREADS / 32)), S_THREADS, 0, s>>>(
            A.n_rows, A.row_ptr, A.col, lanes, elem_bytes, hist);
    } else if (A.format == GBSP_SELL) {
        sectors_sell_kernel<<<grid_for(ceil_div(ceil_div(A.n_rows, 32), S_THREADS / 32)), S_THREADS, 0, s>>>(
            A.n_rows, A.rlen, A.blk_ptr, A.col, elem_bytes, hist);
    } else {
        sectors_jds_kernel<<<grid_for(ceil_div(ceil_div(A.n_rows, 32), S_THREADS / 32)), S_THREADS, 0, s>>>(
            A.n_rows, A.n_diag, A.jd_ptr, A.col, elem_bytes, hist);
    }
    GBSP_LAUNCH_CHECK("warp sectors kernel");
    return GBSP_OK;
}
