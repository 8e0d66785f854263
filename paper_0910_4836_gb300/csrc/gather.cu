// Basic sparse vector operations (Sect. 4.1, the table of ADD and SCP
// kernels): one sum over i < n of B(idx(i)) (ADD) or A(i) * B(idx(i)) (SCP),
// where idx(i) = i (PD, packed dense), k * i (CS, constant stride computed in
// the loop) or ind(i) (IS / IR, read from an index array).  The paper uses
// them to separate the cost of the x gather from the rest of the SpMVM
// inner loop; here they measure the same thing on GB300, where the unit of
// waste is the 32-byte L2 sector rather than the 64-byte cache line.
//
// Kernel shape: a grid-stride loop with U independent loads in flight per
// thread (lane i of a warp takes element i, so PD, the index array and A are
// read coalesced), a fixed-order sum per thread, a fixed shuffle tree per
// warp and a fixed-order sum over the warps of a CTA into one partial per
// CTA; a one-CTA kernel then sums the partials in a fixed order.  The result
// is the same on every run for a given grid.
#include "internal.cuh"
#include "accum.cuh"

namespace gbsp {

namespace {

constexpr int G_THREADS = 256;
constexpr int G_UNROLL = 8;
constexpr int G_CTAS_PER_SM = 8;

__device__ __forceinline__ double block_sum(double s, double *warp_sums) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) warp_sums[warp] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_sums[w];
    return t;  // meaningful in thread 0 only
}

template <int OP, int ACCESS>
__device__ __forceinline__ int64_t gather_index(int64_t i, int64_t k, const int32_t *__restrict__ ind) {
    if (ACCESS == GBSP_ACCESS_PD) return i;
    if (ACCESS == GBSP_ACCESS_CS) return k * i;
    return (int64_t)ld_stream(ind + i);
}

template <int OP, int ACCESS>
__global__ void __launch_bounds__(G_THREADS)
    gather_sum_kernel(int64_t n, int64_t k, const double *__restrict__ a, const double *__restrict__ b,
                      int64_t len_b, const int32_t *__restrict__ ind, double *__restrict__ partials,
                      int32_t *status) {
    __shared__ double warp_sums[G_THREADS / 32];
    const int64_t T = (int64_t)gridDim.x * G_THREADS;
    int64_t i = (int64_t)blockIdx.x * G_THREADS + threadIdx.x;
    double s = 0.0;
    bool bad = false;
    // U elements per thread per step: indices first, then the loads, then the
    // adds in ascending i
    for (; i + (int64_t)(G_UNROLL - 1) * T < n; i += (int64_t)G_UNROLL * T) {
        int64_t j[G_UNROLL];
        double av[G_UNROLL], bv[G_UNROLL];
#pragma unroll
        for (int u = 0; u < G_UNROLL; ++u) j[u] = gather_index<OP, ACCESS>(i + u * T, k, ind);
#pragma unroll
        for (int u = 0; u < G_UNROLL; ++u) {
            // PD and CS ranges are checked on the host; the index array here
            const bool ok = ACCESS != GBSP_ACCESS_IND || (uint64_t)j[u] < (uint64_t)len_b;
            bad |= !ok;
            bv[u] = ok ? __ldg(b + j[u]) : 0.0;
            av[u] = OP == GBSP_GATHER_SCP ? ld_stream(a + i + u * T) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < G_UNROLL; ++u) s = OP == GBSP_GATHER_ADD ? s + bv[u] : fma(av[u], bv[u], s);
    }
    for (; i < n; i += T) {
        const int64_t j = gather_index<OP, ACCESS>(i, k, ind);
        const bool ok = ACCESS != GBSP_ACCESS_IND || (uint64_t)j < (uint64_t)len_b;
        bad |= !ok;
        const double bv = ok ? __ldg(b + j) : 0.0;
        s = OP == GBSP_GATHER_ADD ? s + bv : fma(ld_stream(a + i), bv, s);
    }
    if (bad && status) *status = (int32_t)GBSP_ERR_ARG;
    const double t = block_sum(s, warp_sums);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(G_THREADS)
    gather_final_kernel(const double *__restrict__ partials, int32_t count, double *__restrict__ out) {
    __shared__ double warp_sums[G_THREADS / 32];
    double s = 0.0;
    for (int32_t p = threadIdx.x; p < count; p += G_THREADS) s += partials[p];
    const double t = block_sum(s, warp_sums);
    if (threadIdx.x == 0) *out = t;
}

int32_t gather_grid(int64_t n) {
    const int64_t per_cta = (int64_t)G_THREADS * G_UNROLL;
    return (int32_t)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, per_cta), (int64_t)num_sms() * G_CTAS_PER_SM));
}

template <int OP>
void launch_gather(int32_t access, int32_t grid, int64_t n, int64_t k, const double *a, const double *b,
                   int64_t len_b, const int32_t *ind, double *partials, int32_t *status, cudaStream_t s) {
    switch (access) {
        case GBSP_ACCESS_PD:
            gather_sum_kernel<OP, GBSP_ACCESS_PD><<<grid, G_THREADS, 0, s>>>(n, k, a, b, len_b, ind, partials, status);
            break;
        case GBSP_ACCESS_CS:
            gather_sum_kernel<OP, GBSP_ACCESS_CS><<<grid, G_THREADS, 0, s>>>(n, k, a, b, len_b, ind, partials, status);
            break;
        default:
            gather_sum_kernel<OP, GBSP_ACCESS_IND><<<grid, G_THREADS, 0, s>>>(n, k, a, b, len_b, ind, partials, status);
            break;
    }
}

// FP64 FMA issue rate.  The paper compares SpMVM against each machine's
// peak Flop rate as well as its memory bandwidth; on GB300 the FP64 rate is
// low enough to be a second roofline, so it is measured, not assumed.  Each
// thread runs F independent chains x <- fma(x, a, b) for `iters` steps
// (independent, so the pipe, not latency, is the limit).  Lanes at or above
// `active` skip the loop: the FMAs of their warp still issue, so the time of
// a launch shows what an idle lane costs.  out[t] = the sum of the thread's
// chains in a fixed order (0 for skipped lanes).
constexpr int F_CHAINS = 8;

__global__ void __launch_bounds__(G_THREADS)
    fma_chain_kernel(int64_t n, int32_t active, int32_t iters, const double *__restrict__ in,
                     double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * G_THREADS + threadIdx.x;
    if (t >= n) return;
    const double a = __ldg(in + 1), b = __ldg(in + 2);
    double x[F_CHAINS];
#pragma unroll
    for (int j = 0; j < F_CHAINS; ++j) x[j] = __ldg(in) + (double)j;
    double s = 0.0;
    if ((int)(threadIdx.x & 31) < active) {
        for (int32_t k = 0; k < iters; ++k) {
#pragma unroll
            for (int j = 0; j < F_CHAINS; ++j) x[j] = fma(x[j], a, b);
        }
#pragma unroll
        for (int j = 0; j < F_CHAINS; ++j) s += x[j];
    }
    out[t] = s;
}

}  // namespace

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_gather_partials(int64_t n, int32_t *n_partials) {
    if (n < 0 || !n_partials) return arg_error("gbsp_gather_partials: bad arguments");
    *n_partials = gather_grid(n);
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_gather_sum(int32_t op, int32_t access, int64_t n, int64_t stride,
                                       const double *d_a, const double *d_b, int64_t len_b,
                                       const int32_t *d_ind, double *d_partials, int32_t n_partials,
                                       double *d_out, int32_t *d_status, void *stream) {
    if (op != GBSP_GATHER_ADD && op != GBSP_GATHER_SCP) return arg_error("gbsp_gather_sum: unknown op");
    if (access != GBSP_ACCESS_PD && access != GBSP_ACCESS_CS && access != GBSP_ACCESS_IND)
        return arg_error("gbsp_gather_sum: unknown access");
    if (n < 0 || len_b < 0 || !d_out || !d_partials) return arg_error("gbsp_gather_sum: bad sizes or NULL output");
    if (n > 0) {
        if (!d_b) return arg_error("gbsp_gather_sum: NULL B");
        if (op == GBSP_GATHER_SCP && !d_a) return arg_error("gbsp_gather_sum: NULL A for SCP");
        if (access == GBSP_ACCESS_IND && !d_ind) return arg_error("gbsp_gather_sum: NULL index array");
        if (access == GBSP_ACCESS_PD && n > len_b) return arg_error("gbsp_gather_sum: n exceeds len_b");
        if (access == GBSP_ACCESS_CS) {
            if (stride < 1) return arg_error("gbsp_gather_sum: stride must be >= 1");
            if ((n - 1) > (INT64_MAX / stride) || (n - 1) * stride >= len_b)
                return arg_error("gbsp_gather_sum: (n-1)*stride exceeds len_b");
        }
    }
    const int32_t grid = gather_grid(n);
    if (n_partials < grid) return arg_error("gbsp_gather_sum: partials buffer smaller than gbsp_gather_partials");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0) {
        if (op == GBSP_GATHER_ADD)
            launch_gather<GBSP_GATHER_ADD>(access, grid, n, stride, d_a, d_b, len_b, d_ind, d_partials, d_status, s);
        else
            launch_gather<GBSP_GATHER_SCP>(access, grid, n, stride, d_a, d_b, len_b, d_ind, d_partials, d_status, s);
        GBSP_LAUNCH_CHECK("gather_sum_kernel");
    }
    gather_final_kernel<<<1, G_THREADS, 0, s>>>(d_partials, n > 0 ? grid : 0, d_out);
    GBSP_LAUNCH_CHECK("gather_final_kernel");
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_fma_chain(int64_t n_threads, int32_t active_lanes, int32_t iters, const double *d_in,
                                      double *d_out, void *stream) {
    if (n_threads < 0 || active_lanes < 0 || active_lanes > 32 || iters < 0)
        return arg_error("gbsp_fma_chain: bad sizes");
    if (n_threads == 0) return GBSP_OK;
    if (!d_in || !d_out) return arg_error("gbsp_fma_chain: NULL pointer");
    const int64_t grid = ceil_div(n_threads, G_THREADS);
    if (grid > INT32_MAX) return arg_error("gbsp_fma_chain: too many threads");
    fma_chain_kernel<<<(unsigned)grid, G_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        n_threads, active_lanes, iters, d_in, d_out);
    GBSP_LAUNCH_CHECK("fma_chain_kernel");
    return GBSP_OK;
}
