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
#include <cuda.h>

#include <mutex>

#include "internal.cuh"
#include "accum.cuh"
#include "sm100.cuh"

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

// IND through the tensor memory accelerator: B seen as a 2-D tensor of
// len_b / 2 rows of two doubles (16 bytes, the least a tensor copy moves),
// and every 32 indices of a warp fetched by eight tile::gather4 copies (four
// rows each) into shared memory, completing on an mbarrier.  Each warp keeps
// T_STAGES chunks of 32 in flight.  The sum per lane runs over its chunks in
// order, then the fixed trees of the other modes.  This is the GB300 path
// that gathers without the L1TEX tag stage: it is what the basic IR
// operation costs when every lane's gather is turned into part of a TMA
// request instead of a load of its own.
constexpr int T_STAGES = 4;
constexpr int T_WARPS = G_THREADS / 32;
constexpr uint64_t T_WAIT_NS = 1000000000ull;  // 1 s bound on one stage's copies

struct __align__(128) GatherSlot {
    double d[16];  // one gather4 fills the first 64 bytes
};

template <int OP>
__global__ void __launch_bounds__(G_THREADS)
    gather_tma_kernel(int64_t n, const double *__restrict__ a, const double *__restrict__ b, int64_t len_b,
                      const int32_t *__restrict__ ind, const __grid_constant__ CUtensorMap tmap,
                      double *__restrict__ partials, int32_t *status) {
    __shared__ GatherSlot slots[T_WARPS][T_STAGES][8];
    __shared__ uint64_t bars[T_WARPS][T_STAGES];
    __shared__ double warp_sums[G_THREADS / 32];
    __shared__ int abort_flag;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) abort_flag = 0;
    if (lane == 0)
        for (int st = 0; st < T_STAGES; ++st) mbar_init(&bars[w][st], 1);
    fence_mbar_init();
    __syncthreads();
    const int64_t rows = len_b / 2;  // tensor rows; an odd last element is read directly
    const int64_t nchunks = (n + 31) / 32;
    const int64_t wg = (int64_t)blockIdx.x * T_WARPS + w, nw = (int64_t)gridDim.x * T_WARPS;
    int32_t idx[T_STAGES];
    uint32_t phase = 0;
    bool bad = false, timed_out = false;
    double s = 0.0;
    auto issue = [&](int64_t c, int st) {
        const int64_t i = c * 32 + lane;
        const int32_t j = i < n ? ld_stream(ind + i) : -1;
        idx[st] = j;
        const int32_t row = (j >= 0 && (int64_t)j < 2 * rows) ? (j >> 1) : 0;
        const int32_t q0 = __shfl_sync(0xffffffffu, row, (4 * lane) & 31);
        const int32_t q1 = __shfl_sync(0xffffffffu, row, (4 * lane + 1) & 31);
        const int32_t q2 = __shfl_sync(0xffffffffu, row, (4 * lane + 2) & 31);
        const int32_t q3 = __shfl_sync(0xffffffffu, row, (4 * lane + 3) & 31);
        fence_proxy_async_smem();  // this stage's earlier reads before the copies overwrite it
        if (lane == 0) mbar_arrive_expect_tx(&bars[w][st], 8 * 64);
        __syncwarp();
        if (lane < 8)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
                "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(&slots[w][st][lane])),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(0), "r"(q0), "r"(q1), "r"(q2), "r"(q3),
                "r"(smem_u32(&bars[w][st]))
                : "memory");
    };
    auto wait = [&](int st) -> bool {
        const bool ok = mbar_wait_bounded(&bars[w][st], (phase >> st) & 1u, &abort_flag, T_WAIT_NS);
        phase ^= 1u << st;
        return ok;
    };
    for (int st = 0; st < T_STAGES; ++st)
        if (wg + (int64_t)st * nw < nchunks) issue(wg + (int64_t)st * nw, st);
    for (int64_t k = 0; wg + k * nw < nchunks; ++k) {
        const int st = (int)(k % T_STAGES);
        if (!wait(st)) {
            // give up: report, then wait (bounded) for this warp's other copies
            timed_out = true;
            if (lane == 0) abort_flag = 1;
            for (int jx = 1; jx < T_STAGES; ++jx)
                if (wg + (k + jx) * nw < nchunks) wait((int)((k + jx) % T_STAGES));
            break;
        }
        const int64_t i = (wg + k * nw) * 32 + lane;
        const int32_t j = idx[st];
        double bv = 0.0;
        if (i < n) {
            if (j >= 0 && (int64_t)j < 2 * rows) bv = slots[w][st][lane >> 2].d[(lane & 3) * 2 + (j & 1)];
            else if (j >= 0 && (int64_t)j < len_b) bv = __ldg(b + j);
            else bad = true;
            s = OP == GBSP_GATHER_ADD ? s + bv : fma(ld_stream(a + i), bv, s);
        }
        __syncwarp();  // every lane has read the stage before it is refilled
        const int64_t cn = wg + (k + T_STAGES) * nw;
        if (cn < nchunks) issue(cn, st);
    }
    if (status) {
        if (timed_out && lane == 0) atomicExch(status, (int32_t)GBSP_ERR_TIMEOUT);
        else if (bad) *status = (int32_t)GBSP_ERR_ARG;
    }
    const double t = block_sum(s, warp_sums);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Every CTA (one per SM) reads all of B once into shared memory: thread 0
// streams it in SW_CHUNK-byte bulk copies (cp.async.bulk) through a ring of
// SW_BUFS buffers, so SW_BUFS * SW_CHUNK bytes are in flight per SM, and the
// CTA waits for each chunk before the buffer is reused.  Its time is what a
// column-panel design for uniformly random indices costs at least: each SM
// needs every panel of B, so B crosses from L2 to each SM once per product.
// out[blockIdx.x] = the sum of the first double of every chunk (keeps the
// copies live and gives the test a closed form).
constexpr int SW_BUFS = 4;
constexpr int SW_CHUNK = 32768;
constexpr uint64_t SW_WAIT_NS = 1000000000ull;

__global__ void __launch_bounds__(256) stage_sweep_kernel(const double *__restrict__ b, int64_t len_b,
                                                          double *__restrict__ out, int32_t *status) {
    extern __shared__ __align__(128) unsigned char sw_smem[];
    __shared__ uint64_t bars[SW_BUFS];
    __shared__ int abort_flag;
    const int64_t bytes = len_b * 8;
    const int64_t whole = bytes / 16 * 16;  // the bulk copies move 16-byte multiples
    const int64_t nchunks = (whole + SW_CHUNK - 1) / SW_CHUNK;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int q = 0; q < SW_BUFS; ++q) mbar_init(&bars[q], 1);
    }
    fence_mbar_init();
    __syncthreads();
    auto issue = [&](int64_t c) {
        const int q = (int)(c % SW_BUFS);
        const uint32_t nb = (uint32_t)min((int64_t)SW_CHUNK, whole - c * SW_CHUNK);
        mbar_arrive_expect_tx(&bars[q], nb);
        bulk_g2s(sw_smem + q * SW_CHUNK, reinterpret_cast<const char *>(b) + c * SW_CHUNK, nb, &bars[q]);
    };
    if (threadIdx.x == 0)
        for (int64_t c = 0; c < SW_BUFS && c < nchunks; ++c) issue(c);
    double s = 0.0;
    bool ok = true;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int q = (int)(c % SW_BUFS);
        const uint32_t parity = (uint32_t)((c / SW_BUFS) & 1);
        if (ok && !mbar_wait_bounded(&bars[q], parity, &abort_flag, SW_WAIT_NS)) {
            ok = false;
            abort_flag = 1;
        }
        if (threadIdx.x == 0 && ok) s += reinterpret_cast<const double *>(sw_smem + q * SW_CHUNK)[0];
        __syncthreads();  // every thread is past chunk c before its buffer is refilled
        if (!ok || abort_flag) {
            // give up: report, then wait (bounded) for the copies still in flight
            if (threadIdx.x == 0) {
                if (status) atomicExch(status, (int32_t)GBSP_ERR_TIMEOUT);
                for (int64_t c2 = c; c2 < c + SW_BUFS && c2 < nchunks; ++c2)
                    mbar_wait_bounded(&bars[c2 % SW_BUFS], (uint32_t)((c2 / SW_BUFS) & 1), &abort_flag, SW_WAIT_NS);
            }
            break;
        }
        if (threadIdx.x == 0 && c + SW_BUFS < nchunks) {
            fence_proxy_async_smem();
            issue(c + SW_BUFS);
        }
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry-point lookup
// (the library links only the CUDA runtime); NULL when unavailable.
EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
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
    if (access != GBSP_ACCESS_PD && access != GBSP_ACCESS_CS && access != GBSP_ACCESS_IND &&
        access != GBSP_ACCESS_IND_TMA)
        return arg_error("gbsp_gather_sum: unknown access");
    if (n < 0 || len_b < 0 || !d_out || !d_partials) return arg_error("gbsp_gather_sum: bad sizes or NULL output");
    if (n > 0) {
        if (!d_b) return arg_error("gbsp_gather_sum: NULL B");
        if (op == GBSP_GATHER_SCP && !d_a) return arg_error("gbsp_gather_sum: NULL A for SCP");
        if ((access == GBSP_ACCESS_IND || access == GBSP_ACCESS_IND_TMA) && !d_ind)
            return arg_error("gbsp_gather_sum: NULL index array");
        if (access == GBSP_ACCESS_IND_TMA) {
            if (len_b < 2) return arg_error("gbsp_gather_sum: IND_TMA needs len_b >= 2");
            if (len_b / 2 > INT32_MAX) return arg_error("gbsp_gather_sum: IND_TMA needs len_b / 2 < 2^31");
            if (reinterpret_cast<uintptr_t>(d_b) & 15) return arg_error("gbsp_gather_sum: IND_TMA needs B 16-byte aligned");
        }
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
    if (n > 0 && access == GBSP_ACCESS_IND_TMA) {
        EncodeTiledFn enc = encode_tiled();
        if (!enc) {
            set_error("gbsp_gather_sum: cuTensorMapEncodeTiled is not available from the driver");
            return GBSP_ERR_UNSUPPORTED;
        }
        CUtensorMap tm;
        const cuuint64_t dims[2] = {2, (cuuint64_t)(len_b / 2)};
        const cuuint64_t strides[1] = {16};
        const cuuint32_t box[2] = {2, 1};  // gather4: one row per coordinate, 16 bytes
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(d_b), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error("gbsp_gather_sum: cuTensorMapEncodeTiled failed (%d)", (int)r);
            return GBSP_ERR_CUDA;
        }
        if (op == GBSP_GATHER_ADD)
            gather_tma_kernel<GBSP_GATHER_ADD><<<grid, G_THREADS, 0, s>>>(n, d_a, d_b, len_b, d_ind, tm, d_partials,
                                                                          d_status);
        else
            gather_tma_kernel<GBSP_GATHER_SCP><<<grid, G_THREADS, 0, s>>>(n, d_a, d_b, len_b, d_ind, tm, d_partials,
                                                                          d_status);
        GBSP_LAUNCH_CHECK("gather_tma_kernel");
    } else if (n > 0) {
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

extern "C" gbsp_status gbsp_stage_sweep(const double *d_b, int64_t len_b, double *d_out, int32_t n_out,
                                        int32_t *d_status, void *stream) {
    if (len_b < 0 || !d_out) return arg_error("gbsp_stage_sweep: bad arguments");
    if (len_b > 0 && !d_b) return arg_error("gbsp_stage_sweep: NULL B");
    if (reinterpret_cast<uintptr_t>(d_b) & 15) return arg_error("gbsp_stage_sweep: B must be 16-byte aligned");
    const int grid = num_sms();
    if (n_out < grid) return arg_error("gbsp_stage_sweep: out needs one double per SM");
    const int smem = SW_BUFS * SW_CHUNK;
    // the attribute belongs to the kernel on one device: set it on every
    // call (cheap; a per-device flag would need the device-index table)
    GBSP_CUDA(cudaFuncSetAttribute(stage_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    stage_sweep_kernel<<<grid, 256, smem, static_cast<cudaStream_t>(stream)>>>(d_b, len_b, d_out, d_status);
    GBSP_LAUNCH_CHECK("stage_sweep_kernel");
    return GBSP_OK;
}
