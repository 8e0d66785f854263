// TILED CRS product on GB300: entries streamed into shared memory by bulk
// asynchronous copies, one DFMA per entry with every lane busy.
//
// Why this shape.  On GB300 a warp-wide FP64 FMA occupies the FP64 pipe of
// an SM sub-partition for many cycles, so FP64 SpMVM is limited by the FP64
// pipe almost as much as by HBM: the kernel must issue exactly one FMA per
// stored entry, with all 32 lanes doing useful work, and no extra FP64
// reduction steps.  It must also keep the gathers of x local, because each
// random gather costs a 32-byte L2 sector.
//
// Rows are grouped into tiles by their merge coordinate m(r) = row_ptr[r] + r
// (tile t holds the rows with m(r) in [t*T, (t+1)*T)), so a tile has at most T
// rows and, except possibly its last row, at most T entries.  A persistent CTA
// owns a contiguous range of tiles and walks it in row order, which keeps the
// band structure of x in L1.  Per CTA:
//   producer warp:  for each tile, bulk-copies (cp.async.bulk, mbarrier
//                   completion) the tile's slices of val, col and row_ptr into
//                   one of S shared-memory stages; ragged ends that a 16-byte
//                   bulk copy cannot cover are loaded with plain loads;
//   8 consumer warps, per tile:
//     A. gather x[col] for all staged entries (entry-parallel, many loads in
//        flight) while sorting the tile's rows by length (counting sort);
//     B. thread i sums the i-th longest row from shared memory with an FMA
//        chain -- sorted rows give the lanes of a warp near-equal lengths;
//        rows longer than kShort are summed by whole warps; a last row too
//        long for the stage is summed by all consumers from global memory.
// Every row is summed by a fixed thread in a fixed order: deterministic.
#include <atomic>
#include <algorithm>

#include "accum.cuh"
#include "internal.cuh"
#include "sm100.cuh"

namespace gbsp {

constexpr int kConsumers = 256;            // 8 consumer warps
constexpr int kStreamThreads = kConsumers + 32;  // + 1 producer warp
constexpr int kShort = 63;                 // longest row summed by one thread
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on every wait

template <int VM, int T, int S>
struct StreamSmem {
    typedef typename ValT<VM>::T V;
    V val[S][T + 8];
    int32_t col[S][T + 8];
    int32_t rp[S][T + 8];
    int4 meta[S];
    V xs[T + 4];
    int16_t order[T];
    int32_t cnt[kShort + 1];
    int32_t longl[T / (kShort + 1) + 2];
    int32_t n_long;
    int32_t go;
    int32_t abort;
    Acc<VM> part[kConsumers / 32];
    uint64_t full[S], empty[S];
};

// tile_rows[t] = first row r with row_ptr[r] + r >= t*T (tile_rows[n_tiles] =
// n_rows).  Thread r in [0, n_rows] writes the tiles whose start falls in
// (m(r-1), m(r)], m(n_rows) counting as +infinity.
__global__ void tile_rows_kernel(int64_t n_rows, int64_t n_tiles, int32_t T,
                                 const int32_t *__restrict__ row_ptr, int32_t *tile_rows) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_rows) return;
    const int64_t t_lo = r == 0 ? 0 : ((int64_t)row_ptr[r - 1] + (r - 1)) / T + 1;
    const int64_t t_hi = r == n_rows ? n_tiles : ((int64_t)row_ptr[r] + r) / T;
    for (int64_t t = t_lo; t <= t_hi && t <= n_tiles; ++t) tile_rows[t] = (int32_t)r;
}

// meta[t] = {r0, r1 (or -r1-1 when the last row is read directly), k0,
// end of the staged entries}.
__global__ void tile_meta_kernel(int64_t n_tiles, int32_t T, const int32_t *__restrict__ tile_rows,
                                 const int32_t *__restrict__ row_ptr, int4 *meta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int32_t r0 = tile_rows[t], r1 = tile_rows[t + 1];
    if (r0 == r1) {
        meta[t] = make_int4(r0, r1, 0, 0);
        return;
    }
    const int32_t k0 = row_ptr[r0], kend = row_ptr[r1];
    const bool direct = (int64_t)kend - k0 > T;
    const int32_t kst = direct ? row_ptr[r1 - 1] : kend;
    meta[t] = make_int4(r0, direct ? -r1 - 1 : r1, k0, kst);
}

template <int VM, int T, int S>
__global__ void __launch_bounds__(kStreamThreads)
crs_stream_kernel(int64_t n_tiles, const int4 *__restrict__ tile_meta, int64_t n_rows, int64_t nnz,
                  const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                  const typename ValT<VM>::T *__restrict__ val,
                  const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                  typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate,
                  int32_t *status) {
    typedef typename ValT<VM>::T V;
    typedef StreamSmem<VM, T, S> Sm;
    constexpr int VMASK = 16 / (int)sizeof(V) - 1;  // elements per 16 bytes - 1
    constexpr int PER = T / kConsumers;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    const int64_t G = gridDim.x;
    const int64_t t_begin = n_tiles * blockIdx.x / G, t_end = n_tiles * (blockIdx.x + 1) / G;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (wid == kConsumers / 32) {
        // ------------------------------------------------------ producer --
        if (lane != 0) return;
        int64_t fill = 0;
        bool ok = true;
        int4 m_next = t_begin < t_end ? __ldg(tile_meta + t_begin) : make_int4(0, 0, 0, 0);
        for (int64_t t = t_begin; t < t_end && ok; ++t) {
            const int4 m = m_next;
            if (t + 1 < t_end) m_next = __ldg(tile_meta + t + 1);  // prefetch the next tile's offsets
            const int32_t r1 = m.y < 0 ? -m.y - 1 : m.y;
            if (m.x == r1) continue;  // no row starts in this tile
            const int s = (int)(fill % S);
            if (fill >= S && !mbar_wait_bounded(&sm.empty[s], (uint32_t)((fill / S - 1) & 1), &sm.abort,
                                                kWaitLimitNs)) {
                ok = false;
                break;
            }
            const int32_t r0 = m.x, k0 = m.z, kst = m.w;
            const int32_t rs_end = (m.y < 0 ? r1 - 1 : r1) + 1;  // rp entries [r0, rs_end)
            // The bulk copies start at the 16-byte boundary below each range
            // and end at the one above it when that stays inside the array
            // (the extra elements are never used); only a range that ends in
            // the array's last 16 bytes leaves a ragged end for plain loads.
            const int32_t vlo = k0 & ~VMASK, clo = k0 & ~3, rlo = r0 & ~3;
            const int64_t vup = ((int64_t)kst + VMASK) & ~(int64_t)VMASK;
            const int64_t cup = ((int64_t)kst + 3) & ~(int64_t)3;
            const int64_t rup = ((int64_t)rs_end + 3) & ~(int64_t)3;
            const int32_t vhi = vup <= nnz ? (int32_t)vup : (kst & ~VMASK);
            const int32_t chi = cup <= nnz ? (int32_t)cup : (kst & ~3);
            const int32_t rhi = rup <= n_rows + 1 ? (int32_t)rup : (rs_end & ~3);
            for (int32_t e = max(vhi, k0); e < kst; ++e) sm.val[s][e - vlo] = val[e];
            for (int32_t e = max(chi, k0); e < kst; ++e) sm.col[s][e - clo] = col[e];
            for (int32_t e = max(rhi, r0); e < rs_end; ++e) sm.rp[s][e - rlo] = row_ptr[e];
            sm.meta[s] = m;
            const uint32_t vb = vhi > vlo ? (uint32_t)(vhi - vlo) * sizeof(V) : 0u;
            const uint32_t cb = chi > clo ? (uint32_t)(chi - clo) * 4u : 0u;
            const uint32_t rb = rhi > rlo ? (uint32_t)(rhi - rlo) * 4u : 0u;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&sm.full[s], vb + cb + rb);
            if (vb) bulk_g2s(&sm.val[s][0], val + vlo, vb, &sm.full[s]);
            if (cb) bulk_g2s(&sm.col[s][0], col + clo, cb, &sm.full[s]);
            if (rb) bulk_g2s(&sm.rp[s][0], row_ptr + rlo, rb, &sm.full[s]);
            ++fill;
        }
        if (ok) {
            // sentinel stage: tells the consumers that the range is done
            const int s = (int)(fill % S);
            if (fill < S || mbar_wait_bounded(&sm.empty[s], (uint32_t)((fill / S - 1) & 1), &sm.abort,
                                              kWaitLimitNs)) {
                sm.meta[s] = make_int4(-1, 0, 0, 0);
                mbar_arrive(&sm.full[s]);
                return;
            }
        }
        // abort: report, then give the copies already issued time to land
        sm.abort = 1;
        if (status) atomicExch(status, (int32_t)GBSP_ERR_TIMEOUT);
        for (int64_t f = max((int64_t)0, fill - S); f < fill; ++f)
            mbar_wait_bounded(&sm.full[f % S], (uint32_t)((f / S) & 1), &sm.abort, 100000000ull);
        return;
    }

    // ------------------------------------------------------- consumers --
    for (int64_t it = 0;; ++it) {
        const int s = (int)(it % S);
        const uint32_t par = (uint32_t)((it / S) & 1);
        if (tid == 0) sm.go = mbar_wait_bounded(&sm.full[s], par, &sm.abort, kWaitLimitNs) ? 1 : 0;
        named_barrier(1, kConsumers);
        if (!sm.go) {
            if (tid == 0) {
                sm.abort = 1;
                if (status) atomicExch(status, (int32_t)GBSP_ERR_TIMEOUT);
            }
            break;
        }
        // the phase is complete: this acquire succeeds at once for every thread
        mbar_wait_bounded(&sm.full[s], par, &sm.abort, kWaitLimitNs);
        const int4 m = sm.meta[s];
        if (m.x < 0) break;
        const bool direct = m.y < 0;
        const int32_t r0 = m.x, r1 = direct ? -m.y - 1 : m.y;
        const int32_t k0 = m.z, kst = m.w;
        const int32_t nr = (direct ? r1 - 1 : r1) - r0;  // staged rows
        const int32_t vlo = k0 & ~VMASK, clo = k0 & ~3, roff = r0 - (r0 & ~3);
        const V *vs = sm.val[s];
        const int32_t *cs = sm.col[s];
        const int32_t *rps = sm.rp[s] + roff;  // rps[i] = row_ptr[r0 + i]

        // A. gather x for the staged entries; sort the rows by length
        V xr[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int32_t k = k0 + tid + u * kConsumers;
            xr[u] = k < kst ? ld_vec(x + (int64_t)cs[k - clo] * ldx) : V(0);
        }
        if (tid <= kShort) sm.cnt[tid] = 0;
        if (tid == 0) sm.n_long = 0;
        named_barrier(1, kConsumers);
        int16_t rlen[PER], rtk[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int32_t i = tid + q * kConsumers;
            rlen[q] = -1;
            if (i < nr) {
                const int32_t len = rps[i + 1] - rps[i];
                if (len <= kShort) {
                    rlen[q] = (int16_t)len;
                    rtk[q] = (int16_t)atomicAdd(&sm.cnt[len], 1);
                } else {
                    sm.longl[atomicAdd(&sm.n_long, 1)] = i;
                }
            }
        }
        named_barrier(1, kConsumers);
        if (wid == 0) {
            // exclusive prefix over lengths in decreasing order: lane l owns
            // lengths 63-2l and 62-2l
            const int la = kShort - 2 * lane, lb = la - 1;
            const int32_t ca = sm.cnt[la], cb2 = sm.cnt[lb];
            int32_t incl = ca + cb2;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int32_t t2 = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t2;
            }
            const int32_t excl = incl - ca - cb2;
            sm.cnt[la] = excl;
            sm.cnt[lb] = excl + ca;
        }
        named_barrier(1, kConsumers);
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (rlen[q] >= 0) sm.order[sm.cnt[rlen[q]] + rtk[q]] = (int16_t)(tid + q * kConsumers);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int32_t k = k0 + tid + u * kConsumers;
            if (k < kst) sm.xs[k - k0] = xr[u];
        }
        named_barrier(1, kConsumers);

        // B. rows, longest first: one thread per short row
        const int32_t n_short = nr - sm.n_long;
        for (int32_t j = tid; j < n_short; j += kConsumers) {
            const int32_t i = sm.order[j];
            const int32_t a = rps[i], b = rps[i + 1];
            Acc<VM> acc;
            acc.init();
            for (int32_t k = a; k < b; ++k) acc.add(vs[k - vlo], sm.xs[k - k0]);
            const int64_t r = r0 + i;
            if (accumulate) acc.add_value(y[r * ldy]);
            y[r * ldy] = acc.result();
        }
        // longer staged rows: one warp per row
        for (int32_t l = wid; l < sm.n_long; l += kConsumers / 32) {
            const int32_t i = sm.longl[l];
            const int32_t a = rps[i], b = rps[i + 1];
            Acc<VM> acc;
            acc.init();
            for (int32_t k = a + lane; k < b; k += 32) acc.add(vs[k - vlo], sm.xs[k - k0]);
            group_reduce<32, VM>(acc);
            if (lane == 0) {
                const int64_t r = r0 + i;
                if (accumulate) acc.add_value(y[r * ldy]);
                y[r * ldy] = acc.result();
            }
        }
        // a last row too long for the stage: all consumers, from global memory
        if (direct) {
            const int32_t kend = __ldg(row_ptr + r1);
            Acc<VM> acc;
            acc.init();
            for (int32_t k = kst + tid; k < kend; k += kConsumers)
                acc.add(ld_stream(val + k), ld_vec(x + (int64_t)ld_stream(col + k) * ldx));
            group_reduce<32, VM>(acc);
            if (lane == 0) sm.part[wid] = acc;
            named_barrier(1, kConsumers);
            if (tid == 0) {
                Acc<VM> tot = sm.part[0];
                for (int w = 1; w < kConsumers / 32; ++w) tot.merge(sm.part[w]);
                const int64_t r = r1 - 1;
                if (accumulate) tot.add_value(y[r * ldy]);
                y[r * ldy] = tot.result();
            }
        }
        named_barrier(1, kConsumers);
        if (tid == 0) mbar_arrive(&sm.empty[s]);
    }
}

// ------------------------------------------------------------------ host --

constexpr int kStreamMaxDevices = 64;

static int64_t n_tiles_for(const Mat &A, int32_t tile) { return ceil_div(A.n_rows + A.nnz, tile); }

int64_t crs_tile_table_bytes(const Mat &A, int32_t tile) {
    const int64_t nt = n_tiles_for(A, tile);
    return ((4 * (nt + 1) + 15) / 16) * 16 + 16 * nt;
}

gbsp_status crs_prepare_tiles(Mat &A, int32_t tile, int32_t *table, cudaStream_t s) {
    const int64_t nt = n_tiles_for(A, tile);
    int32_t *tile_rows = table;
    int4 *meta = reinterpret_cast<int4 *>(reinterpret_cast<char *>(table) + ((4 * (nt + 1) + 15) / 16) * 16);
    tile_rows_kernel<<<(unsigned)ceil_div(A.n_rows + 1, 256), 256, 0, s>>>(A.n_rows, nt, tile, A.row_ptr,
                                                                           tile_rows);
    if (nt > 0)
        tile_meta_kernel<<<(unsigned)ceil_div(nt, 256), 256, 0, s>>>(nt, tile, tile_rows, A.row_ptr, meta);
    GBSP_LAUNCH_CHECK("tile table kernels");
    A.tile_rows = tile_rows;
    A.tile_meta = meta;
    A.n_tiles = nt;
    A.tile = tile;
    return GBSP_OK;
}

template <int VM, int T, int S>
static gbsp_status launch_stream_T(const Mat &A, const VecArgs &v, cudaStream_t st) {
    typedef typename ValT<VM>::T V;
    const size_t smem = sizeof(StreamSmem<VM, T, S>);
    // the attribute belongs to the kernel on one device: set it once per
    // device (it is cheap, and allowed during stream capture, so a device
    // index out of the table's range simply sets it on every launch)
    static std::atomic<int> configured[kStreamMaxDevices];
    int dev = 0;
    GBSP_CUDA(cudaGetDevice(&dev));
    const bool tracked = dev >= 0 && dev < kStreamMaxDevices;
    if (!tracked || !configured[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(crs_stream_kernel<VM, T, S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(crs_stream_kernel)");
        if (tracked) configured[dev].store(1);
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crs_stream_kernel<VM, T, S>,
                                                                  kStreamThreads, smem);
    if (e != cudaSuccess) return cuda_status(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(A.n_tiles, (int64_t)num_sms() * per_sm));
    crs_stream_kernel<VM, T, S><<<(unsigned)grid, kStreamThreads, smem, st>>>(
        A.n_tiles, A.tile_meta, A.n_rows, A.nnz, A.row_ptr, A.col, static_cast<const V *>(A.val),
        static_cast<const V *>(v.x), v.ldx, static_cast<V *>(v.y), v.ldy, v.accumulate, A.status);
    return GBSP_OK;
}

template <int VM>
static gbsp_status launch_stream(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (A.tile == 2048) return launch_stream_T<VM, 2048, 2>(A, v, s);
    return launch_stream_T<VM, 1024, 3>(A, v, s);
}

gbsp_status crs_tiled_launch(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (A.n_tiles == 0) return GBSP_OK;
    gbsp_status st;
    if (A.dtype == GBSP_F64) st = launch_stream<VM_F64>(A, v, s);
    else if (A.kopt.accum == GBSP_ACC_COMPENSATED) st = launch_stream<VM_F32C>(A, v, s);
    else st = launch_stream<VM_F32>(A, v, s);
    if (st != GBSP_OK) return st;
    GBSP_LAUNCH_CHECK("crs_stream_kernel");
    return GBSP_OK;
}

}  // namespace gbsp
