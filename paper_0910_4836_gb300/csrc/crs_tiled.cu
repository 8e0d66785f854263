// TILED CRS product: load-balanced tiles of rows, entries staged through
// shared memory.
//
// Rows are grouped by their merge coordinate m(r) = row_ptr[r] + r (rows +
// entries before row r, strictly increasing): tile t holds the rows with
// m(r) in [t*T, (t+1)*T).  A tile therefore has at most T rows, and every
// row of it except the last has fewer than T entries; only the last row of
// a tile can be long.  The tile table (first row of every tile) is a pure
// function of row_ptr, built once by tile_table_kernel.
//
// One CTA per tile:
//   1. stream: every thread loads entries k0+tid, k0+tid+256, ... of the
//      tile's contiguous entry range (coalesced, evict-first), gathers x and
//      stores the product in shared memory; all loads of a thread are issued
//      before the gathers, so ~T*12 bytes per CTA are in flight;
//   2. reduce: thread i sums row i of the tile from shared memory (rows up to
//      kShortRow entries); longer rows are summed by whole warps;
//   3. a last row longer than the staging buffer is summed by the whole CTA
//      straight from global memory (coalesced) with a block reduction.
// Sums are formed in a fixed order, so results are deterministic.
#include <algorithm>

#include "accum.cuh"
#include "internal.cuh"

namespace gbsp {

constexpr int kTileThreads = 256;
constexpr int kShortRow = 32;

template <int VM> struct Prod { typedef typename ValT<VM>::T T; T p; };
template <> struct Prod<VM_F32C> { float p, e; };

template <int VM>
__device__ __forceinline__ Prod<VM> make_prod(typename ValT<VM>::T a, typename ValT<VM>::T x) {
    Prod<VM> q;
    q.p = a * x;
    return q;
}
template <>
__device__ __forceinline__ Prod<VM_F32C> make_prod<VM_F32C>(float a, float x) {
    Prod<VM_F32C> q;
    q.p = a * x;
    q.e = fmaf(a, x, -q.p);
    return q;
}

template <int VM>
__device__ __forceinline__ void acc_prod(Acc<VM> &a, const Prod<VM> &q) { a.add_value(q.p); }
template <>
__device__ __forceinline__ void acc_prod<VM_F32C>(Acc<VM_F32C> &a, const Prod<VM_F32C> &q) {
    float t;
    two_sum(a.s, q.p, a.s, t);
    a.c += t + q.e;
}

// tile_rows[t] = first row r with row_ptr[r] + r >= t*T; tile_rows[n_tiles]
// = n_rows.  Thread r in [0, n_rows] writes the tiles whose start falls in
// (m(r-1), m(r)], m(n_rows) counting as +infinity.
__global__ void tile_table_kernel(int64_t n_rows, int64_t n_tiles, int32_t T,
                                  const int32_t *__restrict__ row_ptr, int32_t *tile_rows) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n_rows) return;
    const int64_t t_lo = r == 0 ? 0 : ((int64_t)row_ptr[r - 1] + (r - 1)) / T + 1;
    const int64_t t_hi = r == n_rows ? n_tiles : ((int64_t)row_ptr[r] + r) / T;
    for (int64_t t = t_lo; t <= t_hi && t <= n_tiles; ++t) tile_rows[t] = (int32_t)r;
}

template <int VM, int T_ITEMS>
__global__ void __launch_bounds__(kTileThreads)
crs_tiled_kernel(int64_t n_tiles, const int32_t *__restrict__ tile_rows,
                 const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                 const typename ValT<VM>::T *__restrict__ val,
                 const typename ValT<VM>::T *__restrict__ x, int64_t ldx,
                 typename ValT<VM>::T *__restrict__ y, int64_t ldy, int accumulate) {
    typedef typename ValT<VM>::T T;
    constexpr int PER = T_ITEMS / kTileThreads;
    __shared__ Prod<VM> prod[T_ITEMS];
    __shared__ int32_t rp[T_ITEMS + 1];
    __shared__ int32_t long_rows[T_ITEMS / kShortRow + 1];
    __shared__ int32_t n_long;
    __shared__ Acc<VM> warp_part[kTileThreads / 32];

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int32_t r0 = __ldg(tile_rows + t), r1 = __ldg(tile_rows + t + 1);
        if (r0 == r1) continue;
        const int32_t nrows = r1 - r0;
        const int32_t k0 = __ldg(row_ptr + r0);
        const int32_t klast = __ldg(row_ptr + r1 - 1);
        const int32_t kend = __ldg(row_ptr + r1);
        // the staged range: all rows, or all but a last row that does not fit
        const bool last_direct = (kend - k0) > T_ITEMS;
        const int32_t kstage = last_direct ? klast : kend;
        const int32_t nstage_rows = last_direct ? nrows - 1 : nrows;
        if (tid == 0) n_long = 0;
        for (int i = tid; i <= nstage_rows; i += kTileThreads) rp[i] = __ldg(row_ptr + r0 + i) - k0;

        // 1. stream entries and gather x
        {
            int c[PER];
            T v[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int32_t k = k0 + tid + u * kTileThreads;
                const bool ok = k < kstage;
                c[u] = ok ? ld_stream(col + k) : 0;
                v[u] = ok ? ld_stream(val + k) : T(0);
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int32_t k = k0 + tid + u * kTileThreads;
                if (k < kstage) prod[k - k0] = make_prod<VM>(v[u], ld_vec(x + (int64_t)c[u] * ldx));
            }
        }
        __syncthreads();

        // 2a. short rows: one thread per row
        for (int i = tid; i < nstage_rows; i += kTileThreads) {
            const int32_t a = rp[i], b = rp[i + 1];
            if (b - a > kShortRow) {
                const int slot = atomicAdd(&n_long, 1);
                long_rows[slot] = i;
                continue;
            }
            Acc<VM> acc;
            acc.init();
            for (int32_t j = a; j < b; ++j) acc_prod<VM>(acc, prod[j]);
            const int64_t r = r0 + i;
            if (accumulate) acc.add_value(y[r * ldy]);
            y[r * ldy] = acc.result();
        }
        __syncthreads();
        // 2b. longer staged rows: one warp per row
        for (int l = wid; l < n_long; l += kTileThreads / 32) {
            const int i = long_rows[l];
            const int32_t a = rp[i], b = rp[i + 1];
            Acc<VM> acc;
            acc.init();
            for (int32_t j = a + lane; j < b; j += 32) acc_prod<VM>(acc, prod[j]);
            group_reduce<32, VM>(acc);
            if (lane == 0) {
                const int64_t r = r0 + i;
                if (accumulate) acc.add_value(y[r * ldy]);
                y[r * ldy] = acc.result();
            }
        }
        // 3. a last row too long to stage: the whole CTA from global memory
        if (last_direct) {
            Acc<VM> acc;
            acc.init();
            for (int32_t k = klast + tid; k < kend; k += kTileThreads)
                acc.add(ld_stream(val + k), ld_vec(x + (int64_t)ld_stream(col + k) * ldx));
            group_reduce<32, VM>(acc);
            if (lane == 0) warp_part[wid] = acc;
            __syncthreads();
            if (tid == 0) {
                Acc<VM> tot = warp_part[0];
                for (int w = 1; w < kTileThreads / 32; ++w) tot.merge(warp_part[w]);
                const int64_t r = r1 - 1;
                if (accumulate) tot.add_value(y[r * ldy]);
                y[r * ldy] = tot.result();
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host --

gbsp_status crs_prepare_tiles(Mat &A, int32_t tile, int32_t *table, cudaStream_t s) {
    const int64_t n_tiles = ceil_div(A.n_rows + A.nnz, tile);
    const int64_t threads = A.n_rows + 1;
    tile_table_kernel<<<(unsigned)ceil_div(threads, 256), 256, 0, s>>>(A.n_rows, n_tiles, tile,
                                                                      A.row_ptr, table);
    GBSP_LAUNCH_CHECK("tile_table_kernel");
    A.tile_rows = table;
    A.n_tiles = n_tiles;
    A.tile = tile;
    return GBSP_OK;
}

template <int VM, int TI>
static void launch_tiled_T(const Mat &A, const VecArgs &v, cudaStream_t s) {
    typedef typename ValT<VM>::T T;
    const int64_t cap = (int64_t)num_sms() * 64;  // eight waves of eight CTAs per SM
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(A.n_tiles, cap));
    crs_tiled_kernel<VM, TI><<<grid, kTileThreads, 0, s>>>(
        A.n_tiles, A.tile_rows, A.row_ptr, A.col, static_cast<const T *>(A.val),
        static_cast<const T *>(v.x), v.ldx, static_cast<T *>(v.y), v.ldy, v.accumulate);
}

template <int VM>
static void launch_tiled(const Mat &A, const VecArgs &v, cudaStream_t s) {
    switch (A.tile) {
        case 512: launch_tiled_T<VM, 512>(A, v, s); break;
        case 1024: launch_tiled_T<VM, 1024>(A, v, s); break;
        default: launch_tiled_T<VM, 2048>(A, v, s); break;
    }
}

gbsp_status crs_tiled_launch(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (A.dtype == GBSP_F64) launch_tiled<VM_F64>(A, v, s);
    else if (A.kopt.accum == GBSP_ACC_COMPENSATED) launch_tiled<VM_F32C>(A, v, s);
    else launch_tiled<VM_F32>(A, v, s);
    GBSP_LAUNCH_CHECK("crs_tiled_kernel");
    return GBSP_OK;
}

}  // namespace gbsp
