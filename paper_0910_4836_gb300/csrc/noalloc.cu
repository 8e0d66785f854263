// One-call CRS product that allocates nothing.
//
// The TILED kernel needs a tile table (the first row and the entry offsets
// of every tile) in device memory.  gbsp_crs_prepare puts it in caller
// memory; this entry point instead builds it, on every call, in a fixed
// array of device memory that is part of the library image, so a caller
// passes only the matrix, x and y.
#include <mutex>

#include "internal.cuh"

namespace gbsp {

// 8 MiB of tile table per GPU that loads the library, enough for
// (n_rows + nnz) up to about 4.1e8 with 1024-item tiles.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int32_t kNoAllocTile = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
// per device: the context the address was looked up in, and the address
static void *g_noalloc_ctx[kMaxDevices] = {nullptr};
static void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// cuCtxGetCurrent through the runtime's driver entry-point lookup (the
// library links only the CUDA runtime).  NULL if the lookup failed.
typedef int (*CtxGetCurrentFn)(void **);
static CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(f);
    }
    return fn;
}

// Device address of the scratch array in the current context.  The
// host-side name of a __device__ array is only a stand-in, so the address
// comes from cudaGetSymbolAddress, with the device current.  It is looked up
// again whenever the device's current context differs from the one it was
// looked up in (the module can load at another address after a device reset
// or a new primary context); if the context cannot be identified, on every
// call.
static gbsp_status noalloc_scratch(void **out) {
    int dev = 0;
    GBSP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return arg_error("gbsp_crs_spmv_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    CtxGetCurrentFn get = ctx_get_current();
    void *ctx = nullptr;
    bool known = get != nullptr && get(&ctx) == 0 && ctx != nullptr;
    if (!known || !g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
        void *p = nullptr;
        // also makes the runtime's context of this device current, if none was
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(noalloc scratch)");
        ctx = nullptr;
        known = get != nullptr && get(&ctx) == 0 && ctx != nullptr;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = known ? ctx : nullptr;
    }
    *out = g_noalloc_ptr[dev];
    return GBSP_OK;
}

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_crs_spmv_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                             const int32_t *d_row_ptr, const int32_t *d_col,
                                             const void *d_val, gbsp_dtype dtype, int32_t accumulate,
                                             const void *d_x, void *d_y, void *stream) {
    if (n_rows < 0 || n_cols < 0 || nnz < 0) return arg_error("gbsp_crs_spmv_noalloc: negative size");
    if (nnz >= (int64_t(1) << 31) - (int64_t(1) << 16) || n_rows >= (int64_t(1) << 31) - 1 ||
        n_cols >= (int64_t(1) << 31) - 1)
        return arg_error("gbsp_crs_spmv_noalloc: sizes must fit int32 indices");
    if (dtype != GBSP_F64 && dtype != GBSP_F32) return arg_error("gbsp_crs_spmv_noalloc: bad dtype");
    if (!d_row_ptr || (nnz > 0 && (!d_col || !d_val)) || (n_rows > 0 && !d_y) || (n_cols > 0 && !d_x))
        return arg_error("gbsp_crs_spmv_noalloc: NULL array");
    const uintptr_t es = dtype == GBSP_F64 ? 8 : 4;
    if ((reinterpret_cast<uintptr_t>(d_row_ptr) & 15) || (reinterpret_cast<uintptr_t>(d_col) & 15) ||
        (reinterpret_cast<uintptr_t>(d_val) & 15))
        return arg_error("gbsp_crs_spmv_noalloc: row_ptr, col and val must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(d_x) & (es - 1)) || (reinterpret_cast<uintptr_t>(d_y) & (es - 1)))
        return arg_error("gbsp_crs_spmv_noalloc: misaligned x or y");
    {
        const char *x0 = static_cast<const char *>(d_x), *y0 = static_cast<const char *>(d_y);
        const size_t xb = (size_t)n_cols * es, yb = (size_t)n_rows * es;
        if (xb && yb && x0 < y0 + yb && y0 < x0 + xb) return arg_error("gbsp_crs_spmv_noalloc: x and y overlap");
    }
    Mat A;
    A.kind = KIND_CRS;
    A.n_rows = n_rows;
    A.n_cols = n_cols;
    A.nnz = nnz;
    A.dtype = dtype;
    A.row_ptr = d_row_ptr;
    A.col = d_col;
    A.val = d_val;
    crs_default_opts(A);
    const int64_t need = crs_tile_table_bytes(A, kNoAllocTile);
    if (need > (int64_t)kNoAllocScratchBytes) {
        set_error("gbsp_crs_spmv_noalloc: n_rows + nnz = %lld needs a %lld-byte tile table, more than the "
                  "%lld-byte static scratch; use gbsp_crs_prepare with caller memory",
                  (long long)(n_rows + nnz), (long long)need, (long long)kNoAllocScratchBytes);
        return GBSP_ERR_ARG;
    }
    if (n_rows == 0) return GBSP_OK;
    void *scratch = nullptr;
    gbsp_status st = noalloc_scratch(&scratch);
    if (st != GBSP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // every table entry is rewritten here, so earlier contents do not matter
    st = crs_prepare_tiles(A, kNoAllocTile, static_cast<int32_t *>(scratch), s);
    if (st != GBSP_OK) return st;
    A.kopt.kernel = GBSP_KERNEL_TILED;
    VecArgs v{};
    v.x = d_x;
    v.y = d_y;
    v.ldx = 1;
    v.ldy = 1;
    v.k = 1;
    v.accumulate = accumulate ? 1 : 0;
    return crs_tiled_launch(A, v, s);
}
