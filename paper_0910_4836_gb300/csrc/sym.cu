// Symmetric SpMVM from one triangle.  Sect. 4.2 notes that the Hamiltonian
// is symmetric, which would allow a further saving of data transfer, and
// does not pursue it.  Here the stored entries S (the upper triangle of a
// symmetric A: col >= row) are read once and applied twice:
//     y = (S + S^T - diag S) x,
// each off-diagonal s_ij adding s_ij x_j to y_i and s_ij x_i to y_j.  The
// second update lands on another thread's row, so every update of y is an
// FP64 atomic add at L2 (y must be zeroed first, or hold the value to add
// to).  The order of those adds varies from run to run: the result is not
// bit-reproducible (it is exact whenever every partial sum is, e.g. integer
// data), unlike every other product of this library.
//
// Two walks: CRS (thread per row) and SELL-32-sigma with the row-only
// permutation (warp per 32-row block, rows permuted inside windows; the
// stored columns are original indices, row r of the layout is original row
// perm[r]).
#include "internal.cuh"
#include "accum.cuh"

namespace gbsp {

namespace {

__device__ __forceinline__ void red_add(double *p, double v) { atomicAdd(p, v); }

// entries with col >= row, per row
__global__ void upper_count_kernel(int64_t n, const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, int32_t *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) c += col[e] >= i;
    cnt[i] = c;
}

template <typename T>
__global__ void upper_fill_kernel(int64_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                  const T *__restrict__ val, const int32_t *__restrict__ row_ptr_u,
                                  int32_t *col_u, T *val_u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t pos = row_ptr_u[i];
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
        if (col[e] >= i) {
            col_u[pos] = col[e];
            val_u[pos] = val[e];
            ++pos;
        }
}

// CRS walk: thread per stored row i, U entries per step.
template <int U>
__global__ void __launch_bounds__(256) sym_crs_kernel(int64_t n, const int32_t *__restrict__ row_ptr,
                                                      const int32_t *__restrict__ col,
                                                      const double *__restrict__ val,
                                                      const double *__restrict__ x, double *y) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) {
        const double xi = __ldg(x + i);
        const int64_t e1 = __ldg(row_ptr + i + 1);
        double s = 0.0;
        for (int64_t e = __ldg(row_ptr + i); e < e1; e += U) {
            int32_t c[U];
            double v[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = e + j < e1;
                c[j] = ok ? ld_stream(col + e + j) : -1;
                v[j] = ok ? ld_stream(val + e + j) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (c[j] < 0) continue;
                s = fma(v[j], __ldg(x + c[j]), s);
                if (c[j] != i) red_add(y + c[j], v[j] * xi);
            }
        }
        red_add(y + i, s);
    }
}

// SELL-32-sigma walk (row-only permutation): the block layout of the SELL
// product kernel, each stored entry applied to both of its rows.
template <int U>
__global__ void __launch_bounds__(1024) sym_sell_kernel(int64_t n, const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ rlen,
                                                        const int32_t *__restrict__ blk_ptr,
                                                        const int32_t *__restrict__ col,
                                                        const double *__restrict__ val,
                                                        const double *__restrict__ x, double *y) {
    const int lane = threadIdx.x & 31;
    const int64_t nb = ceil_div_dev(n, 32);
    const int wpc = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5;
    // the SELL walk's rotations, as running 32-bit counters
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
        const int64_t r = b * 32 + lane;
        const int32_t len = r < n ? __ldg(rlen + r) : 0;
        const int32_t width = __shfl_sync(0xffffffffu, len, 0);
        const int64_t i = r < n ? (int64_t)__ldg(perm + r) : 0;
        const double xi = r < n ? __ldg(x + i) : 0.0;
        int64_t off = __ldg(blk_ptr + b);
        double s = 0.0;
        for (int32_t d0 = 0; d0 < width; d0 += U) {
            int c[U];
            double v[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const bool ok = len > d0 + j;
                c[j] = ok ? ld_stream(col + off + lane) : -1;
                v[j] = ok ? ld_stream(val + off + lane) : 0.0;
                off += __popc(__ballot_sync(0xffffffffu, ok));
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                if (c[j] < 0) continue;
                s = fma(v[j], __ldg(x + c[j]), s);
                if (c[j] != i) red_add(y + c[j], v[j] * xi);
            }
        }
        if (r < n) red_add(y + i, s);
    }
}

}  // namespace

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_upper_workspace(int64_t n_rows, int64_t *bytes) {
    if (n_rows < 0 || !bytes) return arg_error("gbsp_upper_workspace: bad arguments");
    *bytes = scan_ws_bytes(n_rows + 1);
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_upper_plan(gbsp_handle crs, int32_t *d_row_ptr_u, void *d_ws, int64_t ws_bytes,
                                       void *stream, int64_t *nnz_upper) {
    if (!crs || !d_row_ptr_u || !nnz_upper) return arg_error("gbsp_upper_plan: NULL argument");
    if (crs->kind != KIND_CRS) return arg_error("gbsp_upper_plan: not a CRS handle");
    if (crs->n_rows != crs->n_cols) {
        set_error("gbsp_upper_plan: the matrix must be square");
        return GBSP_ERR_UNSUPPORTED;
    }
    if (ws_bytes < scan_ws_bytes(crs->n_rows + 1) || !d_ws) return arg_error("gbsp_upper_plan: workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = crs->n_rows;
    if (n > 0) {
        upper_count_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, crs->row_ptr, crs->col, d_row_ptr_u);
        GBSP_LAUNCH_CHECK("upper_count_kernel");
    }
    gbsp_status st = scan_exclusive(d_row_ptr_u, n, d_row_ptr_u, d_row_ptr_u + n, static_cast<int32_t *>(d_ws), s);
    if (st != GBSP_OK) return st;
    int32_t total = 0;
    GBSP_CUDA(cudaMemcpyAsync(&total, d_row_ptr_u + n, 4, cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    *nnz_upper = total;
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_upper_build(gbsp_handle crs, const int32_t *d_row_ptr_u, int32_t *d_col_u,
                                        void *d_val_u, int64_t nnz_upper, void *stream, gbsp_handle *out) {
    if (!crs || !d_row_ptr_u || !out) return arg_error("gbsp_upper_build: NULL argument");
    if (crs->kind != KIND_CRS || crs->n_rows != crs->n_cols) return arg_error("gbsp_upper_build: needs a square CRS");
    if (nnz_upper < 0 || nnz_upper > crs->nnz || (nnz_upper > 0 && (!d_col_u || !d_val_u)))
        return arg_error("gbsp_upper_build: bad upper-triangle buffers");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = crs->n_rows;
    if (n > 0 && nnz_upper > 0) {
        if (crs->dtype == GBSP_F64)
            upper_fill_kernel<double><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                n, crs->row_ptr, crs->col, static_cast<const double *>(crs->val), d_row_ptr_u, d_col_u,
                static_cast<double *>(d_val_u));
        else
            upper_fill_kernel<float><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                n, crs->row_ptr, crs->col, static_cast<const float *>(crs->val), d_row_ptr_u, d_col_u,
                static_cast<float *>(d_val_u));
        GBSP_LAUNCH_CHECK("upper_fill_kernel");
    }
    return gbsp_crs_create(n, n, nnz_upper, d_row_ptr_u, d_col_u, d_val_u, (gbsp_dtype)crs->dtype, out);
}

extern "C" gbsp_status gbsp_spmv_symmetric(gbsp_handle S, const void *d_x, void *d_y, int32_t accumulate,
                                           void *stream) {
    if (!S) return arg_error("gbsp_spmv_symmetric: NULL handle");
    if (S->n_rows != S->n_cols) return arg_error("gbsp_spmv_symmetric: the matrix must be square");
    if (S->n_rows > 0 && (!d_x || !d_y)) return arg_error("gbsp_spmv_symmetric: NULL vector");
    if (S->dtype != GBSP_F64) {
        set_error("gbsp_spmv_symmetric: FP64 only");
        return GBSP_ERR_UNSUPPORTED;
    }
    const bool sell = S->kind == KIND_JDS && S->format == GBSP_SELL && S->perm_mode == GBSP_PERM_ROW_ONLY;
    if (S->kind != KIND_CRS && !sell) {
        set_error("gbsp_spmv_symmetric: needs a CRS handle or a SELL handle with the row-only permutation");
        return GBSP_ERR_UNSUPPORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = S->n_rows;
    const double *x = static_cast<const double *>(d_x);
    double *y = static_cast<double *>(d_y);
    if (!accumulate && n > 0) GBSP_CUDA(cudaMemsetAsync(y, 0, 8 * n, s));
    if (n == 0) return GBSP_OK;
    if (sell) {
        const int64_t nb = ceil_div(n, 32);
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb * 32, 1024), (int64_t)num_sms() * 2));
        const double *val = static_cast<const double *>(S->val);
        if (S->unroll <= 2)
            sym_sell_kernel<2><<<(unsigned)grid, 1024, 0, s>>>(n, S->perm, S->rlen, S->blk_ptr, S->col, val, x, y);
        else
            sym_sell_kernel<4><<<(unsigned)grid, 1024, 0, s>>>(n, S->perm, S->rlen, S->blk_ptr, S->col, val, x, y);
    } else {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8));
        sym_crs_kernel<4><<<(unsigned)grid, 256, 0, s>>>(n, S->row_ptr, S->col, static_cast<const double *>(S->val),
                                                          x, y);
    }
    GBSP_LAUNCH_CHECK("symmetric product kernel");
    return GBSP_OK;
}
