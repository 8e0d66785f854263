// C ABI entry points: handle management, argument checks and dispatch.
#include <algorithm>
#include <cstdarg>
#include <new>

#include "internal.cuh"

namespace gbsp {

static thread_local char g_err[512] = {0};

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

gbsp_status cuda_status(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return GBSP_ERR_CUDA;
}

static size_t elem_size(int dtype) { return dtype == GBSP_F64 ? 8 : 4; }

static bool is_jds_family(int f) {
    return f == GBSP_JDS || f == GBSP_NBJDS || f == GBSP_RBJDS || f == GBSP_NUJDS ||
           f == GBSP_SOJDS || f == GBSP_JDS_LITERAL || f == GBSP_SELL ||
           f == GBSP_PSELL;
}

// [a, a+na) and [b, b+nb) in bytes
static bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

// Strided k-column blocks X (ldx) and Y (ldy): they overlap if their byte
// spans meet and, for equal leading dimensions, their columns coincide
// modulo ld (interleaved columns of one row-major block are disjoint).
static bool blocks_overlap(const void *x, size_t xb, int64_t ldx, const void *y, size_t yb, int64_t ldy,
                           int32_t k, int dtype) {
    if (!overlap(x, xb, y, yb)) return false;
    const int64_t es = (int64_t)(dtype == GBSP_F64 ? 8 : 4);
    const int64_t diff = static_cast<const char *>(y) - static_cast<const char *>(x);
    if (ldx != ldy || ldx <= k || diff % es != 0) return true;
    const int64_t d = diff / es;
    const int64_t r = ((d % ldx) + ldx) % ldx;
    return r < k || r > ldx - k;
}

static size_t span_bytes(int64_t rows, int64_t ld, int32_t k, int dtype) {
    if (rows <= 0) return 0;
    return (size_t)((rows - 1) * ld + k) * elem_size(dtype);
}

}  // namespace gbsp

using namespace gbsp;

extern "C" {

const char *gbsp_status_string(gbsp_status s) {
    switch (s) {
        case GBSP_OK: return "GBSP_OK";
        case GBSP_ERR_ARG: return "GBSP_ERR_ARG";
        case GBSP_ERR_MATRIX: return "GBSP_ERR_MATRIX";
        case GBSP_ERR_CUDA: return "GBSP_ERR_CUDA";
        case GBSP_ERR_NOMEM: return "GBSP_ERR_NOMEM";
        case GBSP_ERR_UNSUPPORTED: return "GBSP_ERR_UNSUPPORTED";
        case GBSP_ERR_TIMEOUT: return "GBSP_ERR_TIMEOUT";
    }
    return "GBSP_UNKNOWN_STATUS";
}

const char *gbsp_last_error(void) { return g_err; }

int32_t gbsp_version(void) { return 10000; }

gbsp_status gbsp_destroy(gbsp_handle h) {
    if (!h) return GBSP_OK;
    if (h->split_side) {
        cudaStreamSynchronize(h->split_side);
        cudaStreamDestroy(h->split_side);
        cudaEventDestroy(h->split_fork);
        cudaEventDestroy(h->split_join);
    }
    if (h->owns_transpose && h->transpose) delete static_cast<gbsp_mat *>(h->transpose);
    delete h;
    return GBSP_OK;
}

gbsp_status gbsp_read_status(const int32_t *d_status, void *stream, int32_t *h_out) {
    if (!d_status || !h_out) return arg_error("gbsp_read_status: NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GBSP_CUDA(cudaMemcpyAsync(h_out, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    return GBSP_OK;
}

gbsp_status gbsp_crs_create(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *d_row_ptr,
                            const int32_t *d_col, const void *d_val, gbsp_dtype dtype,
                            gbsp_handle *out) {
    if (!out) return arg_error("gbsp_crs_create: out is NULL");
    *out = nullptr;
    if (n_rows < 0 || n_cols < 0 || nnz < 0) return arg_error("gbsp_crs_create: negative size");
    if (nnz >= (int64_t(1) << 31) - (int64_t(1) << 16) || n_rows >= (int64_t(1) << 31) - 1 ||
        n_cols >= (int64_t(1) << 31) - 1)
        return arg_error("gbsp_crs_create: sizes must fit int32 indices");
    if (dtype != GBSP_F64 && dtype != GBSP_F32) return arg_error("gbsp_crs_create: bad dtype");
    if (!d_row_ptr) return arg_error("gbsp_crs_create: row_ptr is NULL");
    if (nnz > 0 && (!d_col || !d_val)) return arg_error("gbsp_crs_create: col/val NULL with nnz > 0");
    if ((reinterpret_cast<uintptr_t>(d_row_ptr) & 3) || (reinterpret_cast<uintptr_t>(d_col) & 3) ||
        (reinterpret_cast<uintptr_t>(d_val) & (elem_size(dtype) - 1)))
        return arg_error("gbsp_crs_create: misaligned array");
    gbsp_mat *h = new (std::nothrow) gbsp_mat();
    if (!h) return arg_error("gbsp_crs_create: out of host memory");
    h->kind = KIND_CRS;
    h->n_rows = n_rows;
    h->n_cols = n_cols;
    h->nnz = nnz;
    h->dtype = dtype;
    cudaGetDevice(&h->device);
    h->row_ptr = d_row_ptr;
    h->col = d_col;
    h->val = d_val;
    h->format = GBSP_CRS;
    crs_default_opts(*h);
    *out = h;
    return GBSP_OK;
}

gbsp_status gbsp_crs_validate(gbsp_handle crs, int32_t *d_status, void *stream) {
    if (!crs || !d_status) return arg_error("gbsp_crs_validate: NULL argument");
    if (crs->kind != KIND_CRS) return arg_error("gbsp_crs_validate: not a CRS handle");
    return crs_validate_launch(*crs, d_status, static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_set_kernel(gbsp_handle h, const gbsp_kernel_opts *o) {
    if (!h || !o) return arg_error("gbsp_set_kernel: NULL argument");
    if (o->kernel < 0 || o->kernel > GBSP_KERNEL_RUNS) return arg_error("gbsp_set_kernel: bad kernel");
    if (o->lanes != 0 && (o->lanes < 1 || o->lanes > 32 || (o->lanes & (o->lanes - 1))))
        return arg_error("gbsp_set_kernel: lanes must be 1, 2, 4, 8, 16 or 32");
    if (o->kernel == GBSP_KERNEL_RUNS) {
        if (o->lanes > 8) return arg_error("gbsp_set_kernel: RUNS lanes must be 1, 2, 4 or 8");
        if (o->rows_per_warp != 0 && o->rows_per_warp != 4 && o->rows_per_warp != 8)
            return arg_error("gbsp_set_kernel: RUNS rows_per_warp must be 4 or 8");
        const int l = o->lanes ? o->lanes : 4, r = o->rows_per_warp ? o->rows_per_warp : (l > 4 ? 8 : 4);
        if (r < l) return arg_error("gbsp_set_kernel: RUNS needs rows_per_warp >= lanes");
    } else if (o->rows_per_warp != 0 && o->rows_per_warp != 1 && o->rows_per_warp != 2 &&
               o->rows_per_warp != 4) {
        return arg_error("gbsp_set_kernel: rows_per_warp must be 1, 2 or 4");
    }
    if (h->kind == KIND_JDS && (o->kernel == GBSP_KERNEL_TILED || o->kernel == GBSP_KERNEL_RUNS))
        return arg_error("gbsp_set_kernel: TILED and RUNS are CRS kernels");
    if (o->tile != 0 && o->tile != 1024 && o->tile != 2048)
        return arg_error("gbsp_set_kernel: tile must be 1024 or 2048");
    if (o->rhs_tile != 0 && (o->rhs_tile < 1 || o->rhs_tile > 32))
        return arg_error("gbsp_set_kernel: rhs_tile must be in 1..32");
    if (o->accum != 0 && o->accum != GBSP_ACC_COMPENSATED)
        return arg_error("gbsp_set_kernel: bad accum");
    if (o->kernel == GBSP_KERNEL_TILED && !h->tile_rows)
        return arg_error("gbsp_set_kernel: TILED needs gbsp_crs_prepare first");
    if (o->kernel != 0) h->kopt.kernel = o->kernel;
    if (o->kernel == GBSP_KERNEL_RUNS) {
        // every field of the pair is RUNS's own: never a VECTOR leftover
        h->kopt.lanes = o->lanes ? o->lanes : 4;
        h->kopt.rows_per_warp = o->rows_per_warp ? o->rows_per_warp : (h->kopt.lanes > 4 ? 8 : 4);
    } else {
        if (o->lanes != 0) h->kopt.lanes = o->lanes;
        if (o->rows_per_warp != 0) h->kopt.rows_per_warp = o->rows_per_warp;
    }
    if (o->rhs_tile != 0) h->kopt.rhs_tile = o->rhs_tile;
    h->kopt.accum = o->accum;
    if (o->kernel == GBSP_KERNEL_AUTO) crs_default_opts(*h);
    return GBSP_OK;
}

gbsp_status gbsp_get_kernel(gbsp_handle h, gbsp_kernel_opts *out) {
    if (!h || !out) return arg_error("gbsp_get_kernel: NULL argument");
    *out = h->kopt;
    out->tile = h->tile;
    out->format = h->kind == KIND_JDS ? h->format : GBSP_CRS;
    out->block = h->kind == KIND_JDS ? h->block : 0;
    out->unroll = h->kind == KIND_JDS ? h->unroll : 0;
    return GBSP_OK;
}

gbsp_status gbsp_set_values(gbsp_handle h, const void *d_val) {
    if (!h) return arg_error("gbsp_set_values: NULL handle");
    if (h->nnz > 0 && !d_val) return arg_error("gbsp_set_values: NULL values");
    if (reinterpret_cast<uintptr_t>(d_val) & (elem_size(h->dtype) - 1))
        return arg_error("gbsp_set_values: misaligned values");
    if (h->kind == KIND_CRS && h->tile_rows && (reinterpret_cast<uintptr_t>(d_val) & 15))
        return arg_error("gbsp_set_values: the prepared TILED kernel needs 16-byte aligned values");
    h->val = d_val;
    return GBSP_OK;
}

gbsp_status gbsp_jds_values(gbsp_handle h, const void *d_src_val, void *stream) {
    if (!h || (h->nnz > 0 && !d_src_val)) return arg_error("gbsp_jds_values: NULL argument");
    if (h->kind != KIND_JDS) return arg_error("gbsp_jds_values: not a JDS-family handle");
    if (!h->vmap) {
        set_error("gbsp_jds_values: handle was built without a value map");
        return GBSP_ERR_UNSUPPORTED;
    }
    return jds_values_launch(*h, d_src_val, static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_crs_tile_bytes(gbsp_handle crs, int32_t tile, int64_t *bytes) {
    if (!crs || !bytes) return arg_error("gbsp_crs_tile_bytes: NULL argument");
    if (tile != 1024 && tile != 2048) return arg_error("gbsp_crs_tile_bytes: tile must be 1024 or 2048");
    *bytes = crs_tile_table_bytes(*crs, tile);
    return GBSP_OK;
}

gbsp_status gbsp_crs_prepare(gbsp_handle crs, int32_t tile, void *d_table, int64_t table_bytes,
                             void *stream) {
    int64_t need = 0;
    gbsp_status st = gbsp_crs_tile_bytes(crs, tile, &need);
    if (st != GBSP_OK) return st;
    if (crs->kind != KIND_CRS) return arg_error("gbsp_crs_prepare: not a CRS handle");
    if (!d_table || (reinterpret_cast<uintptr_t>(d_table) & 15))
        return arg_error("gbsp_crs_prepare: table must be a 16-byte aligned device buffer");
    // the bulk copies of the TILED kernel need 16-byte aligned arrays
    if ((reinterpret_cast<uintptr_t>(crs->row_ptr) & 15) || (reinterpret_cast<uintptr_t>(crs->col) & 15) ||
        (reinterpret_cast<uintptr_t>(crs->val) & 15))
        return arg_error("gbsp_crs_prepare: TILED needs row_ptr, col and val 16-byte aligned");
    if (table_bytes < need) {
        set_error("gbsp_crs_prepare: table needs %lld bytes", (long long)need);
        return GBSP_ERR_NOMEM;
    }
    return crs_prepare_tiles(*crs, tile, static_cast<int32_t *>(d_table),
                             static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_set_status_word(gbsp_handle h, int32_t *d_status) {
    if (!h) return arg_error("gbsp_set_status_word: NULL handle");
    if (reinterpret_cast<uintptr_t>(d_status) & 3) return arg_error("gbsp_set_status_word: misaligned");
    h->status = d_status;
    return GBSP_OK;
}

gbsp_status gbsp_jds_plan(gbsp_handle crs, const gbsp_jds_opts *opts, int32_t *d_scratch,
                          void *stream, gbsp_jds_sizes *out) {
    if (!crs || !opts || !out || !d_scratch) return arg_error("gbsp_jds_plan: NULL argument");
    if (crs->kind != KIND_CRS) return arg_error("gbsp_jds_plan: not a CRS handle");
    if (!is_jds_family(opts->format)) return arg_error("gbsp_jds_plan: format is not a JDS variant");
    if (opts->perm_mode != GBSP_PERM_SYMMETRIC && opts->perm_mode != GBSP_PERM_ROW_ONLY)
        return arg_error("gbsp_jds_plan: bad perm_mode");
    if (opts->block < 0 || opts->unroll < 0) return arg_error("gbsp_jds_plan: negative block/unroll");
    if (opts->perm_mode == GBSP_PERM_SYMMETRIC && crs->n_rows != crs->n_cols) {
        set_error("gbsp_jds_plan: the symmetric permutation needs a square matrix");
        return GBSP_ERR_UNSUPPORTED;
    }
    return jds_plan_impl(*crs, *opts, d_scratch, static_cast<cudaStream_t>(stream), out);
}

gbsp_status gbsp_jds_build(gbsp_handle crs, const gbsp_jds_opts *opts, const gbsp_jds_buffers *bufs,
                           const gbsp_jds_sizes *sizes, void *stream, gbsp_handle *out) {
    if (!crs || !opts || !bufs || !sizes || !out) return arg_error("gbsp_jds_build: NULL argument");
    *out = nullptr;
    if (crs->kind != KIND_CRS) return arg_error("gbsp_jds_build: not a CRS handle");
    if (!is_jds_family(opts->format)) return arg_error("gbsp_jds_build: format is not a JDS variant");
    if (opts->perm_mode == GBSP_PERM_SYMMETRIC && crs->n_rows != crs->n_cols) {
        set_error("gbsp_jds_build: the symmetric permutation needs a square matrix");
        return GBSP_ERR_UNSUPPORTED;
    }
    if (sizes->n_rows != crs->n_rows || sizes->nnz != crs->nnz)
        return arg_error("gbsp_jds_build: sizes do not come from this matrix");
    const bool sell = opts->format == GBSP_SELL || opts->format == GBSP_PSELL;
    const bool blocked = opts->format == GBSP_RBJDS || opts->format == GBSP_SOJDS || sell;
    if (sell && crs->n_rows > 0 && !bufs->rlen) return arg_error("gbsp_jds_build: SELL needs rlen");
    if ((!sell && !bufs->jd_ptr) || (crs->n_rows > 0 && (!bufs->perm || !bufs->iperm)) ||
        (crs->nnz > 0 && (!bufs->col || !bufs->val)) || (blocked && !bufs->blk_ptr) ||
        (sizes->workspace_bytes > 0 && !bufs->workspace))
        return arg_error("gbsp_jds_build: a required buffer is NULL");
    gbsp_mat *J = new (std::nothrow) gbsp_mat();
    if (!J) return arg_error("gbsp_jds_build: out of host memory");
    gbsp_status st = jds_build_impl(*crs, *opts, *bufs, *sizes, static_cast<cudaStream_t>(stream), J);
    if (st != GBSP_OK) {
        delete J;
        return st;
    }
    *out = J;
    return GBSP_OK;
}

gbsp_status gbsp_set_grid_limit(gbsp_handle h, int32_t max_ctas) {
    if (!h || max_ctas < 0) return arg_error("gbsp_set_grid_limit: bad arguments");
    h->grid_limit = max_ctas;
    return GBSP_OK;
}

gbsp_status gbsp_jds_set_format(gbsp_handle h, int32_t format, int32_t block, int32_t unroll) {
    if (!h) return arg_error("gbsp_jds_set_format: NULL handle");
    if (h->kind != KIND_JDS || !is_jds_family(format))
        return arg_error("gbsp_jds_set_format: not a JDS-family handle / format");
    if (block < 0 || unroll < 0) return arg_error("gbsp_jds_set_format: negative block/unroll");
    const bool was_blocked = h->built_block > 0;
    const bool to_blocked =
        format == GBSP_RBJDS || format == GBSP_SOJDS || format == GBSP_SELL || format == GBSP_PSELL;
    if (was_blocked != to_blocked || (was_blocked && format != h->format) ||
        (was_blocked && block != 0 && block != h->built_block)) {
        set_error("gbsp_jds_set_format: storage layout differs; rebuild instead");
        return GBSP_ERR_UNSUPPORTED;
    }
    h->format = format;
    if (block > 0) h->block = block;
    if (unroll > 0) h->unroll = unroll;
    return GBSP_OK;
}

gbsp_status gbsp_jds_split_bytes(gbsp_handle h, int32_t depth, int32_t chunk, int64_t *bytes) {
    if (!h || !bytes) return arg_error("gbsp_jds_split_bytes: NULL argument");
    if (h->kind != KIND_JDS || h->built_block > 0)
        return arg_error("gbsp_jds_split_bytes: needs a JDS / NUJDS handle (JDS storage)");
    if (depth < 1 || chunk < 1) return arg_error("gbsp_jds_split_bytes: depth and chunk must be >= 1");
    return jds_split_bytes_impl(*h, depth, chunk, bytes);
}

gbsp_status gbsp_jds_split(gbsp_handle h, int32_t depth, int32_t chunk, void *d_ws, int64_t ws_bytes,
                           void *stream) {
    if (!h) return arg_error("gbsp_jds_split: NULL handle");
    if (h->kind != KIND_JDS || h->built_block > 0)
        return arg_error("gbsp_jds_split: needs a JDS / NUJDS handle (JDS storage)");
    if (depth == 0) {
        h->split_k = 0;
        h->split_depth = 0;
        return GBSP_OK;
    }
    if (depth < 1 || chunk < 1 || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255))
        return arg_error("gbsp_jds_split: bad depth / chunk, or workspace not 256-byte aligned");
    return jds_split_impl(*h, depth, chunk, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_jds_info(gbsp_handle h, gbsp_jds_sizes *out, gbsp_jds_opts *opts) {
    if (!h) return arg_error("gbsp_jds_info: NULL handle");
    if (h->kind != KIND_JDS) return arg_error("gbsp_jds_info: not a JDS-family handle");
    if (out) {
        out->n_rows = h->n_rows;
        out->n_cols = h->n_cols;
        out->nnz = h->nnz;
        out->n_diag = h->n_diag;
        out->n_blocks = h->n_blocks;
        out->workspace_bytes = 0;
    }
    if (opts) {
        opts->format = h->format;
        opts->perm_mode = h->perm_mode;
        opts->block = h->block;
        opts->unroll = h->unroll;
    }
    return GBSP_OK;
}

gbsp_status gbsp_permute_vec(gbsp_handle h, int32_t dir, int32_t k, const void *d_in, int64_t ld_in,
                             void *d_out, int64_t ld_out, void *stream) {
    if (!h || (h->n_rows > 0 && (!d_in || !d_out))) return arg_error("gbsp_permute_vec: NULL argument");
    if (h->kind != KIND_JDS) return arg_error("gbsp_permute_vec: not a JDS-family handle");
    if ((dir != 0 && dir != 1) || k < 1 || ld_in < k || ld_out < k)
        return arg_error("gbsp_permute_vec: bad dir / k / leading dimension");
    if (overlap(d_in, span_bytes(h->n_rows, ld_in, k, h->dtype), d_out,
                span_bytes(h->n_rows, ld_out, k, h->dtype)))
        return arg_error("gbsp_permute_vec: in and out overlap");
    return permute_launch(*h, dir, k, d_in, ld_in, d_out, ld_out, static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_spmm(gbsp_handle A, int32_t op, int32_t basis, int32_t k, const void *d_X,
                      int64_t ldx, void *d_Y, int64_t ldy, int32_t accumulate, void *stream) {
    if (!A) return arg_error("gbsp_spmm: NULL handle");
    if (op != GBSP_OP_N && op != GBSP_OP_T) return arg_error("gbsp_spmm: bad op");
    if (basis != GBSP_BASIS_PERMUTED && basis != GBSP_BASIS_ORIGINAL) return arg_error("gbsp_spmm: bad basis");
    if (k < 1 || ldx < k || ldy < k) return arg_error("gbsp_spmm: need k >= 1 and ld >= k");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (op == GBSP_OP_T) {
        if (!A->transpose) {
            set_error("gbsp_spmm: OP_T needs an attached transpose (gbsp_transpose_build)");
            return GBSP_ERR_UNSUPPORTED;
        }
        if (A->kind == KIND_JDS && basis == GBSP_BASIS_PERMUTED) {
            set_error("gbsp_spmm: OP_T runs in the original basis only");
            return GBSP_ERR_UNSUPPORTED;
        }
        return gbsp_spmm(static_cast<gbsp_handle>(A->transpose), GBSP_OP_N, GBSP_BASIS_ORIGINAL, k, d_X, ldx, d_Y, ldy,
                         accumulate, stream);
    }
    const size_t xb = span_bytes(A->n_cols, ldx, k, A->dtype), yb = span_bytes(A->n_rows, ldy, k, A->dtype);
    if ((xb > 0 && !d_X) || (yb > 0 && !d_Y)) return arg_error("gbsp_spmm: NULL vector");
    if (blocks_overlap(d_X, xb, ldx, d_Y, yb, ldy, k, A->dtype)) return arg_error("gbsp_spmm: x and y overlap");
    const uintptr_t am = elem_size(A->dtype) - 1;
    if ((reinterpret_cast<uintptr_t>(d_X) & am) || (reinterpret_cast<uintptr_t>(d_Y) & am))
        return arg_error("gbsp_spmm: misaligned vector");
    VecArgs v{};
    v.x = d_X;
    v.y = d_Y;
    v.ldx = ldx;
    v.ldy = ldy;
    v.k = k;
    v.accumulate = accumulate ? 1 : 0;
    if (A->kind == KIND_CRS) return crs_launch(*A, v, s);
    if (A->kind == KIND_DIA) return dia_launch(*A, v, s);
    if (basis == GBSP_BASIS_ORIGINAL) {
        v.y_perm = A->perm;
        v.x_perm = A->perm_mode == GBSP_PERM_SYMMETRIC ? A->perm : nullptr;
    }
    return jds_launch(*A, v, s);
}

gbsp_status gbsp_spmv(gbsp_handle A, int32_t op, int32_t basis, int32_t accumulate, const void *d_x,
                      void *d_y, void *stream) {
    return gbsp_spmm(A, op, basis, 1, d_x, 1, d_y, 1, accumulate, stream);
}

gbsp_status gbsp_spmv_host(gbsp_handle A, int32_t op, int32_t basis, int32_t accumulate, const void *h_x,
                           void *h_y, void *d_x_stage, void *d_y_stage, void *stream) {
    if (!A) return arg_error("gbsp_spmv_host: NULL handle");
    if (op != GBSP_OP_N && op != GBSP_OP_T) return arg_error("gbsp_spmv_host: bad op");
    const int64_t n_in = op == GBSP_OP_N ? A->n_cols : A->n_rows;
    const int64_t n_out = op == GBSP_OP_N ? A->n_rows : A->n_cols;
    const size_t es = elem_size(A->dtype);
    if ((n_in > 0 && (!h_x || !d_x_stage)) || (n_out > 0 && (!h_y || !d_y_stage)))
        return arg_error("gbsp_spmv_host: NULL vector or stage");
    if (overlap(d_x_stage, (size_t)n_in * es, d_y_stage, (size_t)n_out * es))
        return arg_error("gbsp_spmv_host: the stages overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_in > 0) GBSP_CUDA(cudaMemcpyAsync(d_x_stage, h_x, (size_t)n_in * es, cudaMemcpyHostToDevice, s));
    if (accumulate && n_out > 0)
        GBSP_CUDA(cudaMemcpyAsync(d_y_stage, h_y, (size_t)n_out * es, cudaMemcpyHostToDevice, s));
    gbsp_status st = gbsp_spmm(A, op, basis, 1, d_x_stage, 1, d_y_stage, 1, accumulate, stream);
    if (st != GBSP_OK) return st;
    if (n_out > 0) GBSP_CUDA(cudaMemcpyAsync(h_y, d_y_stage, (size_t)n_out * es, cudaMemcpyDeviceToHost, s));
    return GBSP_OK;
}

gbsp_status gbsp_transpose_workspace(gbsp_handle crs, int64_t *bytes) {
    if (!crs || !bytes) return arg_error("gbsp_transpose_workspace: NULL argument");
    if (crs->kind != KIND_CRS) return arg_error("gbsp_transpose_workspace: not a CRS handle");
    return transpose_workspace_impl(*crs, bytes);
}

gbsp_status gbsp_transpose_build(gbsp_handle crs, const gbsp_transpose_buffers *bufs,
                                 int64_t workspace_bytes, void *stream, gbsp_handle *out) {
    if (!crs || !bufs || !out) return arg_error("gbsp_transpose_build: NULL argument");
    *out = nullptr;
    if (crs->kind != KIND_CRS) return arg_error("gbsp_transpose_build: not a CRS handle");
    if (!bufs->t_row_ptr || (crs->nnz > 0 && (!bufs->t_col || !bufs->t_val || !bufs->tmap || !bufs->workspace)))
        return arg_error("gbsp_transpose_build: a required buffer is NULL");
    gbsp_mat *T = new (std::nothrow) gbsp_mat();
    if (!T) return arg_error("gbsp_transpose_build: out of host memory");
    gbsp_status st = transpose_build_impl(*crs, *bufs, workspace_bytes, static_cast<cudaStream_t>(stream), T);
    if (st != GBSP_OK) {
        delete T;
        return st;
    }
    if (crs->owns_transpose && crs->transpose) delete static_cast<gbsp_mat *>(crs->transpose);
    crs->transpose = T;
    crs->owns_transpose = false;  // the caller owns the returned handle
    *out = T;
    return GBSP_OK;
}

gbsp_status gbsp_transpose_values(gbsp_handle crs, void *stream) {
    if (!crs) return arg_error("gbsp_transpose_values: NULL handle");
    const Mat *T = crs->transpose;
    if (!T || !T->tmap || T->transpose_src != crs) {
        set_error("gbsp_transpose_values: no transpose built from this handle");
        return GBSP_ERR_UNSUPPORTED;
    }
    return transpose_values_impl(*T, static_cast<cudaStream_t>(stream));
}

gbsp_status gbsp_attach_transpose(gbsp_handle A, gbsp_handle at) {
    if (!A || !at) return arg_error("gbsp_attach_transpose: NULL handle");
    if (at->n_rows != A->n_cols || at->n_cols != A->n_rows || at->dtype != A->dtype)
        return arg_error("gbsp_attach_transpose: shape or dtype does not match A^T");
    A->transpose = at;
    A->owns_transpose = false;
    return GBSP_OK;
}

gbsp_status gbsp_dval(gbsp_handle crs, const void *d_g, const void *d_x, void *d_dval,
                      int32_t accumulate, void *stream) {
    return gbsp_dval_multi(crs, 1, d_g, 1, d_x, 1, d_dval, accumulate, stream);
}

gbsp_status gbsp_dval_multi(gbsp_handle crs, int32_t m, const void *d_G, int64_t ldg, const void *d_X,
                            int64_t ldx, void *d_dval, int32_t accumulate, void *stream) {
    if (m < 1 || ldg < m || ldx < m) return arg_error("gbsp_dval: need m >= 1 and ld >= m");
    return gbsp_dval_multi_strided(crs, m, d_G, ldg, 1, d_X, ldx, 1, d_dval, accumulate, stream);
}

// bytes from the first to one past the last element of a rows x m array
static size_t strided_span_bytes(int64_t rows, int64_t row_stride, int32_t m, int64_t t_stride, int dtype) {
    if (rows <= 0 || m <= 0) return 0;
    return (size_t)((rows - 1) * row_stride + (int64_t)(m - 1) * t_stride + 1) * elem_size(dtype);
}

gbsp_status gbsp_dval_multi_strided(gbsp_handle crs, int32_t m, const void *d_G, int64_t g_row, int64_t g_t,
                                    const void *d_X, int64_t x_row, int64_t x_t, void *d_dval,
                                    int32_t accumulate, void *stream) {
    if (!crs) return arg_error("gbsp_dval: NULL handle");
    if (crs->kind != KIND_CRS) return arg_error("gbsp_dval: needs the CRS handle");
    if (m < 1 || g_row < 1 || g_t < 1 || x_row < 1 || x_t < 1)
        return arg_error("gbsp_dval: need m >= 1 and positive strides");
    if (crs->nnz > 0 && (!d_G || !d_X || !d_dval)) return arg_error("gbsp_dval: NULL vector");
    const size_t out_bytes = (size_t)crs->nnz * elem_size(crs->dtype);
    if (overlap(d_dval, out_bytes, d_G, strided_span_bytes(crs->n_rows, g_row, m, g_t, crs->dtype)) ||
        overlap(d_dval, out_bytes, d_X, strided_span_bytes(crs->n_cols, x_row, m, x_t, crs->dtype)))
        return arg_error("gbsp_dval: output overlaps an input");
    return crs_dval_launch(*crs, m, d_G, g_row, g_t, d_X, x_row, x_t, d_dval, accumulate ? 1 : 0,
                           static_cast<cudaStream_t>(stream));
}

}  // extern "C"
