// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/gbspmv.h"

namespace gbsp {

enum HandleKind { KIND_CRS = 0, KIND_JDS = 1, KIND_DIA = 2 };

struct Mat {
    int kind = KIND_CRS;
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    int dtype = GBSP_F64;
    int device = 0;

    // CRS arrays (CRS handles) / col+val in storage order (JDS handles)
    const int32_t *row_ptr = nullptr;
    const int32_t *col = nullptr;
    const void *val = nullptr;

    // kernel options
    gbsp_kernel_opts kopt{};

    // TILED CRS tile table (first row of every tile, then one int4 per tile)
    const int32_t *tile_rows = nullptr;
    const int4 *tile_meta = nullptr;
    int64_t n_tiles = 0;
    int32_t tile = 0;

    // optional device status word for bounded-wait timeouts
    int32_t *status = nullptr;

    // largest grid (CTAs) of the SELL, JDS-walk and CRS-vector product
    // kernels; 0 = no limit (a measurement knob: throughput against the
    // number of CTAs in use)
    int32_t grid_limit = 0;

    // JDS family
    int format = GBSP_CRS;
    int perm_mode = GBSP_PERM_SYMMETRIC;
    int32_t block = 0, unroll = 0;
    int32_t built_block = 0;  // block size the RBJDS/SOJDS layout was built with
    int64_t n_diag = 0, n_blocks = 0;
    const int32_t *jd_ptr = nullptr, *perm = nullptr, *iperm = nullptr, *blk_ptr = nullptr;
    const int32_t *vmap = nullptr;  // JDS position -> CRS entry (optional)
    const int32_t *rlen = nullptr;  // SELL: length of every permuted row
    int32_t window = 0;             // SELL: rows per sorting window

    // JDS / NUJDS deep-diagonal split (caller workspace): diagonals >= split_depth
    // are summed in chunks by a separate kernel into ragged partial sums
    int32_t split_depth = 0, split_chunk = 0, split_k = 0;
    int64_t split_items_total = 0;
    const int4 *split_table = nullptr;  // per chunk {d_begin, d_end, rows, partial offset}
    const int32_t *split_items = nullptr;  // per chunk: first CTA item (k+1 entries)
    void *split_part = nullptr;
    void *split_shallow = nullptr;  // walk sums of the rows deeper than split_depth
    int64_t split_rows = 0;         // those rows: [0, split_rows)
    int64_t split_wide_rows = 0;    // rows with more than 8 chunks: [0, split_wide_rows)
    // SELL with x staged in shared memory: per 1024-row group (32 blocks)
    // up to stage_pages_per_group pages of 1024 x entries, and the columns
    // re-encoded (staged entries as ~(slot*1024 + col % 1024))
    const int32_t *stage_col = nullptr;
    const int32_t *stage_pages = nullptr;
    int32_t stage_pages_per_group = 0;
    // the deep kernel runs on a side stream of the handle, forked from and
    // joined back to the caller's stream with these events
    cudaStream_t split_side = nullptr;
    cudaEvent_t split_fork = nullptr, split_join = nullptr;
    std::vector<int32_t> h_jd_ptr;  // host copy, read back once at build (literal launches)

    // transposed structure (CRS handle built by gbsp_transpose_build)
    const int32_t *tmap = nullptr;  // set on the transpose handle itself
    const Mat *transpose_src = nullptr;  // the CRS this transpose was built from
    Mat *transpose = nullptr;        // attached handle used for OP_T
    bool owns_transpose = false;
};

// error reporting ---------------------------------------------------------
void set_error(const char *fmt, ...);
gbsp_status cuda_status(cudaError_t e, const char *what);

#define GBSP_CUDA(call)                                             \
    do {                                                            \
        cudaError_t e__ = (call);                                   \
        if (e__ != cudaSuccess) return gbsp::cuda_status(e__, #call); \
    } while (0)

#define GBSP_LAUNCH_CHECK(what)                                          \
    do {                                                                 \
        cudaError_t e__ = cudaGetLastError();                            \
        if (e__ != cudaSuccess) return gbsp::cuda_status(e__, what);     \
    } while (0)

inline gbsp_status arg_error(const char *msg) {
    set_error("%s", msg);
    return GBSP_ERR_ARG;
}

inline int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// a launcher's grid under a handle's grid limit (0 = none)
inline int64_t limit_grid(int64_t grid, int32_t limit) { return limit > 0 && grid > limit ? limit : grid; }

// device exclusive scan of int32 (convert.cu): out[0..n) = exclusive scan of
// in, *total_out = the total when given; ws holds scan_ws_bytes(n) bytes
int64_t scan_ws_bytes(int64_t n);
// stable LSD radix sort of bare uint32 keys (convert.cu)
int64_t sort_keys_ws_bytes(int64_t n);
gbsp_status sort_keys(uint32_t *keys, int64_t n, int bits, void *ws, cudaStream_t s, uint32_t **sorted);
gbsp_status scan_exclusive(const int32_t *in, int64_t n, int32_t *out, int32_t *total_out, int32_t *ws,
                           cudaStream_t s);

// launchers implemented in crs.cu -----------------------------------------
struct VecArgs {
    const void *x;
    void *y;
    int64_t ldx, ldy;   // row-major leading dims (1 for plain vectors)
    int32_t k;          // right-hand sides
    int32_t accumulate;
    const int32_t *x_perm;   // optional: x index = x_perm[col]
    const int32_t *y_perm;   // optional: y row = y_perm[row]
};

// DIA part of the hybrid storage (dia.cu): y (+)= sum_k dia[k][i] x[i+o_k]
gbsp_status dia_launch(const Mat &A, const VecArgs &v, cudaStream_t s);


gbsp_status crs_launch(const Mat &A, const VecArgs &v, cudaStream_t s);
gbsp_status crs_prepare_tiles(Mat &A, int32_t tile, int32_t *table, cudaStream_t s);
int64_t crs_tile_table_bytes(const Mat &A, int32_t tile);
gbsp_status crs_tiled_launch(const Mat &A, const VecArgs &v, cudaStream_t s);
gbsp_status crs_validate_launch(const Mat &A, int32_t *d_status, cudaStream_t s);
gbsp_status crs_dval_launch(const Mat &A, int32_t m, const void *G, int64_t g_row, int64_t g_t,
                            const void *X, int64_t x_row, int64_t x_t, void *dval, int32_t accumulate,
                            cudaStream_t s);
void crs_default_opts(Mat &A);

// jds.cu ----------------------------------------------------------------
gbsp_status jds_launch(const Mat &A, const VecArgs &v, cudaStream_t s);
gbsp_status permute_launch(const Mat &A, int32_t dir, int32_t k, const void *in, int64_t ld_in,
                           void *out, int64_t ld_out, cudaStream_t s);
gbsp_status jds_split_bytes_impl(const Mat &A, int32_t depth, int32_t chunk, int64_t *bytes);
gbsp_status jds_split_impl(Mat &A, int32_t depth, int32_t chunk, void *ws, int64_t bytes, cudaStream_t s);

// convert.cu ------------------------------------------------------------
gbsp_status jds_plan_impl(const Mat &A, const gbsp_jds_opts &o, int32_t *d_scratch,
                          cudaStream_t s, gbsp_jds_sizes *out);
gbsp_status jds_build_impl(const Mat &A, const gbsp_jds_opts &o, const gbsp_jds_buffers &b,
                           const gbsp_jds_sizes &sz, cudaStream_t s, Mat *J);
gbsp_status transpose_workspace_impl(const Mat &A, int64_t *bytes);
gbsp_status transpose_build_impl(const Mat &A, const gbsp_transpose_buffers &b, int64_t ws_bytes,
                                 cudaStream_t s, Mat *T);
gbsp_status transpose_values_impl(const Mat &T, cudaStream_t s);
gbsp_status jds_values_launch(const Mat &J, const void *src, cudaStream_t s);
gbsp_status gather_values_launch(int64_t n, const int32_t *map, const void *src, void *dst, int dtype,
                                 cudaStream_t s);

}  // namespace gbsp

struct gbsp_mat : gbsp::Mat {};
