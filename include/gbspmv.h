/*
 * gbspmv -- sparse matrix-vector multiplication on GB300 (sm_103a).
 *
 * C ABI of the library.  It implements y = A*x for a sparse A stored in the
 * two schemes studied by Schubert, Hager & Fehske, "Performance limitations
 * for sparse matrix-vector multiplications on current multicore
 * environments" (Sect. 2): compressed row storage (CRS) and jagged diagonal
 * storage (JDS) with its refinements NBJDS, RBJDS, NUJDS and SOJDS; plus
 * multiple right-hand sides, the adjoint A^T*g, the per-entry value gradient,
 * a batched persistent launch and an FP32 path with compensated sums.
 *
 * Section numbers follow the paper's own order: 1 Introduction, 2 Common
 * storage schemes, 3 Test bed, 4 Limitations of serial performance (4.1
 * Basic sparse vector operations, 4.2 Resulting performance for SpMVM),
 * 5 Shared-memory parallel SpMVM (5.1 Intra-socket, 5.2 Inter-socket,
 * 5.3 HLRB-II scalability), 6 Conclusion and outlook.
 *
 * Conventions used by every entry point
 *   - Indices are 0-based int32; sizes and counts are int64.
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device;
 *     h_* are host pointers.  `stream` is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).
 *   - The library never allocates device memory: every device buffer is
 *     allocated by the caller and only borrowed.  A handle keeps the
 *     pointers it was given, so the caller must keep those buffers alive and
 *     unchanged in shape until gbsp_destroy.  Values may be overwritten in
 *     place between calls (e.g. by an optimiser) without rebuilding.
 *   - Every entry point returns a gbsp_status and never throws.  Kernel
 *     launches are asynchronous: a GBSP_OK return means the work was queued
 *     on `stream`.  Device-side checks (validation, bounded waits) report
 *     into a caller-provided int32 status word in device memory.
 *   - All kernels are deterministic: the same inputs give bit-identical
 *     outputs on every run (no floating-point atomics) -- except
 *     gbsp_spmv_symmetric, whose FP64 atomic adds make it reproducible only
 *     within rounding.
 */
#ifndef GBSPMV_H
#define GBSPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbsp_mat *gbsp_handle;
typedef struct gbsp_batch_s *gbsp_batch;

typedef enum {
    GBSP_OK = 0,
    GBSP_ERR_ARG = -1,         /* bad argument: null pointer, negative size, misaligned, mismatch */
    GBSP_ERR_MATRIX = -2,      /* malformed CRS: row_ptr not monotone, col out of range, nnz mismatch */
    GBSP_ERR_CUDA = -3,        /* a CUDA runtime call failed (message: gbsp_last_error) */
    GBSP_ERR_NOMEM = -4,       /* a caller buffer is smaller than the size the plan asked for */
    GBSP_ERR_UNSUPPORTED = -5, /* valid request this handle / build cannot serve */
    GBSP_ERR_TIMEOUT = -6      /* a bounded device-side wait gave up */
} gbsp_status;

typedef enum { GBSP_F64 = 0, GBSP_F32 = 1 } gbsp_dtype;

/* Storage schemes (Sect. 2).  JDS, NBJDS and NUJDS share one storage
 * pattern and differ in how the kernel walks it; RBJDS and SOJDS store each
 * row block consecutively.  JDS_LITERAL is the paper's diagonal-after-
 * diagonal loop with a result-vector round trip per diagonal.  SELL is the
 * RBJDS layout with blocks of 32 rows (one warp) and the decreasing-length
 * row sort restricted to windows of `window` rows -- SELL-32-sigma of
 * Kreutzer, Hager, Wellein, Fehske & Bishop (SIAM J. Sci. Comput. 2014),
 * the same group's follow-up; with one window it is RBJDS with block 32.
 * Rows stay near their original position, so the gathers of x keep the
 * matrix's locality while the lanes of a warp still do equal work.
 * PSELL (a GB300 layout of this library; the paper has none) pairs rows
 * inside each length-sorted window of `window` rows (a multiple of 64): the
 * row of rank q shares a lane with the row of rank m-1-q (m rows in the
 * window), so one lane walks a long row and then a short one and the lanes
 * of a warp do nearly equal work with far fewer idle slots than SELL at the
 * same window.  Block g holds lanes 32g'..32g'+31 of a window and owns the
 * permuted rows 64g .. 64g+R-1 (R = min(64, n-64g), L = ceil(R/2) lanes):
 * lane p's first row is permuted row 64g+p, its second (if any) 64g+L+p.
 * Storage is slot-major per block: slot t holds, in lane order, each lane
 * whose two rows together have more than t entries, with the lane's t-th
 * entry (first row's entries, then the second row's). */
typedef enum {
    GBSP_CRS = 0,
    GBSP_JDS = 1,
    GBSP_NBJDS = 2,
    GBSP_RBJDS = 3,
    GBSP_NUJDS = 4,
    GBSP_SOJDS = 5,
    GBSP_JDS_LITERAL = 6,
    GBSP_SELL = 7,
    GBSP_PSELL = 8
} gbsp_format;

/* Sect. 2: JDS permutes rows AND columns (A_{p(i),p(j)}), so all work runs in
 * the permuted basis (SYMMETRIC, the paper's scheme; square matrices only).
 * ROW_ONLY permutes rows only and keeps original column numbers (a
 * GPU-friendly deviation that preserves the locality of x). */
typedef enum { GBSP_PERM_SYMMETRIC = 0, GBSP_PERM_ROW_ONLY = 1 } gbsp_perm_mode;

typedef enum { GBSP_OP_N = 0, GBSP_OP_T = 1 } gbsp_op;

/* Basis of x and y for JDS-family handles.  PERMUTED: x is indexed like the
 * stored columns (x_p = P x under SYMMETRIC, x itself under ROW_ONLY) and y
 * comes out in permuted row order y_p = P y.  ORIGINAL: x and y in the
 * user's numbering; the kernel gathers through perm on the fly. */
typedef enum { GBSP_BASIS_PERMUTED = 0, GBSP_BASIS_ORIGINAL = 1 } gbsp_basis;

/* Accumulation mode for FP32 handles.  PLAIN: float products and sums.
 * COMPENSATED: per-row Dot2 (Ogita, Rump & Oishi 2005) -- exact products by
 * fmaf, TwoSum accumulation, carried through the lane reduction; result
 * rounded to float once.  FP64 handles ignore it. */
typedef enum { GBSP_ACC_PLAIN = 0, GBSP_ACC_COMPENSATED = 1 } gbsp_accum;

/* CRS kernel choice.  VECTOR: `lanes` threads of a warp per row, each warp
 * working on `rows_per_warp` rows at a time (lanes * rows in flight).
 * TILED: rows grouped into tiles of `tile` merge items (rows + entries);
 * a persistent CTA streams its tiles' val, col and row_ptr slices into
 * shared memory with bulk asynchronous copies (a producer warp, mbarrier
 * stages) and sums each row with one thread, rows sorted by length inside
 * the tile so that the lanes of a warp do equal work; needs
 * gbsp_crs_prepare.  RUNS: like VECTOR, a group of `lanes` threads owns
 * `rows_per_warp` consecutive rows, but it strides through their entries as
 * one contiguous run (CRS stores consecutive rows back to back), so a group
 * issues one FMA slot per entry of the run instead of one per entry of its
 * longest row; rows longer than 64 entries are cut out of the runs and
 * summed by the whole warp.  Suits irregular row lengths; lanes in
 * {1, 2, 4, 8}, rows_per_warp in {4, 8} and at least `lanes`.  AUTO picks
 * VECTOR from the row-length mean. */
typedef enum {
    GBSP_KERNEL_AUTO = 0,
    GBSP_KERNEL_VECTOR = 1,
    GBSP_KERNEL_TILED = 2,
    GBSP_KERNEL_RUNS = 3
} gbsp_kernel;

typedef struct {
    int32_t kernel;        /* gbsp_kernel */
    int32_t lanes;         /* VECTOR: 1, 2, 4, 8, 16 or 32; RUNS: 1, 2, 4 or 8 (0 = auto) */
    int32_t rows_per_warp; /* VECTOR: rows per lane group handled together, 1, 2 or 4;
                              RUNS: 4 or 8 (0 = auto) */
    int32_t tile;          /* TILED: merge items (rows + entries) per tile, 1024 or 2048 (0 = auto) */
    int32_t rhs_tile;      /* SpMM: right-hand sides handled per pass, 1..16 (0 = auto) */
    int32_t accum;         /* gbsp_accum (FP32 handles) */
    int32_t format;        /* JDS-family handles: walk in use (read only; set with gbsp_jds_set_format) */
    int32_t block;         /* NBJDS rows per block (read only) */
    int32_t unroll;        /* NUJDS diagonals per step (read only) */
} gbsp_kernel_opts;

/* ---------------------------------------------------------------- misc -- */

/* Human-readable name of a status code (static storage). */
const char *gbsp_status_string(gbsp_status s);

/* Text of the last CUDA or argument error seen by the calling thread
 * (thread-local, static storage, empty if none). */
const char *gbsp_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH (library plumbing; no
 * counterpart in the paper). */
int32_t gbsp_version(void);

/* Release a matrix handle (never the borrowed buffers).  NULL is a no-op.
 * Library plumbing; no counterpart in the paper. */
gbsp_status gbsp_destroy(gbsp_handle h);

/* Copy a device status word to *h_out (synchronises `stream`).  Library
 * plumbing for the bounded waits; no counterpart in the paper. */
gbsp_status gbsp_read_status(const int32_t *d_status, void *stream, int32_t *h_out);

/* Library plumbing, no counterpart in the paper.
 * Give a handle a device status word (int32, caller memory, NULL to clear).
 * Kernels with bounded waits (the TILED pipeline) store GBSP_ERR_TIMEOUT
 * there if a wait exceeds its limit (2 s) instead of hanging; the caller
 * resets it to 0.  Without a word such a timeout is silent. */
gbsp_status gbsp_set_status_word(gbsp_handle h, int32_t *d_status);

/* ----------------------------------------------------------------- CRS -- */

/* Create a CRS handle (Sect. 2, compressed row storage: val, col_idx and
 * row_ptr, row i owning entries row_ptr[i] .. row_ptr[i+1]-1).
 *   0 <= n_rows, n_cols < 2^31 - 1 and 0 <= nnz <= 2^31 - 2^16 - 1: the
 *   int32 index arrays, with 2^16 entries of headroom for padded layouts.
 *   d_row_ptr: int32[n_rows+1], d_col: int32[nnz], d_val: double[nnz]
 *   (GBSP_F64) or float[nnz] (GBSP_F32).  d_col and d_val may be NULL only
 *   when nnz == 0.  Entries inside a row may be in any column order.
 * Borrowed pointers; nothing is read here (no device work).  Errors:
 * GBSP_ERR_ARG on sizes outside those ranges, NULL pointers, misaligned
 * arrays or a bad dtype. */
gbsp_status gbsp_crs_create(int64_t n_rows, int64_t n_cols, int64_t nnz,
                            const int32_t *d_row_ptr, const int32_t *d_col,
                            const void *d_val, gbsp_dtype dtype, gbsp_handle *out);

/* Sect. 2 storage: the val array of a handle.
 * Point a CRS or JDS-family handle at new values (same pattern, same dtype,
 * d_val borrowed like the original).  Host-side only: no device work.  For
 * a JDS-family handle built with a value map (gbsp_jds_buffers.vmap) use
 * gbsp_jds_values to re-gather its values instead. */
gbsp_status gbsp_set_values(gbsp_handle h, const void *d_val);

/* Sect. 2, the CRS arrays and what they must satisfy.
 * Check the CRS arrays on the device: row_ptr[0] == 0, row_ptr
 * non-decreasing, row_ptr[n_rows] == nnz, 0 <= col < n_cols.  Writes 0 to
 * *d_status when all hold, else a GBSP_ERR_MATRIX code (no trap, no abort).
 * d_status: int32 in device memory.  Asynchronous on `stream`. */
gbsp_status gbsp_crs_validate(gbsp_handle crs, int32_t *d_status, void *stream);

/* Sect. 2 CRS kernel; the lane / row / tile shapes are the GPU's own.
 * Choose the kernel used by gbsp_spmv / gbsp_spmm for this CRS handle.
 * Only fields that differ from 0 override the current choice.  Errors:
 * GBSP_ERR_ARG for out-of-range values. */
gbsp_status gbsp_set_kernel(gbsp_handle h, const gbsp_kernel_opts *opts);
gbsp_status gbsp_get_kernel(gbsp_handle h, gbsp_kernel_opts *out);

/* Sect. 2 CRS kernel, TILED GPU variant (no counterpart in the paper).
 * TILED kernel set-up: bytes of the tile table for `tile` (1024 or 2048)
 * merge items per tile (the first row of every tile, then 16 bytes of
 * offsets per tile), and a device pass that fills it into caller memory
 * (16-byte aligned; borrowed until destroy or the next prepare).  The table
 * is a pure function of row_ptr.  TILED reads the matrix with bulk copies,
 * so gbsp_crs_prepare returns GBSP_ERR_ARG unless row_ptr, col and val are
 * 16-byte aligned. */
gbsp_status gbsp_crs_tile_bytes(gbsp_handle crs, int32_t tile, int64_t *bytes);
gbsp_status gbsp_crs_prepare(gbsp_handle crs, int32_t tile, void *d_table, int64_t table_bytes,
                             void *stream);

/* ----------------------------------------------------- CRS -> JDS family -- */

typedef struct {
    int32_t format;     /* gbsp_format, one of the JDS family */
    int32_t perm_mode;  /* gbsp_perm_mode */
    int32_t block;      /* NBJDS / RBJDS / SOJDS: rows per block (>= 1; 0 = 256) */
    int32_t unroll;     /* NUJDS / SELL: diagonals per step u (>= 1; 0 = 4) */
    int32_t window;     /* SELL: rows per sorting window, a multiple of 32 (PSELL: of 64) (0 = 1024) */
} gbsp_jds_opts;

typedef struct {
    int64_t n_rows, n_cols, nnz;
    int64_t n_diag;           /* N_j = longest row */
    int64_t n_blocks;         /* RBJDS / SOJDS blocks, SELL 32-row / PSELL 64-row blocks, else 0 */
    int64_t workspace_bytes;  /* scratch for gbsp_jds_build only */
} gbsp_jds_sizes;

/* Caller-allocated outputs of the conversion (device memory). */
typedef struct {
    int32_t *jd_ptr;   /* [n_diag+1] start of each jagged diagonal (Sect. 2 jd_ptr); SELL: unused */
    int32_t *col;      /* [nnz] column indices in storage order */
    void *val;         /* [nnz] values, same dtype as the CRS handle */
    int32_t *perm;     /* [n_rows] perm[new] = old row */
    int32_t *iperm;    /* [n_rows] iperm[old] = new row */
    int32_t *blk_ptr;  /* [n_blocks+1] RBJDS / SOJDS only, else may be NULL */
    void *workspace;   /* [workspace_bytes] scratch, free after the build completes */
    int32_t *vmap;     /* optional [nnz]: CRS entry index of every stored entry, kept by the
                          handle for gbsp_jds_values (NULL: not built) */
    int32_t *rlen;     /* SELL / PSELL only: [n_rows] length of every permuted row */
} gbsp_jds_buffers;

/* Sizes for converting `crs` (Sect. 2 JDS construction).  Reads the row
 * lengths on the device (d_scratch: at least 4 bytes of device memory used
 * for the longest-row reduction) and SYNCHRONISES `stream` to learn N_j.
 * Errors: GBSP_ERR_UNSUPPORTED for SYMMETRIC on a non-square matrix,
 * GBSP_ERR_ARG for a format outside the JDS family. */
gbsp_status gbsp_jds_plan(gbsp_handle crs, const gbsp_jds_opts *opts, int32_t *d_scratch,
                          void *stream, gbsp_jds_sizes *out);

/* Sect. 2, JDS construction and its refinements (NBJDS, RBJDS, NUJDS,
 * SOJDS); SELL / PSELL have no counterpart in the paper.
 * Build the JDS-family arrays on the device and return a handle over them
 * (borrowing `bufs`, except workspace).  Steps: row lengths; stable sort by
 * decreasing length (ties keep original row order, empty rows last) giving
 * perm / iperm; jd_ptr from #{rows with length > d}; entries shifted left
 * (slot d = the row's d-th stored entry) and scattered diagonal by
 * diagonal; columns renumbered by iperm under SYMMETRIC.  RBJDS re-lays
 * each block of `block` permuted rows contiguously, diagonal-major;
 * SOJDS additionally re-orders each row inside its block so that block
 * columns read x with stride one where possible (nearest-column greedy:
 * slot d of row r takes the unplaced entry whose column is closest to
 * 1 + the column in slot d of row r-1, ties to the smaller column; the first
 * row of a block keeps its order).  SELL / PSELL sort only inside windows of
 * `window` rows (stable, decreasing length); when the (window, length) pair
 * does not fit one 32-bit radix key, the sort runs as two stable passes,
 * length first, then window.  Output arrays are bit-exact functions of the
 * input.  `bufs` sizes must match gbsp_jds_plan. */
gbsp_status gbsp_jds_build(gbsp_handle crs, const gbsp_jds_opts *opts,
                           const gbsp_jds_buffers *bufs, const gbsp_jds_sizes *sizes,
                           void *stream, gbsp_handle *out);

/* Cap the grid (number of CTAs) of the handle's SELL, JDS / NUJDS walk and
 * CRS VECTOR product kernels at max_ctas (0 removes the cap).  A measurement
 * knob, the GPU counterpart of running the paper's OpenMP kernels on fewer
 * threads (Sect. 5.1, "Intra-socket performance"): the SELL kernel places at most
 * two 1024-thread CTAs per SM, the JDS / NUJDS walk up to eight 256-thread
 * CTAs, CRS VECTOR up to 21 CTAs of 64 threads (two warps, 48 registers).
 * Host-side only.  Errors: GBSP_ERR_ARG for a negative cap. */
gbsp_status gbsp_set_grid_limit(gbsp_handle h, int32_t max_ctas);

/* Sect. 2: JDS, NBJDS and NUJDS read the same storage.
 * Switch a built JDS-family handle between the formats that share its
 * storage pattern (JDS <-> NBJDS <-> NUJDS <-> JDS_LITERAL) and set block
 * or unroll.  RBJDS / SOJDS handles accept only a block size equal to the
 * one they were built with.  Errors: GBSP_ERR_UNSUPPORTED otherwise. */
gbsp_status gbsp_jds_set_format(gbsp_handle jds, int32_t format, int32_t block, int32_t unroll);

/* Sect. 2 storage: the permuted val array.
 * Re-gather a JDS-family handle's values from CRS-ordered values d_src_val
 * (nnz entries, the handle's dtype): val[i] = d_src_val[vmap[i]].  For
 * values that change while the pattern stays (training, time stepping).
 * Errors: GBSP_ERR_UNSUPPORTED if the handle was built without vmap. */
gbsp_status gbsp_jds_values(gbsp_handle jds, const void *d_src_val, void *stream);

/* Shared-memory staging of x for a SELL handle (GB300 addition; the paper
 * has none).  A warp-wide gather costs the L1TEX stage about one clock per
 * distinct cache line it touches, so scattered gathers, not bytes, bound
 * the SELL product on banded matrices.  Staging: for every group of 32
 * blocks (1024 permuted rows) the product kernel first copies up to
 * `pages_per_group` pages of x (1024 consecutive entries each; the pages
 * the group's entries reference most, each referenced at least `min_refs`
 * times, ties to the smaller page) into shared memory with coalesced loads,
 * then reads those entries' x values from there.  The arithmetic is
 * unchanged: staged and unstaged products are bit-identical.
 * gbsp_sell_stage_bytes: sizes of d_col_staged (int32, nnz entries), d_pages
 *   (int32, one row of pages_per_group per group) and the device workspace.
 * gbsp_sell_stage: builds both arrays (borrowed by the handle until destroy
 *   or the next call) and switches SpMVs with k = 1 whose x is not
 *   gathered through the permutation (row-only permutation, or the permuted
 *   basis) to the staged kernel.  pages_per_group: 1..14 (FP64) or 1..16
 *   (FP32) -- each page takes 8 or 4 KB of shared memory per CTA, two CTAs
 *   per SM; 0 removes the staging.  Synchronises `stream`.
 * Errors: GBSP_ERR_ARG (not SELL, bad counts, undersized buffers),
 * GBSP_ERR_UNSUPPORTED when (group, page) keys exceed 32 bits. */
gbsp_status gbsp_sell_stage_bytes(gbsp_handle sell, int32_t pages_per_group, int64_t *col_bytes,
                                  int64_t *pages_bytes, int64_t *ws_bytes);
gbsp_status gbsp_sell_stage(gbsp_handle sell, int32_t pages_per_group, int32_t min_refs, int32_t *d_col_staged,
                            int32_t *d_pages, void *d_ws, int64_t ws_bytes, void *stream);

/* Deep-diagonal split for the JDS and NUJDS walks (GB300 addition; the
 * paper has none).  The thread of a permuted row walks its jagged diagonals
 * one after another, so a few very long rows (heavy-tailed row lengths)
 * would serialise the whole product.  With a split, diagonals >= depth are
 * summed by a separate kernel in chunks of `chunk` diagonals -- one thread
 * per (row, chunk), so the long rows are spread over many threads -- into
 * partial sums in caller workspace, and the row walk stops at `depth` and
 * adds the row's partial sums (deterministic; the grouping of the sum
 * differs from the unsplit walk): rows with at most 8 chunks add them in
 * chunk order, longer rows in a fixed lane-strided tree.  Three launches per
 * product: the deep kernel runs on a stream of the handle (created here),
 * forked from `stream` and joined back with events, so it overlaps the walk;
 * the merge kernel follows on `stream` (capturable in a CUDA graph).  Calls
 * on one split handle must not overlap (they share the workspace and the
 * side stream).  k = 1 only (SpMM ignores the split).  depth = 0 removes the
 * split.
 * Workspace bytes from gbsp_jds_split_bytes; 256-byte aligned; borrowed
 * until destroy or the next gbsp_jds_split.  Synchronises `stream`. */
gbsp_status gbsp_jds_split_bytes(gbsp_handle jds, int32_t depth, int32_t chunk, int64_t *bytes);
gbsp_status gbsp_jds_split(gbsp_handle jds, int32_t depth, int32_t chunk, void *d_ws,
                           int64_t ws_bytes, void *stream);

/* Read back the JDS-family shape (host-side, no device work).  Library
 * plumbing; no counterpart in the paper. */
gbsp_status gbsp_jds_info(gbsp_handle jds, gbsp_jds_sizes *out, gbsp_jds_opts *opts);

/* Vector basis change (Sect. 2, "all further calculations are performed in
 * this permuted basis"): dir 0 writes out[r] = in[perm[r]] (to permuted),
 * dir 1 writes out[perm[r]] = in[r] (back).  k columns, row-major with
 * leading dimension ld (>= k) for both.  n = n_rows of the handle. */
gbsp_status gbsp_permute_vec(gbsp_handle jds, int32_t dir, int32_t k, const void *d_in,
                             int64_t ld_in, void *d_out, int64_t ld_out, void *stream);

/* ------------------------------------------------------------- products -- */

/* y = op(A) x, or y += op(A) x when accumulate != 0 (the paper's listings
 * update resvec in place; Sect. 2).  For CRS:
 *   y_i = sum_{j=row_ptr[i]}^{row_ptr[i+1]-1} val_j x[col_j].
 * For JDS-family handles the sum runs over the row's jagged-diagonal
 * entries; `basis` chooses the vector numbering (see gbsp_basis).
 * op = GBSP_OP_T needs a transpose attached (gbsp_transpose_build or
 * gbsp_attach_transpose) and uses basis ORIGINAL.
 * x: n_cols (op N) or n_rows (op T) elements of the handle's dtype, y the
 * other size; both contiguous device vectors that must not overlap.
 * Errors: GBSP_ERR_ARG (NULL, overlap), GBSP_ERR_UNSUPPORTED (op T without
 * transpose, op T in the permuted basis), GBSP_ERR_CUDA (launch). */
gbsp_status gbsp_spmv(gbsp_handle A, int32_t op, int32_t basis, int32_t accumulate,
                      const void *d_x, void *d_y, void *stream);

/* Sect. 2 product; the host transfers are library plumbing.
 * gbsp_spmv with the vectors in host memory: copies h_x into the device
 * stage d_x_stage (and h_y into d_y_stage when accumulate), runs the
 * product into d_y_stage, and copies it back to h_y, all in order on
 * `stream` and asynchronous to the host: h_y holds the result once the
 * stream has been synchronised, and h_x and the stages must stay untouched
 * until then.  Host vectors in page-locked memory move at the full speed of
 * the host link; pageable ones are staged by the driver.  The stages are
 * caller-allocated device vectors of the input and output sizes; calls on
 * different streams with their own stages overlap one product with the
 * copies of another.  Errors: those of gbsp_spmv, GBSP_ERR_ARG for NULL
 * vectors or overlapping stages, GBSP_ERR_CUDA for a failed copy. */
gbsp_status gbsp_spmv_host(gbsp_handle A, int32_t op, int32_t basis, int32_t accumulate,
                           const void *h_x, void *h_y, void *d_x_stage, void *d_y_stage,
                           void *stream);

/* The Sect. 2 sums applied to k vectors at once (no counterpart in the paper).
 * Y = op(A) X (+ Y) for k right-hand sides.  X and Y row-major: entry (i, c)
 * at [i*ld + c], ld >= k.  Every stored entry of A is read once per pass of
 * `rhs_tile` columns.  k = 1 with ld > 1 computes one strided column.
 * Performance: on a CRS handle a group of lanes covers the right-hand sides
 * of one row, so X's rows are read contiguously; the JDS-family walks give a
 * thread a row and gather k values of X per entry from rows far apart.  For
 * k >= 8 the CRS handle is the faster one by about 1.7x (HH-like 6M rows,
 * k = 16: 2.66 ms against 4.65 ms for SELL-32-sigma).  The batched launch's
 * autotuner picks the format per matrix with that in mind; a single handle
 * keeps the format it was built in. */
gbsp_status gbsp_spmm(gbsp_handle A, int32_t op, int32_t basis, int32_t k, const void *d_X,
                      int64_t ldx, void *d_Y, int64_t ldy, int32_t accumulate, void *stream);

/* ------------------------------------------------------- adjoint, dval -- */

/* Transpose of the Sect. 2 CRS sum, for the adjoint A^T g (no counterpart
 * in the paper).
 * Transposed structure of a CRS handle: a CRS of A^T (n_cols rows) whose
 * entries are listed per column of A in ascending entry order, plus
 * tmap[t] = index in A of transposed entry t.  Values are gathered with
 * gbsp_transpose_values (again whenever A's values change).  The result
 * handle is attached to `crs` so that gbsp_spmv(crs, OP_T, ...) uses it.
 *   bufs: t_row_ptr int32[n_cols+1], t_col int32[nnz] (= row of A),
 *         t_val [nnz] of A's dtype, tmap int32[nnz], workspace. */
typedef struct {
    int32_t *t_row_ptr;
    int32_t *t_col;
    void *t_val;
    int32_t *tmap;
    void *workspace;
} gbsp_transpose_buffers;

gbsp_status gbsp_transpose_workspace(gbsp_handle crs, int64_t *bytes);
gbsp_status gbsp_transpose_build(gbsp_handle crs, const gbsp_transpose_buffers *bufs,
                                 int64_t workspace_bytes, void *stream, gbsp_handle *out);
/* Transpose of the Sect. 2 CRS sum (no counterpart in the paper).
 * t_val[t] = val[tmap[t]] for the transpose built from `crs`. */
gbsp_status gbsp_transpose_values(gbsp_handle crs, void *stream);

/* Transpose of the Sect. 2 CRS sum (no counterpart in the paper).
 * Make `at` (any handle holding A^T, e.g. a JDS of the transpose) the one
 * used for gbsp_spmv(A, OP_T, ...).  Borrowed; no checks of its content. */
gbsp_status gbsp_attach_transpose(gbsp_handle A, gbsp_handle at);

/* Derivative of the Sect. 2 sum with respect to val (no counterpart in
 * the paper).
 * Value gradient of a CRS product: dval_k = g[row_k] * x[col_k] (the
 * derivative of g.(A x) with respect to val_k), written (or added with one
 * fused multiply-add, if accumulate) in CRS entry order.  g: n_rows,
 * x: n_cols, dval: nnz. */
gbsp_status gbsp_dval(gbsp_handle crs, const void *d_g, const void *d_x, void *d_dval,
                      int32_t accumulate, void *stream);

/* Derivative of iterated Sect. 2 products A^m x (Sect. 1: eigensolvers).
 * Fused multi-step value gradient: d = (accumulate ? dval_k : 0), then
 * d = fma(G[row_k, t], X[col_k, t], d) for t = 0 .. m-1, with G (n_rows x m,
 * ld ldg) and X (n_cols x m, ld ldx) row-major: one pass over the entries
 * for m product pairs of an iterated product A^m x.  The fixed order makes
 * the result independent of how the t range is split over calls. */
gbsp_status gbsp_dval_multi(gbsp_handle crs, int32_t m, const void *d_G, int64_t ldg,
                            const void *d_X, int64_t ldx, void *d_dval, int32_t accumulate,
                            void *stream);

/* Derivative of iterated Sect. 2 products A^m x (Sect. 1: eigensolvers).
 * The same with any element layout: G[row, t] at d_G + row*g_row + t*g_t and
 * X[col, t] at d_X + col*x_row + t*x_t (elements; all strides >= 1).  With
 * g_row = x_row = 1 and g_t = x_t = the vector length, G and X are m
 * separate contiguous vectors (column-major), the layout in which each of
 * the iterated products reads and writes its vector with unit stride.
 * Same order of operations, hence the same result, as gbsp_dval_multi on
 * the same values.  Errors: GBSP_ERR_ARG for m < 1, a stride < 1, NULL
 * arrays, or dval overlapping G or X. */
gbsp_status gbsp_dval_multi_strided(gbsp_handle crs, int32_t m, const void *d_G, int64_t g_row,
                                    int64_t g_t, const void *d_X, int64_t x_row, int64_t x_t,
                                    void *d_dval, int32_t accumulate, void *stream);

/* -------------------------------------------------------------- batched -- */

/* One item of a batch: Y_b = A_b X_b with k_b right-hand sides (row-major,
 * leading dimensions ldx/ldy).  A_b is a CRS or JDS-family handle of
 * either dtype; its current kernel options give the rows per warp and
 * right-hand-side tile used inside the batch.  JDS items run in the
 * permuted basis. */
typedef struct {
    gbsp_handle A;
    int32_t k;
    const void *X;
    int64_t ldx;
    void *Y;
    int64_t ldy;
} gbsp_batch_item;

/* Many Sect. 2 products in one launch (no counterpart in the paper).
 * Bytes of the device work table for n items (work items of about
 * `chunk` entries each; 0 = 4096). */
gbsp_status gbsp_batch_plan(int32_t n, const gbsp_batch_item *items, int32_t chunk,
                            int64_t *table_bytes);

/* Many Sect. 2 products in one launch (no counterpart in the paper).
 * Write the work table into caller memory d_table (256-byte aligned,
 * table_bytes from the plan) and return a batch object.  Reads each
 * matrix's row pointers back to the host once and synchronises `stream`.
 * d_ready (may be NULL): an int32 flag in device or host-mapped memory;
 * when given, every launch first waits until it is non-zero -- set by the
 * host or by work finished earlier on the stream, never by a kernel
 * running at the same time -- for at most 1 s. */
gbsp_status gbsp_batch_create(int32_t n, const gbsp_batch_item *items, int32_t chunk,
                              void *d_table, int64_t table_bytes, const int32_t *d_ready,
                              void *stream, gbsp_batch *out);

/* Many Sect. 2 products in one launch (no counterpart in the paper).
 * All items in one persistent launch: CTAs take work items from the table
 * through a device counter (reset by a memset on `stream` first, so the
 * memset + kernel pair can be captured in a CUDA graph and replayed).
 * Items are written, never accumulated.  CRS items use the VECTOR
 * arithmetic of their handle (lanes per row), JDS-family items their
 * thread-per-row walk, so each result is bit-identical to gbsp_spmm of the
 * same handle with the VECTOR / JDS kernel.  d_status (may be NULL)
 * receives GBSP_ERR_TIMEOUT if the wait for d_ready ran out (the launch then
 * does no work); the caller resets it. */
gbsp_status gbsp_batch_run(gbsp_batch b, int32_t *d_status, void *stream);

/* Number of work items and persistent CTAs of a batch (host-side).
 * Library plumbing; no counterpart in the paper. */
gbsp_status gbsp_batch_info(gbsp_batch b, int64_t *n_work, int32_t *grid);
gbsp_status gbsp_batch_destroy(gbsp_batch b);

/* ------------------------------------------------------ allocation-free -- */

/* y = A x (or y += A x) for a CRS matrix in ONE call that allocates
 * nothing: no handle, no plan buffer, no cudaMalloc / cudaFree and no
 * allocating library routine.  It is for callers that cannot allocate
 * device memory themselves -- for example a solver whose device memory all
 * belongs to a host application's pool, or code on a path where an
 * allocation is not allowed because it would synchronise the device.  (The
 * paper has no counterpart; this is a library convenience.)
 *
 * Arguments are those of gbsp_crs_create plus x (n_cols), y (n_rows) and
 * `accumulate`; row_ptr, col and val must be 16-byte aligned.  It runs the
 * TILED kernel with 1024-item tiles, whose tile table is built on every call
 * in a fixed 8 MiB array of device memory inside the library (held by every
 * GPU that loads the library until the process exits), so n_rows + nnz may
 * be at most about 4.1e8; larger sizes return GBSP_ERR_ARG with a message.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make the first call on each device before any
 * stream capture.  The address is looked up again when the device's current
 * context changes (after cudaDeviceReset, for example), so that call too
 * should come before any capture.  All calls share the one array and
 * rewrite it fully: calls that can overlap on the GPU (different streams
 * without ordering) race and give wrong results; calls ordered on one stream
 * are safe.  The TILED kernel's bounded waits have no status word here: if
 * one gives up (a stalled copy; none was ever observed), y is left partly
 * written and the call still returned GBSP_OK.  Callers that need that
 * reported use a handle with gbsp_set_status_word. */
gbsp_status gbsp_crs_spmv_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                  const int32_t *d_row_ptr, const int32_t *d_col,
                                  const void *d_val, gbsp_dtype dtype, int32_t accumulate,
                                  const void *d_x, void *d_y, void *stream);

/* ------------------------------------------------ basic gather operations -- */

/* The basic sparse vector operations of Sect. 4.1 ("Basic sparse vector operations"; its table of ADD and SCP
 * kernels), which isolate the cost of the indirect x access of the SpMVM
 * inner loop:
 *     ADD:  s = sum_{i<n} B(idx(i))        SCP:  s = sum_{i<n} A(i) * B(idx(i))
 * with idx(i) = i (PD, packed dense), stride*i (CS, constant stride computed
 * in the loop) or ind(i) (IND: the paper's IS with ind(i) = k*i and IR with
 * random strides differ only in the index array the caller passes). */
typedef enum { GBSP_GATHER_ADD = 0, GBSP_GATHER_SCP = 1 } gbsp_gather_op;
/* IND_TMA is IND with B fetched by the tensor memory accelerator (tile::
 * gather4 copies of 16-byte rows into shared memory) instead of one load
 * per lane: the GB300 alternative for gathers that miss L1, measured beside
 * IND.  It needs len_b >= 2, len_b / 2 < 2^31 and B 16-byte aligned. */
typedef enum { GBSP_ACCESS_PD = 0, GBSP_ACCESS_CS = 1, GBSP_ACCESS_IND = 2, GBSP_ACCESS_IND_TMA = 3 } gbsp_access;

/* Sect. 4.1, the basic sparse vector operations.
 * Number of FP64 partial sums gbsp_gather_sum needs for n elements on the
 * current device (one per CTA of its grid). */
gbsp_status gbsp_gather_partials(int64_t n, int32_t *n_partials);

/* Sect. 4.1, the basic sparse vector operations.
 * *d_out = the sum above, FP64.  d_a [n] (SCP only), d_b [len_b], d_ind [n]
 * (IND only) int32, all device memory borrowed for the call; d_partials is
 * caller scratch of n_partials doubles (>= gbsp_gather_partials(n)).  Each
 * thread sums its elements in ascending i, then fixed reduction trees: the
 * result is the same on every run on a given device.  Two launches on
 * `stream`, asynchronous.  n = 0 gives 0.
 * Errors: GBSP_ERR_ARG for an unknown op or access, NULL pointers, PD with
 * n > len_b, CS with stride < 1 or (n-1)*stride >= len_b, or n_partials
 * too small.  IND entries outside [0, len_b) are skipped (they add nothing)
 * and set *d_status = GBSP_ERR_ARG when d_status (device int32) is given;
 * the call never clears *d_status. */
gbsp_status gbsp_gather_sum(int32_t op, int32_t access, int64_t n, int64_t stride,
                            const double *d_a, const double *d_b, int64_t len_b,
                            const int32_t *d_ind, double *d_partials, int32_t n_partials,
                            double *d_out, int32_t *d_status, void *stream);

/* Sect. 4.1, the cost of the other way around the indirect access: stage
 * the gathered vector in shared memory by panels and read it from there.
 * For uniformly random indices every SM needs every panel, so B crosses
 * from L2 into each SM's shared memory once per product; this launch does
 * exactly that and nothing else (one CTA per SM, each streaming the whole
 * 16-byte blocks of d_b [len_b] into shared memory with 32 KB bulk copies,
 * four in flight), so its time is a floor for any column-panel gather of
 * such indices.  d_out [n_out >= the SM count] receives, per CTA, the sum
 * of the first double of every 32 KB chunk.  A bounded wait that gives up
 * (1 s) writes GBSP_ERR_TIMEOUT to *d_status when d_status (device int32)
 * is given.  One launch on `stream`.  Errors: GBSP_ERR_ARG for NULL
 * pointers, B not 16-byte aligned or n_out too small. */
gbsp_status gbsp_stage_sweep(const double *d_b, int64_t len_b, double *d_out, int32_t n_out, int32_t *d_status,
                             void *stream);

/* The FP64 issue rate that bounds every kernel here besides HBM.  The paper
 * sets SpMVM against both the memory bandwidth and the peak Flop rate of
 * each machine (Sect. 4, "Limitations of serial performance"); GB300's FP64
 * rate is low enough to be a roofline of its own, so it is measured.  Each
 * of n_threads threads (256 per CTA) runs 8 independent chains
 * x_j <- fma(x_j, a, b), x_j starting at in[0] + j, for `iters` steps, with
 * a = d_in[1] and b = d_in[2] (device, 3 doubles); d_out[t] (device,
 * n_threads doubles) = the sum of thread t's chains, in chain order.  Lanes
 * >= active_lanes (0..32) of each warp skip the chains and write 0; their
 * warp's FMAs still issue, which is what the count of idle lanes costs.
 * Flops of a launch: 16 * iters * (active lanes in all warps).  One launch
 * on `stream`, asynchronous.  Errors: GBSP_ERR_ARG for negative sizes,
 * active_lanes > 32 or NULL pointers. */
gbsp_status gbsp_fma_chain(int64_t n_threads, int32_t active_lanes, int32_t iters, const double *d_in,
                           double *d_out, void *stream);

/* ------------------------------------- hybrid storage: DIA + remainder -- */

/* Sect. 4.2 ("Resulting performance for SpMVM") observes that most entries of the Holstein-Hubbard matrix sit
 * in a few dense outer secondary diagonals, any of which could be stored
 * densely, and leaves such a hybrid unbuilt.  Here the selected diagonals
 * go to DIA storage (one value per row, zeros where the diagonal has no
 * entry, no column index) and every
 * other entry to a remainder CRS matrix, which may then be converted to any
 * format of this library.  The product is y = DIA x followed by the
 * remainder's product with accumulate = 1, so y_i = (DIA sum) + (remainder
 * sum).
 *
 * Diagonal of offset o = col - row; its length is the number of in-matrix
 * positions (i, i+o); fill = its entries / its length.  gbsp_dia_plan keeps
 * the offsets with fill >= min_fill (2/3 is the FP64 break-even: 8 bytes a
 * DIA slot against 12 an entry), ranked by entry count (descending), then
 * |o|, then o, at most max_diags (<= GBSP_DIA_MAX).  In each row, the first
 * entry (CRS order) on a selected diagonal goes to DIA; the rest stay.
 *
 * gbsp_dia_plan_workspace: device scratch bytes of gbsp_dia_plan.
 * gbsp_dia_plan: an exact offset histogram on the device, read back
 *   (4 (n_rows + n_cols) bytes) for the selection; fills d_row_ptr_rem
 *   (int32 [n_rows+1], caller memory) with the remainder's row_ptr and *out
 *   with the chosen offsets and counts.  Synchronises `stream`.
 * gbsp_dia_build: d_dia [n_diags * n_rows] (dtype of the CRS; diagonal k
 *   at d_dia + k*n_rows, entry i = row i), d_offsets int32 [n_diags], and the
 *   remainder's d_col_rem [nnz_rem], d_val_rem [nnz_rem].  Returns a DIA
 *   handle (gbsp_spmv / gbsp_spmm with k = 1, OP_N; it borrows d_dia and
 *   d_offsets) and a CRS handle of the remainder.  Synchronises `stream`.
 * Errors: GBSP_ERR_ARG for bad sizes or NULL buffers. */
#define GBSP_DIA_MAX 64
typedef struct {
    int64_t n_rows, n_cols;
    int32_t n_diags;                   /* diagonals selected */
    int32_t offsets[GBSP_DIA_MAX];     /* their offsets, in rank order */
    int64_t nnz_dia;                   /* entries moved to DIA */
    int64_t nnz_rem;                   /* entries left in the remainder */
} gbsp_dia_sizes;

gbsp_status gbsp_dia_plan_workspace(gbsp_handle crs, int64_t *bytes);
gbsp_status gbsp_dia_plan(gbsp_handle crs, int32_t max_diags, double min_fill, int32_t *d_row_ptr_rem,
                          void *d_ws, int64_t ws_bytes, void *stream, gbsp_dia_sizes *out);
gbsp_status gbsp_dia_build(gbsp_handle crs, const gbsp_dia_sizes *sizes, void *d_dia, int32_t *d_offsets,
                           const int32_t *d_row_ptr_rem, int32_t *d_col_rem, void *d_val_rem, void *stream,
                           gbsp_handle *dia_out, gbsp_handle *rem_out);

/* --------------------------------------------- symmetric SpMVM (one triangle) -- */

/* The Hamiltonian of Sect. 4.2 ("Resulting performance for SpMVM") is symmetric, which the paper notes would
 * allow a further saving of data transfer and does not pursue.  These calls
 * store only the upper triangle U (col >= row) of a square CRS matrix and
 * apply it as A = U + U^T - diag(U), reading half of the off-diagonal
 * entries.
 *
 * gbsp_upper_workspace: device scratch bytes gbsp_upper_plan needs.
 * gbsp_upper_plan: counts the upper entries of each row into d_row_ptr_u
 *   (int32 [n_rows+1], caller memory) and scans them, so d_row_ptr_u is U's
 *   row_ptr; *nnz_upper = its last entry.  Synchronises `stream`.
 * gbsp_upper_build: fills d_col_u [nnz_upper] and d_val_u [nnz_upper] (the
 *   CRS dtype) with the upper entries in their CRS order and returns a CRS
 *   handle over (d_row_ptr_u, d_col_u, d_val_u), borrowed as usual.
 * Errors: GBSP_ERR_UNSUPPORTED for a non-square matrix, GBSP_ERR_ARG for
 * NULL or undersized buffers. */
gbsp_status gbsp_upper_workspace(int64_t n_rows, int64_t *bytes);
gbsp_status gbsp_upper_plan(gbsp_handle crs, int32_t *d_row_ptr_u, void *d_ws, int64_t ws_bytes, void *stream,
                            int64_t *nnz_upper);
gbsp_status gbsp_upper_build(gbsp_handle crs, const int32_t *d_row_ptr_u, int32_t *d_col_u, void *d_val_u,
                             int64_t nnz_upper, void *stream, gbsp_handle *out);

/* Sect. 4.2: the Hamiltonian is symmetric (the paper stores it in full).
 * y = (S + S^T - diag S) x for the stored entries S of handle `S` -- A x
 * when S holds the upper triangle of a symmetric A.  S: a CRS handle
 * (thread per row) or a SELL handle with the row-only permutation (warp per
 * 32-row block; vectors in the original basis either way).  FP64 only.
 * Each stored off-diagonal s_ij adds s_ij x_j to y_i and s_ij x_i to y_j;
 * updates of y are FP64 atomic adds, so y is first zeroed (accumulate = 0)
 * or added to (accumulate = 1), and the summation order -- hence the last
 * bits -- may differ between runs; exact when all partial sums are.
 * Asynchronous on `stream` (a memset and one kernel).
 * Errors: GBSP_ERR_UNSUPPORTED for FP32 or other formats, GBSP_ERR_ARG for
 * NULL vectors or a non-square handle. */
gbsp_status gbsp_spmv_symmetric(gbsp_handle S, const void *d_x, void *d_y, int32_t accumulate, void *stream);

/* -------------------------------------------------- access-pattern analysis -- */

/* Stride distribution of the x accesses (Sect. 4.2, "Resulting performance for SpMVM", Fig. 4a).  For a
 * column-index array read in storage order -- the order in which the
 * paper's serial CRS, JDS, RBJDS and SOJDS loops read x -- counts every jump
 * s = col[i+1] - col[i] by size: bin 0 is s = 0, bin b >= 1 holds
 * 2^(b-1) <= |s| < 2^b (x strides of 8*2^(b-1) to 8*2^b - 1 bytes for
 * FP64).  d_hist: int64 [66] device memory, overwritten: [0..32] forward
 * jumps (s >= 0), [33..65] backward jumps (s < 0).  d_col: int32 [nnz]
 * device.  Exact counts (integer atomics).  Asynchronous on `stream`.
 * Errors: GBSP_ERR_ARG for NULL pointers or nnz < 0. */
gbsp_status gbsp_stride_hist(const int32_t *d_col, int64_t nnz, int64_t *d_hist, void *stream);

/* Sectors per warp-wide gather of x (GB300 counterpart of the stride
 * analysis; the paper has none).  For every warp-wide load of x that the
 * handle's product kernel issues, the number c of distinct 32-byte sectors
 * it touches (elem_bytes per x entry: 8 for FP64, 4 for FP32);
 * d_hist[c] (int64 [33], device memory, overwritten) counts such loads.
 * Patterns: CRS with `lanes` lanes per row (1, 2, 4, ..., 32; a warp holds
 * 32/lanes consecutive rows, lane l of a row reads entries l, l+lanes, ...);
 * JDS / NUJDS / NBJDS / JDS_LITERAL storage with a thread per permuted row
 * (a warp holds 32 consecutive rows, one load per jagged diagonal); SELL
 * (a warp holds one 32-row block, one load per slot).  `lanes` is ignored
 * for JDS-family handles.  Asynchronous on `stream`.
 * Errors: GBSP_ERR_ARG (bad lanes or elem_bytes), GBSP_ERR_UNSUPPORTED for
 * RBJDS / SOJDS handles. */
gbsp_status gbsp_warp_sectors(gbsp_handle A, int32_t lanes, int32_t elem_bytes, int64_t *d_hist,
                              void *stream);

/* ------------------------------------------------------------ autotuner -- */

/* Chooses among the Sect. 2 kernels and block sizes, the GPU counterpart
 * of the paper's block-size sweeps (Sect. 4.2).
 * Time the candidate kernels for `A` with k right-hand sides on the device
 * (CUDA events on `stream`, a few repetitions each, X and Y are scratch
 * vectors of the right sizes) and keep the fastest option set on the handle.
 * For CRS handles the candidates are VECTOR with lanes 2..32 and every
 * rows_per_warp, RUNS in six shapes, and TILED (when prepared); for
 * JDS-family handles the formats sharing
 * the handle's storage and their block/unroll values.  *best receives the
 * choice and *best_ms its time.  Synchronises `stream`. */
gbsp_status gbsp_autotune(gbsp_handle A, int32_t k, const void *d_X, void *d_Y, void *stream,
                          gbsp_kernel_opts *best, float *best_ms);

#ifdef __cplusplus
}
#endif

#endif /* GBSPMV_H */
