/*
 * Plain, slow, obviously-correct CPU oracle for sparse matrix-vector
 * multiplication in CRS and JDS storage (Schubert, Hager & Fehske,
 * "Performance limitations for sparse matrix-vector multiplications on
 * current multicore environments", Sect. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline of the benchmark do.  It shares no code, header or constant with
 * the CUDA path.
 *
 * Conventions: 0-based int32 indices, FP64 values, sequential loops in the
 * order the paper writes them.  Build with -ffp-contract=off so that every
 * "a + b*c" is a rounded multiply followed by a rounded add, exactly as the
 * listings read.  fma() appears only where an exact product split is wanted
 * (the accurate reference), never as contraction.
 *
 * Readings of points the paper leaves open:
 *   - resvec starts from zero unless `accumulate` is set (the listings only
 *     show the update "resvec = resvec + ...").
 *   - The JDS row sort is stable: equal row lengths keep ascending original
 *     row order; empty rows end up last.
 *   - Entries keep their CRS storage order inside a row when shifted left
 *     (slot d of a row is its d-th stored entry).
 *   - Blocks for NBJDS / RBJDS / SOJDS are runs of b consecutive permuted
 *     rows, the last one partial; RBJDS stores a block diagonal by diagonal.
 *   - NUJDS with N_j not a multiple of u: the last group has fewer diagonals.
 *   - SOJDS: greedy nearest-column rule, see orc_sojds_build.  The paper fixes
 *     no rule (its storage figure is not available): parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define DIAGLEN(jd, d) ((int64_t)(jd)[(d) + 1] - (int64_t)(jd)[(d)])

/* ------------------------------------------------------------------------
 * CRS  (Sect. 2, CRS kernel): y_i = sum over the entries j of row i of
 *       val_j * x[col_idx_j], added in storage order onto y_i.
 * ---------------------------------------------------------------------- */
void orc_crs_spmv(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *val, const double *invec, double *resvec, int accumulate)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double r = accumulate ? resvec[i] : 0.0;
        for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
            r = r + val[j] * invec[col_idx[j]];
        resvec[i] = r;
    }
}

/* The same loop in single precision (values, vector and sum all float). */
void orc_crs_spmv_f32(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                      const float *val, const float *invec, float *resvec, int accumulate)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        float r = accumulate ? resvec[i] : 0.0f;
        for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
            r = r + val[j] * invec[col_idx[j]];
        resvec[i] = r;
    }
}

/* Sect. 5.2: the paper's best shared-memory setting is the CRS loop with an
 * OpenMP static schedule over rows (first-touch placed arrays).  Same
 * per-row arithmetic as orc_crs_spmv, so the results are bit-identical. */
void orc_crs_spmv_omp(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *invec, double *resvec, int accumulate)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_rows; ++i) {
        double r = accumulate ? resvec[i] : 0.0;
        for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
            r = r + val[j] * invec[col_idx[j]];
        resvec[i] = r;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Multiple right-hand sides: X and Y row-major (n x k, leading dims ldx, ldy);
 * column c of Y is the CRS loop applied to column c of X. */
void orc_crs_spmm(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *val, int64_t k, const double *X, int64_t ldx,
                  double *Y, int64_t ldy, int accumulate)
{
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t c = 0; c < k; ++c) {
            double r = accumulate ? Y[i * ldy + c] : 0.0;
            for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
                r = r + val[j] * X[(int64_t)col_idx[j] * ldx + c];
            Y[i * ldy + c] = r;
        }
}

/* ------------------------------------------------------------------------
 * Accurate reference for y = A x (and y += A x): each product is split
 * exactly, p + e = a*x with e = fma(a, x, -p), and all terms are summed in
 * double-double with Knuth's TwoSum -- the "Dot2" scheme of Ogita, Rump &
 * Oishi (SIAM J. Sci. Comput. 26, 2005).  Its error is at most
 * u|y| + gamma_n^2 sum|a||x| (u = 2^-53), i.e. essentially correctly
 * rounded.  absrow[i] = sum_j |a_ij||x_j| feeds the test tolerance.
 * ---------------------------------------------------------------------- */
static inline void two_sum(double a, double b, double *s, double *e)
{
    double t = a + b;
    double z = t - a;
    *e = (a - (t - z)) + (b - z);
    *s = t;
}

void orc_crs_spmv_exact(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
                        const double *val, const double *invec, double *resvec,
                        double *absrow, int accumulate)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double s = accumulate ? resvec[i] : 0.0, c = 0.0;
        double a = accumulate ? fabs(resvec[i]) : 0.0;
        for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            double p = val[j] * invec[col_idx[j]];
            double e = fma(val[j], invec[col_idx[j]], -p);
            double err;
            two_sum(s, p, &s, &err);
            c = c + (err + e);
            a = a + fabs(val[j]) * fabs(invec[col_idx[j]]);
        }
        resvec[i] = s + c;
        if (absrow) absrow[i] = a;
    }
}

/* Accurate A^T g: per output column the same Dot2 accumulation, with the
 * terms visited in CRS storage order. */
void orc_crs_spmv_t_exact(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr,
                          const int32_t *col_idx, const double *val, const double *g,
                          double *out, double *abscol)
{
    double *c = (double *)calloc((size_t)(n_cols > 0 ? n_cols : 1), sizeof(double));
    for (int64_t j = 0; j < n_cols; ++j) { out[j] = 0.0; if (abscol) abscol[j] = 0.0; }
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col_idx[k];
            double p = val[k] * g[i];
            double e = fma(val[k], g[i], -p);
            double err;
            two_sum(out[j], p, &out[j], &err);
            c[j] = c[j] + (err + e);
            if (abscol) abscol[j] = abscol[j] + fabs(val[k]) * fabs(g[i]);
        }
    for (int64_t j = 0; j < n_cols; ++j) out[j] = out[j] + c[j];
    free(c);
}

/* ------------------------------------------------------------------------
 * Adjoint and value gradient (the transpose of the CRS sum).
 * ---------------------------------------------------------------------- */

/* dx = A^T g by a serial scatter over the stored entries. */
void orc_crs_spmv_t(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr,
                    const int32_t *col_idx, const double *val, const double *g,
                    double *dx, int accumulate)
{
    if (!accumulate)
        for (int64_t j = 0; j < n_cols; ++j) dx[j] = 0.0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            dx[col_idx[k]] = dx[col_idx[k]] + val[k] * g[i];
}

/* dval_k = g[row_k] * x[col_k] for every stored entry k (CRS order):
 * the derivative of g . (A x) with respect to val_k. */
void orc_dval(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx,
              const double *g, const double *x, double *dval, int accumulate)
{
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double d = g[i] * x[col_idx[k]];
            dval[k] = accumulate ? dval[k] + d : d;
        }
}

/* ------------------------------------------------------------------------
 * JDS construction (Sect. 2): permute rows (and, in symmetric mode, columns)
 * so that row length decreases with row index, shift every row's entries to
 * the left and store the resulting jagged diagonals one after another.
 *
 *   (i)   len_i = row_ptr[i+1] - row_ptr[i]
 *   (ii)  stable sort by decreasing length: perm[new] = old, iperm[old] = new
 *   (iii) N_j = max len; diagonal d holds the rows with len > d, so
 *         jd_ptr[d+1] - jd_ptr[d] = #{i : len_i > d}
 *   (iv)  val_jds[jd_ptr[d] + r] = val[row_ptr[perm[r]] + d]
 *   (v)   col_jds = iperm[col] (symmetric: A_{p(i),p(j)}) or col (row-only)
 *
 * jd_ptr must hold max_len+1 entries.  Returns N_j, or -1 when symmetric
 * mode is asked for a non-square matrix.
 * ---------------------------------------------------------------------- */
int64_t orc_max_row_len(int64_t n_rows, const int32_t *row_ptr)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t l = (int64_t)row_ptr[i + 1] - row_ptr[i];
        if (l > m) m = l;
    }
    return m;
}

int64_t orc_jds_build(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr,
                      const int32_t *col_idx, const double *val, int symmetric,
                      int32_t *perm, int32_t *iperm, int32_t *jd_ptr,
                      int32_t *col_jds, double *val_jds)
{
    if (symmetric && n_rows != n_cols) return -1;
    int64_t nj = orc_max_row_len(n_rows, row_ptr);

    /* (ii) counting sort on length, longest first, ties in row order */
    int64_t *count = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    int64_t *start = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    for (int64_t i = 0; i < n_rows; ++i) count[row_ptr[i + 1] - row_ptr[i]]++;
    int64_t pos = 0;
    for (int64_t l = nj; l >= 0; --l) { start[l] = pos; pos += count[l]; }
    for (int64_t i = 0; i < n_rows; ++i) {
        int64_t l = (int64_t)row_ptr[i + 1] - row_ptr[i];
        perm[start[l]++] = (int32_t)i;
    }
    for (int64_t r = 0; r < n_rows; ++r) iperm[perm[r]] = (int32_t)r;

    /* (iii) diagonal d has #{len > d} entries */
    jd_ptr[0] = 0;
    for (int64_t d = 0; d < nj; ++d) {
        int64_t rows_longer = 0;
        for (int64_t l = d + 1; l <= nj; ++l) rows_longer += count[l];
        jd_ptr[d + 1] = (int32_t)(jd_ptr[d] + rows_longer);
    }

    /* (iv), (v) shift left and store diagonal after diagonal */
    for (int64_t d = 0; d < nj; ++d)
        for (int64_t r = 0; r < DIAGLEN(jd_ptr, d); ++r) {
            int64_t src = (int64_t)row_ptr[perm[r]] + d;
            val_jds[jd_ptr[d] + r] = val[src];
            col_jds[jd_ptr[d] + r] = symmetric ? iperm[col_idx[src]] : col_idx[src];
        }
    free(count);
    free(start);
    return nj;
}

/* JDS kernel (Sect. 2, JDS listing): diagonal after diagonal, every row of
 * the diagonal updated, resvec making one round trip per diagonal. */
void orc_jds_spmv(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                  const int32_t *col_jds, const double *val_jds, const double *invec,
                  double *resvec, int accumulate)
{
    if (!accumulate)
        for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    for (int64_t d = 0; d < n_diag; ++d) {
        int64_t len = DIAGLEN(jd_ptr, d), off = jd_ptr[d];
        for (int64_t i = 0; i < len; ++i)
            resvec[i] = resvec[i] + val_jds[off + i] * invec[col_jds[off + i]];
    }
}

/* NBJDS (Sect. 2, standard blocking): the diagonals are cut into blocks of
 * `block` rows; one block of resvec is finished for every diagonal that has
 * entries in it before moving on, skipping through val / col_idx. */
void orc_nbjds_spmv(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                    const int32_t *col_jds, const double *val_jds, int64_t block,
                    const double *invec, double *resvec, int accumulate)
{
    if (!accumulate)
        for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    for (int64_t b0 = 0; b0 < n_rows; b0 += block) {
        int64_t b1 = b0 + block < n_rows ? b0 + block : n_rows;
        for (int64_t d = 0; d < n_diag && DIAGLEN(jd_ptr, d) > b0; ++d) {
            int64_t end = DIAGLEN(jd_ptr, d) < b1 ? DIAGLEN(jd_ptr, d) : b1;
            for (int64_t i = b0; i < end; ++i)
                resvec[i] = resvec[i] + val_jds[jd_ptr[d] + i] * invec[col_jds[jd_ptr[d] + i]];
        }
    }
}

/* NUJDS (Sect. 2, outer-loop unrolling): every resvec element is updated by
 * u diagonals at once.  The last group holds the N_j mod u remaining ones. */
void orc_nujds_spmv(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                    const int32_t *col_jds, const double *val_jds, int64_t u,
                    const double *invec, double *resvec, int accumulate)
{
    if (!accumulate)
        for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    for (int64_t d0 = 0; d0 < n_diag; d0 += u) {
        int64_t d1 = d0 + u < n_diag ? d0 + u : n_diag;
        for (int64_t i = 0; i < DIAGLEN(jd_ptr, d0); ++i) {
            double t = resvec[i];
            for (int64_t d = d0; d < d1 && i < DIAGLEN(jd_ptr, d); ++d)
                t = t + val_jds[jd_ptr[d] + i] * invec[col_jds[jd_ptr[d] + i]];
            resvec[i] = t;
        }
    }
}

/* RBJDS layout (Sect. 2): the elements of each block of `block` permuted rows
 * are stored consecutively, diagonal by diagonal inside the block.
 * blk_ptr[k] is the first element of block k (n_blocks+1 entries). */
void orc_rbjds_build(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                     const int32_t *col_jds, const double *val_jds, int64_t block,
                     int32_t *blk_ptr, int32_t *col_rb, double *val_rb)
{
    int64_t pos = 0, k = 0;
    for (int64_t b0 = 0; b0 < n_rows; b0 += block, ++k) {
        int64_t b1 = b0 + block < n_rows ? b0 + block : n_rows;
        blk_ptr[k] = (int32_t)pos;
        for (int64_t d = 0; d < n_diag && DIAGLEN(jd_ptr, d) > b0; ++d) {
            int64_t end = DIAGLEN(jd_ptr, d) < b1 ? DIAGLEN(jd_ptr, d) : b1;
            for (int64_t i = b0; i < end; ++i, ++pos) {
                val_rb[pos] = val_jds[jd_ptr[d] + i];
                col_rb[pos] = col_jds[jd_ptr[d] + i];
            }
        }
    }
    blk_ptr[k] = (int32_t)pos;
}

/* RBJDS kernel: one contiguous sweep through each block's elements. */
void orc_rbjds_spmv(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                    const int32_t *blk_ptr, const int32_t *col_rb, const double *val_rb,
                    int64_t block, const double *invec, double *resvec, int accumulate)
{
    if (!accumulate)
        for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    int64_t k = 0;
    for (int64_t b0 = 0; b0 < n_rows; b0 += block, ++k) {
        int64_t b1 = b0 + block < n_rows ? b0 + block : n_rows;
        int64_t pos = blk_ptr[k];
        for (int64_t d = 0; d < n_diag && DIAGLEN(jd_ptr, d) > b0; ++d) {
            int64_t end = DIAGLEN(jd_ptr, d) < b1 ? DIAGLEN(jd_ptr, d) : b1;
            for (int64_t i = b0; i < end; ++i, ++pos)
                resvec[i] = resvec[i] + val_rb[pos] * invec[col_rb[pos]];
        }
    }
}

/* SOJDS (Sect. 2): inside each block the entries of a row are re-ordered so
 * that each block column (slot d) reads invec at consecutive indices where
 * it can.  Rule used here (the paper fixes none):
 *   - the first row of a block keeps its order;
 *   - for every later row r, slots d = 0, 1, ... are filled in turn with the
 *     not yet placed entry of row r whose column c minimises
 *     |c - (c_prev(d) + 1)|, c_prev(d) being the column now in slot d of row
 *     r-1; ties go to the smaller column, then to the earlier slot.
 * Output is in RBJDS layout (same blk_ptr).  Plain O(len^2) search per row. */
void orc_sojds_build(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr,
                     const int32_t *col_jds, const double *val_jds, int64_t block,
                     int32_t *blk_ptr, int32_t *col_so, double *val_so)
{
    /* row length of permuted row r = number of diagonals longer than r */
    int64_t maxlen = n_diag;
    int32_t *prev_col = (int32_t *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(int32_t));
    int32_t *cur_col = (int32_t *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(int32_t));
    double *cur_val = (double *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(double));
    char *used = (char *)malloc((size_t)(maxlen > 0 ? maxlen : 1));
    int64_t pos = 0, k = 0;
    for (int64_t b0 = 0; b0 < n_rows; b0 += block, ++k) {
        int64_t b1 = b0 + block < n_rows ? b0 + block : n_rows;
        blk_ptr[k] = (int32_t)pos;
        /* block-local element offset of slot d is the count of the block's
         * entries in diagonals before d */
        int64_t nslots = 0;
        while (nslots < n_diag && DIAGLEN(jd_ptr, nslots) > b0) ++nslots;
        int64_t *slot_off = (int64_t *)malloc((size_t)(nslots + 1) * sizeof(int64_t));
        slot_off[0] = 0;
        for (int64_t d = 0; d < nslots; ++d) {
            int64_t end = DIAGLEN(jd_ptr, d) < b1 ? DIAGLEN(jd_ptr, d) : b1;
            slot_off[d + 1] = slot_off[d] + (end - b0);
        }
        for (int64_t r = b0; r < b1; ++r) {
            int64_t len = 0;
            while (len < n_diag && DIAGLEN(jd_ptr, len) > r) ++len;
            for (int64_t d = 0; d < len; ++d) {
                cur_col[d] = col_jds[jd_ptr[d] + r];
                cur_val[d] = val_jds[jd_ptr[d] + r];
                used[d] = 0;
            }
            for (int64_t d = 0; d < len; ++d) {
                int64_t pick;
                if (r == b0) {
                    pick = d;
                } else {
                    int64_t target = (int64_t)prev_col[d] + 1;
                    pick = -1;
                    for (int64_t e = 0; e < len; ++e) {
                        if (used[e]) continue;
                        if (pick < 0) { pick = e; continue; }
                        int64_t de = llabs((int64_t)cur_col[e] - target);
                        int64_t dp = llabs((int64_t)cur_col[pick] - target);
                        if (de < dp || (de == dp && cur_col[e] < cur_col[pick])) pick = e;
                    }
                }
                used[pick] = 1;
                int64_t dst = pos + slot_off[d] + (r - b0);
                col_so[dst] = cur_col[pick];
                val_so[dst] = cur_val[pick];
                prev_col[d] = cur_col[pick];
            }
        }
        pos += slot_off[nslots];
        free(slot_off);
    }
    blk_ptr[k] = (int32_t)pos;
    free(prev_col);
    free(cur_col);
    free(cur_val);
    free(used);
}

/* Vector basis change for the permuted (JDS) basis: out[r] = in[perm[r]]
 * (to the permuted basis) or out[perm[r]] = in[r] (back). */
void orc_permute(int64_t n, const int32_t *perm, const double *in, double *out, int to_permuted)
{
    for (int64_t r = 0; r < n; ++r) {
        if (to_permuted) out[r] = in[perm[r]];
        else out[perm[r]] = in[r];
    }
}

/* ------------------------------------------------------------------------
 * SELL-32-sigma (Kreutzer, Hager, Wellein, Fehske & Bishop, SIAM J. Sci.
 * Comput. 36, 2014): the RBJDS layout with blocks of C = 32 rows, where the
 * decreasing-length row sort is restricted to windows of `window` rows
 * (window a multiple of 32).  With window >= n_rows it is exactly RBJDS with
 * block 32 of the JDS construction above.
 *   perm      stable sort by (window index, decreasing length)
 *   rlen[r]   length of permuted row r
 *   blk_ptr   start of each block of 32 permuted rows
 *   inside a block: slot 0 of the block's rows, then slot 1 of the rows
 *   that have one, ... (rows are sorted inside a block, so those rows are
 *   always the first ones of the block)
 * Columns are renumbered by iperm when `symmetric`.
 * ---------------------------------------------------------------------- */
int orc_sell_build(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr, const int32_t *col_idx,
                   const double *val, int symmetric, int64_t window, int32_t *perm, int32_t *iperm,
                   int32_t *rlen, int32_t *blk_ptr, int32_t *col_out, double *val_out)
{
    if (symmetric && n_rows != n_cols) return -1;
    if (window < 32 || window % 32) return -2;
    int64_t nj = orc_max_row_len(n_rows, row_ptr);
    int64_t *count = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    int64_t *start = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    for (int64_t w0 = 0; w0 < n_rows; w0 += window) {
        int64_t w1 = w0 + window < n_rows ? w0 + window : n_rows;
        for (int64_t l = 0; l <= nj; ++l) count[l] = 0;
        for (int64_t i = w0; i < w1; ++i) count[row_ptr[i + 1] - row_ptr[i]]++;
        int64_t pos = w0;
        for (int64_t l = nj; l >= 0; --l) { start[l] = pos; pos += count[l]; }
        for (int64_t i = w0; i < w1; ++i) perm[start[row_ptr[i + 1] - row_ptr[i]]++] = (int32_t)i;
    }
    for (int64_t r = 0; r < n_rows; ++r) {
        iperm[perm[r]] = (int32_t)r;
        rlen[r] = row_ptr[perm[r] + 1] - row_ptr[perm[r]];
    }
    int64_t nb = (n_rows + 31) / 32, pos = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t b0 = 32 * b, b1 = b0 + 32 < n_rows ? b0 + 32 : n_rows;
        blk_ptr[b] = (int32_t)pos;
        int64_t width = rlen[b0];
        for (int64_t d = 0; d < width; ++d)
            for (int64_t r = b0; r < b1 && rlen[r] > d; ++r, ++pos) {
                int64_t src = (int64_t)row_ptr[perm[r]] + d;
                val_out[pos] = val[src];
                col_out[pos] = symmetric ? iperm[col_idx[src]] : col_idx[src];
            }
    }
    blk_ptr[nb] = (int32_t)pos;
    free(count);
    free(start);
    return 0;
}

/* SELL kernel in the permuted basis: block after block, slot after slot. */
void orc_sell_spmv(int64_t n_rows, const int32_t *rlen, const int32_t *blk_ptr,
                   const int32_t *col_s, const double *val_s, const double *invec, double *resvec)
{
    for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    int64_t nb = (n_rows + 31) / 32;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t b0 = 32 * b, b1 = b0 + 32 < n_rows ? b0 + 32 : n_rows;
        int64_t pos = blk_ptr[b];
        for (int64_t d = 0; d < rlen[b0]; ++d)
            for (int64_t r = b0; r < b1 && rlen[r] > d; ++r, ++pos)
                resvec[r] = resvec[r] + val_s[pos] * invec[col_s[pos]];
    }
}

/* ------------------------------------------------------------------------
 * Basic sparse vector operations (Sect. 4.1, the table of ADD and SCP
 * kernels): one running sum over i < n of
 *     ADD:  s = s + B(idx(i))          SCP:  s = s + A(i) * B(idx(i))
 * with idx(i) = i (PD, packed dense), k*i (CS, constant stride computed in
 * the loop) or ind(i) (IS / IR, indirect: the two differ only in how ind
 * was generated).  op: 0 = ADD, 1 = SCP.  access: 0 = PD, 1 = CS, 2 = IND.
 * ---------------------------------------------------------------------- */
static inline int64_t gather_index(int access, int64_t i, int64_t k, const int32_t *ind)
{
    return access == 0 ? i : (access == 1 ? k * i : (int64_t)ind[i]);
}

double orc_gather_sum(int op, int access, int64_t n, int64_t k, const double *a,
                      const double *b, const int32_t *ind)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double bj = b[gather_index(access, i, k, ind)];
        s = op == 0 ? s + bj : s + a[i] * bj;
    }
    return s;
}

/* The same sum, accurately (Dot2: exact product split and TwoSum, as in
 * orc_crs_spmv_exact).  out[0] = the sum, out[1] = sum of |term|. */
void orc_gather_sum_exact(int op, int access, int64_t n, int64_t k, const double *a,
                          const double *b, const int32_t *ind, double *out)
{
    double s = 0.0, c = 0.0, abs_sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double bj = b[gather_index(access, i, k, ind)];
        double p = op == 0 ? bj : a[i] * bj;
        double e = op == 0 ? 0.0 : fma(a[i], bj, -p);
        double err;
        two_sum(s, p, &s, &err);
        c = c + (err + e);
        abs_sum = abs_sum + fabs(p);
    }
    out[0] = s + c;
    out[1] = abs_sum;
}

/* ------------------------------------------------------------------------
 * Stride distribution of the invec accesses (Sect. 4.2, Fig. 4a): walking a
 * column-index array in storage order -- the order in which the paper's
 * serial CRS, JDS, RBJDS and SOJDS loops read invec -- every jump
 * s = col[i+1] - col[i] is counted once.  Bins by size: bin 0 holds s = 0,
 * bin b >= 1 holds 2^(b-1) <= |s| < 2^b (for 8-byte elements: strides of
 * 8*2^(b-1) to 8*2^b - 1 bytes).  hist[0..32] counts forward jumps (s >= 0),
 * hist[33..65] backward jumps (s < 0; bin 0 stays empty).
 * ---------------------------------------------------------------------- */
static int stride_bin(int64_t s)
{
    uint64_t a = (uint64_t)(s < 0 ? -s : s);
    int b = 0;
    while (a) {
        ++b;
        a >>= 1;
    }
    return b;
}

void orc_stride_hist(int64_t nnz, const int32_t *col, int64_t *hist)
{
    for (int i = 0; i < 66; ++i) hist[i] = 0;
    for (int64_t i = 0; i + 1 < nnz; ++i) {
        int64_t s = (int64_t)col[i + 1] - (int64_t)col[i];
        hist[(s < 0 ? 33 : 0) + stride_bin(s)] += 1;
    }
}

/* Distinct 32-byte sectors of invec touched by one warp-wide gather: the
 * columns cols[0..m) of the active lanes, elem_bytes per entry. */
static int64_t distinct_sectors(const int64_t *cols, int m, int elem_bytes)
{
    int64_t seen[32];
    int n = 0;
    for (int l = 0; l < m; ++l) {
        int64_t sec = cols[l] * elem_bytes / 32;
        int dup = 0;
        for (int q = 0; q < n; ++q) dup |= seen[q] == sec;
        if (!dup) seen[n++] = sec;
    }
    return n;
}

/* Sectors per warp-wide gather, histogram hist[0..32] (hist[c] = number of
 * warp accesses touching c distinct sectors), for the warp access patterns
 * of the GPU kernels:
 *   CRS, `lanes` lanes per row: a warp holds 32/lanes consecutive rows; at
 *     step t lane l of row group g reads entry row_ptr[r] + t*lanes + l.
 *   JDS storage, thread per permuted row: a warp holds 32 consecutive rows;
 *     for diagonal d it reads jd_ptr[d] + r for its rows r < diagLen(d).
 *   SELL-32: a warp holds one 32-row block; slot d is read by the rows
 *     with rlen > d, from consecutive storage. */
void orc_warp_sectors_crs(int64_t n_rows, const int32_t *row_ptr, const int32_t *col, int lanes,
                          int elem_bytes, int64_t *hist)
{
    int groups = 32 / lanes;
    for (int i = 0; i < 33; ++i) hist[i] = 0;
    for (int64_t r0 = 0; r0 < n_rows; r0 += groups) {
        int64_t maxlen = 0;
        for (int g = 0; g < groups && r0 + g < n_rows; ++g) {
            int64_t len = row_ptr[r0 + g + 1] - row_ptr[r0 + g];
            if (len > maxlen) maxlen = len;
        }
        for (int64_t t = 0; t * lanes < maxlen; ++t) {
            int64_t cols[32];
            int m = 0;
            for (int g = 0; g < groups && r0 + g < n_rows; ++g)
                for (int l = 0; l < lanes; ++l) {
                    int64_t e = (int64_t)row_ptr[r0 + g] + t * lanes + l;
                    if (e < row_ptr[r0 + g + 1]) cols[m++] = col[e];
                }
            if (m) hist[distinct_sectors(cols, m, elem_bytes)] += 1;
        }
    }
}

void orc_warp_sectors_jds(int64_t n_rows, int64_t n_diag, const int32_t *jd_ptr, const int32_t *col,
                          int elem_bytes, int64_t *hist)
{
    for (int i = 0; i < 33; ++i) hist[i] = 0;
    for (int64_t r0 = 0; r0 < n_rows; r0 += 32)
        for (int64_t d = 0; d < n_diag && DIAGLEN(jd_ptr, d) > r0; ++d) {
            int64_t cols[32];
            int m = 0;
            for (int64_t r = r0; r < r0 + 32 && r < DIAGLEN(jd_ptr, d); ++r) cols[m++] = col[jd_ptr[d] + r];
            hist[distinct_sectors(cols, m, elem_bytes)] += 1;
        }
}

void orc_warp_sectors_sell(int64_t n_rows, const int32_t *rlen, const int32_t *blk_ptr, const int32_t *col,
                           int elem_bytes, int64_t *hist)
{
    for (int i = 0; i < 33; ++i) hist[i] = 0;
    int64_t nb = (n_rows + 31) / 32;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t b0 = 32 * b, b1 = b0 + 32 < n_rows ? b0 + 32 : n_rows;
        int64_t pos = blk_ptr[b];
        for (int64_t d = 0; d < rlen[b0]; ++d) {
            int64_t cols[32];
            int m = 0;
            for (int64_t r = b0; r < b1 && rlen[r] > d; ++r, ++pos) cols[m++] = col[pos];
            hist[distinct_sectors(cols, m, elem_bytes)] += 1;
        }
    }
}

/* ------------------------------------------------------------------------
 * Paired SELL (a GB300 layout of this library, not the paper's): the rows of
 * every window of `window` rows (a multiple of 64) are sorted by decreasing
 * length (stable), and the row of rank q is paired with the row of rank
 * m-1-q (m = rows in the window), so that one lane walks a long row and a
 * short one: lane q < ceil(m/2) owns row a = rank q and, when m-1-q > q,
 * row b = rank m-1-q.  Lanes form blocks of 32 consecutive lanes of a
 * window; block g (counted over the whole matrix) owns the permuted rows
 * 64g .. 64g+R-1 (R = min(64, n - 64g)): with L = ceil(R/2) lanes, the
 * a-row of lane p is permuted row 64g + p and its b-row, if any,
 * 64g + L + p.  Storage of block g, slot by slot: slot t holds, in lane
 * order, every lane whose total length len_a + len_b exceeds t, with entry
 * t of the lane's concatenated rows (row a's entries, then row b's).
 * Returns 0, -1 (symmetric and not square) or -2 (bad window).
 * ---------------------------------------------------------------------- */
int orc_psell_build(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr, const int32_t *col_idx,
                    const double *val, int symmetric, int64_t window, int32_t *perm, int32_t *iperm,
                    int32_t *rlen, int32_t *blk_ptr, int32_t *col_out, double *val_out)
{
    if (symmetric && n_rows != n_cols) return -1;
    if (window < 64 || window % 64) return -2;
    int64_t nj = orc_max_row_len(n_rows, row_ptr);
    int64_t *count = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    int64_t *start = (int64_t *)calloc((size_t)(nj + 2), sizeof(int64_t));
    int32_t *sorted = (int32_t *)malloc((size_t)(window > 0 ? window : 1) * sizeof(int32_t));
    for (int64_t w0 = 0; w0 < n_rows; w0 += window) {
        int64_t w1 = w0 + window < n_rows ? w0 + window : n_rows, m = w1 - w0;
        /* stable counting sort of the window by decreasing length */
        for (int64_t l = 0; l <= nj; ++l) count[l] = 0;
        for (int64_t i = w0; i < w1; ++i) count[row_ptr[i + 1] - row_ptr[i]]++;
        int64_t pos = 0;
        for (int64_t l = nj; l >= 0; --l) { start[l] = pos; pos += count[l]; }
        for (int64_t i = w0; i < w1; ++i) sorted[start[row_ptr[i + 1] - row_ptr[i]]++] = (int32_t)i;
        /* pair rank q with rank m-1-q; place the rows by block */
        int64_t lanes = (m + 1) / 2;
        for (int64_t q = 0; q < lanes; ++q) {
            int64_t g = w0 / 64 + q / 32, p = q % 32;
            int64_t R = n_rows - 64 * g < 64 ? n_rows - 64 * g : 64, L = (R + 1) / 2;
            perm[64 * g + p] = sorted[q];
            if (m - 1 - q > q) perm[64 * g + L + p] = sorted[m - 1 - q];
        }
    }
    for (int64_t r = 0; r < n_rows; ++r) {
        iperm[perm[r]] = (int32_t)r;
        rlen[r] = row_ptr[perm[r] + 1] - row_ptr[perm[r]];
    }
    int64_t nb = (n_rows + 63) / 64, pos = 0;
    for (int64_t g = 0; g < nb; ++g) {
        int64_t R = n_rows - 64 * g < 64 ? n_rows - 64 * g : 64, L = (R + 1) / 2;
        int64_t width = 0;
        for (int64_t p = 0; p < L; ++p) {
            int64_t tot = rlen[64 * g + p] + (L + p < R ? rlen[64 * g + L + p] : 0);
            if (tot > width) width = tot;
        }
        blk_ptr[g] = (int32_t)pos;
        for (int64_t t = 0; t < width; ++t)
            for (int64_t p = 0; p < L; ++p) {
                int64_t ra = 64 * g + p, rb = 64 * g + L + p;
                int64_t la = rlen[ra], lb = L + p < R ? rlen[rb] : 0;
                if (t >= la + lb) continue;
                int64_t src = t < la ? (int64_t)row_ptr[perm[ra]] + t : (int64_t)row_ptr[perm[rb]] + (t - la);
                val_out[pos] = val[src];
                col_out[pos] = symmetric ? iperm[col_idx[src]] : col_idx[src];
                ++pos;
            }
    }
    blk_ptr[nb] = (int32_t)pos;
    free(count);
    free(start);
    free(sorted);
    return 0;
}

/* Paired SELL product in the permuted basis: block after block, slot after
 * slot, every lane adding its slot-t entry to the row it is in. */
void orc_psell_spmv(int64_t n_rows, const int32_t *rlen, const int32_t *blk_ptr,
                    const int32_t *col_s, const double *val_s, const double *invec, double *resvec)
{
    for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    int64_t nb = (n_rows + 63) / 64;
    for (int64_t g = 0; g < nb; ++g) {
        int64_t R = n_rows - 64 * g < 64 ? n_rows - 64 * g : 64, L = (R + 1) / 2;
        int64_t width = 0;
        for (int64_t p = 0; p < L; ++p) {
            int64_t tot = rlen[64 * g + p] + (L + p < R ? rlen[64 * g + L + p] : 0);
            if (tot > width) width = tot;
        }
        int64_t pos = blk_ptr[g];
        for (int64_t t = 0; t < width; ++t)
            for (int64_t p = 0; p < L; ++p) {
                int64_t ra = 64 * g + p, rb = 64 * g + L + p;
                int64_t la = rlen[ra], lb = L + p < R ? rlen[rb] : 0;
                if (t >= la + lb) continue;
                int64_t r = t < la ? ra : rb;
                resvec[r] = resvec[r] + val_s[pos] * invec[col_s[pos]];
                ++pos;
            }
    }
}

/* ------------------------------------------------------------------------
 * Symmetric SpMVM from the upper triangle (Sect. 4.2 names the option of
 * using the symmetry of the Hamiltonian to save data transfer and does not
 * pursue it).  U holds the entries with col >= row of a symmetric A, so
 * A = U + U^T - diag(U):
 *     y_i = sum_{j>=i} u_ij x_j + sum_{k<i} u_ki x_k.
 * The loop walks U row by row; every off-diagonal u_ij adds u_ij x_j to
 * y_i and u_ij x_i to y_j.
 * ---------------------------------------------------------------------- */
int64_t orc_upper_count(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) c += col_idx[e] >= i;
    return c;
}

void orc_upper_extract(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                       int32_t *row_ptr_u, int32_t *col_u, double *val_u)
{
    int64_t pos = 0;
    row_ptr_u[0] = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] >= i) {
                col_u[pos] = col_idx[e];
                val_u[pos] = val[e];
                ++pos;
            }
        row_ptr_u[i + 1] = (int32_t)pos;
    }
}

void orc_sym_spmv(int64_t n_rows, const int32_t *row_ptr_u, const int32_t *col_u, const double *val_u,
                  const double *invec, double *resvec)
{
    for (int64_t i = 0; i < n_rows; ++i) resvec[i] = 0.0;
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t e = row_ptr_u[i]; e < row_ptr_u[i + 1]; ++e) {
            int64_t j = col_u[e];
            resvec[i] = resvec[i] + val_u[e] * invec[j];
            if (j != i) resvec[j] = resvec[j] + val_u[e] * invec[i];
        }
}

/* ------------------------------------------------------------------------
 * Hybrid storage (Sect. 4.2: most entries of the Hamiltonian sit in a few
 * dense outer secondary diagonals, any of which could be stored densely):
 * selected diagonals in DIA form, the rest in CRS.
 *
 * Diagonal of offset o = col - row; its length is the number of in-matrix
 * positions (i, i+o).  fill(o) = entries with offset o / length.  The
 * offsets with fill >= min_fill are ranked by entry count (descending),
 * then |o|, then o, and the first max_diags are kept.  DIA values:
 * dia[k*n_rows + i] = the first entry (CRS order) of row i with offset o_k,
 * 0 where none.  Every other entry stays in the remainder CRS, in CRS order.
 * Product: y_i = (sum over k ascending of dia[k][i] x[i+o_k], in-range
 * columns only) + (the remainder row's sum in CRS order).
 * ---------------------------------------------------------------------- */
static int64_t diag_length(int64_t n_rows, int64_t n_cols, int64_t o)
{
    int64_t lo = o < 0 ? -o : 0;                              /* first row */
    int64_t hi = n_rows < n_cols - o ? n_rows : n_cols - o;   /* one past the last row */
    return hi > lo ? hi - lo : 0;
}

/* Selected offsets into offs_out (at most max_diags); returns their number. */
int64_t orc_dia_select(int64_t n_rows, int64_t n_cols, const int32_t *row_ptr, const int32_t *col_idx,
                       int64_t max_diags, double min_fill, int32_t *offs_out)
{
    int64_t span = n_rows + n_cols;  /* offsets -(n_rows-1) .. n_cols-1 */
    int64_t *cnt = (int64_t *)calloc((size_t)(span > 0 ? span : 1), sizeof(int64_t));
    for (int64_t i = 0; i < n_rows; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) cnt[(int64_t)col_idx[e] - i + n_rows] += 1;
    int64_t m = 0;
    for (int64_t k = 0; k < max_diags; ++k) {
        /* the best remaining offset by (count desc, |o| asc, o asc) */
        int64_t best = -1;
        for (int64_t b = 0; b < span; ++b) {
            if (cnt[b] <= 0) continue;
            int64_t o = b - n_rows;
            if ((double)cnt[b] < min_fill * (double)diag_length(n_rows, n_cols, o)) continue;
            if (best < 0) { best = b; continue; }
            int64_t ob = best - n_rows;
            int64_t ao = o < 0 ? -o : o, aob = ob < 0 ? -ob : ob;
            if (cnt[b] > cnt[best] || (cnt[b] == cnt[best] && (ao < aob || (ao == aob && o < ob)))) best = b;
        }
        if (best < 0) break;
        offs_out[m++] = (int32_t)(best - n_rows);
        cnt[best] = 0;
    }
    free(cnt);
    return m;
}

/* DIA values [n_diags][n_rows] and the remainder CRS (row_ptr_rem [n_rows+1],
 * col_rem / val_rem sized for nnz); returns the remainder's entry count. */
int64_t orc_dia_build(int64_t n_rows, const int32_t *row_ptr, const int32_t *col_idx, const double *val,
                      int64_t n_diags, const int32_t *offs, double *dia, int32_t *row_ptr_rem,
                      int32_t *col_rem, double *val_rem)
{
    for (int64_t q = 0; q < n_diags * n_rows; ++q) dia[q] = 0.0;
    char *taken = (char *)calloc((size_t)(n_diags > 0 ? n_diags : 1), 1);
    int64_t pos = 0;
    row_ptr_rem[0] = 0;
    for (int64_t i = 0; i < n_rows; ++i) {
        for (int64_t k = 0; k < n_diags; ++k) taken[k] = 0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t o = (int64_t)col_idx[e] - i, k = 0;
            while (k < n_diags && (offs[k] != o || taken[k])) ++k;
            if (k < n_diags) {
                dia[k * n_rows + i] = val[e];
                taken[k] = 1;
            } else {
                col_rem[pos] = col_idx[e];
                val_rem[pos] = val[e];
                ++pos;
            }
        }
        row_ptr_rem[i + 1] = (int32_t)pos;
    }
    free(taken);
    return pos;
}

void orc_dia_spmv(int64_t n_rows, int64_t n_cols, int64_t n_diags, const int32_t *offs, const double *dia,
                  const int32_t *row_ptr_rem, const int32_t *col_rem, const double *val_rem,
                  const double *invec, double *resvec)
{
    for (int64_t i = 0; i < n_rows; ++i) {
        double d = 0.0;
        for (int64_t k = 0; k < n_diags; ++k) {
            int64_t j = i + offs[k];
            if (j >= 0 && j < n_cols) d = d + dia[k * n_rows + i] * invec[j];
        }
        double r = 0.0;
        for (int64_t e = row_ptr_rem[i]; e < row_ptr_rem[i + 1]; ++e) r = r + val_rem[e] * invec[col_rem[e]];
        resvec[i] = d + r;
    }
}
