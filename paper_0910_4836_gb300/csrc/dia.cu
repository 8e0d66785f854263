// Hybrid storage: dense secondary diagonals in DIA form, the rest in a
// remainder matrix.  Sect. 4.2 observes that most entries of the
// Holstein-Hubbard matrix lie in a few dense outer secondary diagonals, each
// a candidate for a dense storage scheme, and leaves the hybrid unbuilt.
//
// A DIA diagonal stores one value per row (zeros where the diagonal has no
// entry) and no column index, so for FP64 it moves fewer bytes than CRS
// once more than 2/3 of its positions are filled (8 B a slot against 12 B an
// entry).  Its x accesses are contiguous, so a warp's gather is 2 or 3
// sectors instead of up to 32.
//
// Plan: an exact offset histogram on the device (integer atomics,
// warp-aggregated), read back once; the selection of offsets by fill is a
// host decision (same rule and precision as the oracle); then the remainder
// row counts and their scan.  Build: the DIA array and the remainder CRS.
// Product: thread per row, y_i = sum over the diagonals in rank order of
// dia[k][i] x[i+o_k] (in-range columns), added to y when accumulating; the
// remainder is applied after it by any product kernel with accumulate = 1.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "accum.cuh"

namespace gbsp {

namespace {

__global__ void offset_hist_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, int32_t *hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = i < n_rows;
    const int64_t e0 = ok ? row_ptr[i] : 0, e1 = ok ? row_ptr[i + 1] : 0;
    const unsigned len = (unsigned)(e1 - e0);
    const unsigned maxlen = __reduce_max_sync(0xffffffffu, len);
    const int lane = threadIdx.x & 31;
    for (unsigned t = 0; t < maxlen; ++t) {
        const bool act = t < len;
        // bin = col - row + n_rows (>= 1); inactive lanes carry a key of their own
        const long long key = act ? (long long)col[e0 + t] - i + n_rows : -1 - (long long)lane;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (act && (__ffs(grp) - 1) == lane) atomicAdd(hist + key, (int32_t)__popc(grp));
    }
}

// Entries of row i that stay in the remainder: every entry except, per
// selected offset, the first one of the row (CRS order) on that diagonal.
__device__ __forceinline__ int dia_slot(int64_t o, const int32_t *offs, int nd, uint64_t taken) {
    for (int k = 0; k < nd; ++k)
        if (offs[k] == o && !((taken >> k) & 1ull)) return k;
    return -1;
}

__global__ void dia_rem_count_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col, const int32_t *__restrict__ offs, int nd,
                                     int32_t *cnt) {
    __shared__ int32_t so[64];
    for (int k = threadIdx.x; k < nd; k += blockDim.x) so[k] = offs[k];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    uint64_t taken = 0;
    int32_t c = 0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int k = dia_slot((int64_t)col[e] - i, so, nd, taken);
        if (k >= 0) taken |= 1ull << k;
        else ++c;
    }
    cnt[i] = c;
}

template <typename T>
__global__ void dia_fill_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                const T *__restrict__ val, const int32_t *__restrict__ offs, int nd,
                                const int32_t *__restrict__ row_ptr_rem, T *dia, int32_t *col_rem, T *val_rem) {
    __shared__ int32_t so[64];
    for (int k = threadIdx.x; k < nd; k += blockDim.x) so[k] = offs[k];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    uint64_t taken = 0;
    int64_t pos = row_ptr_rem[i];
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int k = dia_slot((int64_t)col[e] - i, so, nd, taken);
        if (k >= 0) {
            taken |= 1ull << k;
            dia[(int64_t)k * n_rows + i] = val[e];
        } else {
            col_rem[pos] = col[e];
            val_rem[pos] = val[e];
            ++pos;
        }
    }
}

// thread per row; the loads of U diagonals are issued together
template <int VM, int U>
__global__ void __launch_bounds__(256) dia_kernel(int64_t n_rows, int64_t n_cols, int nd,
                                                  const int32_t *__restrict__ offs, const void *dia_v,
                                                  const void *x_v, void *y_v, int accumulate) {
    typedef typename ValT<VM>::T T;
    __shared__ int32_t so[64];
    for (int k = threadIdx.x; k < nd; k += blockDim.x) so[k] = offs[k];
    __syncthreads();
    const T *__restrict__ dia = static_cast<const T *>(dia_v);
    const T *__restrict__ x = static_cast<const T *>(x_v);
    T *__restrict__ y = static_cast<T *>(y_v);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows; i += stride) {
        Acc<VM> acc;
        acc.init();
        for (int k0 = 0; k0 < nd; k0 += U) {
            T a[U], b[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = k0 + u;
                const int64_t j = k < nd ? i + so[k] : -1;
                ok[u] = j >= 0 && j < n_cols;
                a[u] = ok[u] ? ld_stream(dia + (int64_t)k * n_rows + i) : T(0);
                b[u] = ok[u] ? ld_vec(x + j) : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) acc.add(a[u], b[u]);
        }
        if (accumulate) acc.add_value(y[i]);
        y[i] = acc.result();
    }
}

}  // namespace

gbsp_status dia_launch(const Mat &A, const VecArgs &v, cudaStream_t s) {
    if (v.k != 1 || v.ldx != 1 || v.ldy != 1) {
        set_error("gbsp_spmm: DIA handles take one right-hand side");
        return GBSP_ERR_UNSUPPORTED;
    }
    if (A.n_rows == 0) return GBSP_OK;
    const int nd = (int)A.n_diag;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(A.n_rows, 256), (int64_t)num_sms() * 8));
    const int VMv = A.dtype == GBSP_F64 ? VM_F64 : (A.kopt.accum == GBSP_ACC_COMPENSATED ? VM_F32C : VM_F32);
    if (VMv == VM_F64)
        dia_kernel<VM_F64, 4><<<(unsigned)grid, 256, 0, s>>>(A.n_rows, A.n_cols, nd, A.col, A.val, v.x, v.y,
                                                              v.accumulate);
    else if (VMv == VM_F32C)
        dia_kernel<VM_F32C, 4><<<(unsigned)grid, 256, 0, s>>>(A.n_rows, A.n_cols, nd, A.col, A.val, v.x, v.y,
                                                               v.accumulate);
    else
        dia_kernel<VM_F32, 4><<<(unsigned)grid, 256, 0, s>>>(A.n_rows, A.n_cols, nd, A.col, A.val, v.x, v.y,
                                                              v.accumulate);
    GBSP_LAUNCH_CHECK("dia_kernel");
    return GBSP_OK;
}

}  // namespace gbsp

using namespace gbsp;

static int64_t dia_diag_length(int64_t n_rows, int64_t n_cols, int64_t o) {
    const int64_t lo = o < 0 ? -o : 0, hi = std::min(n_rows, n_cols - o);
    return hi > lo ? hi - lo : 0;
}

extern "C" gbsp_status gbsp_dia_plan_workspace(gbsp_handle crs, int64_t *bytes) {
    if (!crs || !bytes || crs->kind != KIND_CRS) return arg_error("gbsp_dia_plan_workspace: needs a CRS handle");
    const int64_t span = crs->n_rows + crs->n_cols + 1;
    *bytes = ((4 * span + 255) & ~int64_t(255)) + ((4 * (crs->n_rows + 1) + 255) & ~int64_t(255)) + 256 +
             std::max<int64_t>(scan_ws_bytes(crs->n_rows + 1), 256);
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_dia_plan(gbsp_handle crs, int32_t max_diags, double min_fill, int32_t *d_row_ptr_rem,
                                     void *d_ws, int64_t ws_bytes, void *stream, gbsp_dia_sizes *out) {
    if (!crs || !out || !d_row_ptr_rem || crs->kind != KIND_CRS) return arg_error("gbsp_dia_plan: bad arguments");
    if (max_diags < 0 || max_diags > GBSP_DIA_MAX) return arg_error("gbsp_dia_plan: max_diags must be in 0..64");
    if (!(min_fill >= 0.0)) return arg_error("gbsp_dia_plan: min_fill must be >= 0");
    int64_t need = 0;
    gbsp_dia_plan_workspace(crs, &need);
    if (!d_ws || ws_bytes < need) return arg_error("gbsp_dia_plan: workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = crs->n_rows, span = crs->n_rows + crs->n_cols + 1;
    char *p = static_cast<char *>(d_ws);
    int32_t *hist = reinterpret_cast<int32_t *>(p);
    p += (4 * span + 255) & ~int64_t(255);
    int32_t *cnt = reinterpret_cast<int32_t *>(p);
    p += (4 * (n + 1) + 255) & ~int64_t(255);
    int32_t *d_offs = reinterpret_cast<int32_t *>(p);
    p += 256;
    int32_t *scan_ws = reinterpret_cast<int32_t *>(p);

    // 1. offset histogram, read back
    GBSP_CUDA(cudaMemsetAsync(hist, 0, 4 * span, s));
    if (n > 0) {
        offset_hist_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, crs->row_ptr, crs->col, hist);
        GBSP_LAUNCH_CHECK("offset_hist_kernel");
    }
    std::vector<int32_t> h(span);
    GBSP_CUDA(cudaMemcpyAsync(h.data(), hist, 4 * span, cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));

    // 2. selection: fill >= min_fill, ranked by (count desc, |o| asc, o asc)
    struct Cand {
        int64_t count, o;
    };
    std::vector<Cand> cand;
    for (int64_t b = 0; b < span; ++b) {
        if (h[b] <= 0) continue;
        const int64_t o = b - n;
        if ((double)h[b] < min_fill * (double)dia_diag_length(n, crs->n_cols, o)) continue;
        cand.push_back(Cand{h[b], o});
    }
    std::sort(cand.begin(), cand.end(), [](const Cand &a, const Cand &b) {
        const int64_t aa = a.o < 0 ? -a.o : a.o, ab = b.o < 0 ? -b.o : b.o;
        if (a.count != b.count) return a.count > b.count;
        if (aa != ab) return aa < ab;
        return a.o < b.o;
    });
    const int nd = (int)std::min<int64_t>((int64_t)cand.size(), max_diags);
    std::memset(out, 0, sizeof(*out));
    out->n_rows = n;
    out->n_cols = crs->n_cols;
    out->n_diags = nd;
    for (int k = 0; k < nd; ++k) out->offsets[k] = (int32_t)cand[k].o;

    // 3. remainder row counts -> row_ptr_rem
    if (nd > 0) GBSP_CUDA(cudaMemcpyAsync(d_offs, out->offsets, 4 * nd, cudaMemcpyHostToDevice, s));
    if (n > 0) {
        dia_rem_count_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, crs->row_ptr, crs->col, d_offs, nd, cnt);
        GBSP_LAUNCH_CHECK("dia_rem_count_kernel");
    }
    gbsp_status st = scan_exclusive(cnt, n, d_row_ptr_rem, d_row_ptr_rem + n, scan_ws, s);
    if (st != GBSP_OK) return st;
    int32_t rem = 0;
    GBSP_CUDA(cudaMemcpyAsync(&rem, d_row_ptr_rem + n, 4, cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    out->nnz_rem = rem;
    out->nnz_dia = crs->nnz - rem;
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_dia_build(gbsp_handle crs, const gbsp_dia_sizes *sz, void *d_dia, int32_t *d_offsets,
                                      const int32_t *d_row_ptr_rem, int32_t *d_col_rem, void *d_val_rem,
                                      void *stream, gbsp_handle *dia_out, gbsp_handle *rem_out) {
    if (!crs || !sz || !dia_out || !rem_out || !d_row_ptr_rem || crs->kind != KIND_CRS)
        return arg_error("gbsp_dia_build: bad arguments");
    if (sz->n_rows != crs->n_rows || sz->n_cols != crs->n_cols || sz->n_diags < 0 || sz->n_diags > GBSP_DIA_MAX ||
        sz->nnz_rem + sz->nnz_dia != crs->nnz)
        return arg_error("gbsp_dia_build: sizes do not come from this matrix");
    const int nd = sz->n_diags;
    const int64_t n = crs->n_rows;
    if ((nd > 0 && (!d_dia || !d_offsets)) || (sz->nnz_rem > 0 && (!d_col_rem || !d_val_rem)))
        return arg_error("gbsp_dia_build: a required buffer is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = crs->dtype == GBSP_F64 ? 8 : 4;
    if (nd > 0) {
        GBSP_CUDA(cudaMemcpyAsync(d_offsets, sz->offsets, 4 * nd, cudaMemcpyHostToDevice, s));
        GBSP_CUDA(cudaMemsetAsync(d_dia, 0, es * nd * n, s));
    }
    if (n > 0) {
        if (crs->dtype == GBSP_F64)
            dia_fill_kernel<double><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                n, crs->row_ptr, crs->col, static_cast<const double *>(crs->val), d_offsets, nd, d_row_ptr_rem,
                static_cast<double *>(d_dia), d_col_rem, static_cast<double *>(d_val_rem));
        else
            dia_fill_kernel<float><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(
                n, crs->row_ptr, crs->col, static_cast<const float *>(crs->val), d_offsets, nd, d_row_ptr_rem,
                static_cast<float *>(d_dia), d_col_rem, static_cast<float *>(d_val_rem));
        GBSP_LAUNCH_CHECK("dia_fill_kernel");
    }
    GBSP_CUDA(cudaStreamSynchronize(s));  // sz->offsets is read by the copy above
    gbsp_status st = gbsp_crs_create(n, crs->n_cols, sz->nnz_rem, d_row_ptr_rem, d_col_rem, d_val_rem,
                                     (gbsp_dtype)crs->dtype, rem_out);
    if (st != GBSP_OK) return st;
    gbsp_mat *D = new (std::nothrow) gbsp_mat();
    if (!D) {
        gbsp_destroy(*rem_out);
        *rem_out = nullptr;
        return arg_error("gbsp_dia_build: out of host memory");
    }
    D->kind = KIND_DIA;
    D->n_rows = n;
    D->n_cols = crs->n_cols;
    D->nnz = sz->nnz_dia;
    D->dtype = crs->dtype;
    D->device = crs->device;
    D->val = d_dia;
    D->col = d_offsets;  // the diagonal offsets
    D->n_diag = nd;
    D->format = GBSP_CRS;
    D->kopt = crs->kopt;
    *dia_out = D;
    return GBSP_OK;
}
