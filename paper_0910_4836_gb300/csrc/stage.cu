// Shared-memory staging of x for SELL handles (GB300 addition; the paper's
// CPU kernels rely on the caches).  On GB300 the L1TEX stage handles about
// one distinct cache line per clock for a gather, so a 32-lane gather that
// touches 26 lines costs 26 clocks however few bytes it needs.  For banded
// matrices most gathers of a 1024-row group fall into a few 1024-entry
// pages of x; copying those pages into shared memory with coalesced loads
// (2 lines per 32 entries) and reading the gathers from there removes most
// of that cost.
//
// Build: per entry the key (group, page of its column); a stable radix sort
// of the keys; per group the pages with the most references (at least
// min_refs, ties to the smaller page) up to pages_per_group; the columns
// re-encoded, a staged one as ~(slot * 1024 + col % 1024).  All exact
// integer work, deterministic.
#include <algorithm>

#include "internal.cuh"
#include "accum.cuh"

namespace gbsp {

namespace {

constexpr int kPage = 1024;       // x entries per page (the product kernel's kStagePage)
constexpr int kPageShift = 10;
constexpr int kGroupBlocks = 32;  // SELL blocks (32 rows each) per group
constexpr int kMaxPages = 16;

int bits_of(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

// warp per SELL block: the key of every entry
__global__ void stage_keys_kernel(int64_t nb, const int32_t *__restrict__ blk_ptr, const int32_t *__restrict__ col,
                                  int pbits, uint32_t *keys) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const uint32_t g = (uint32_t)(b / kGroupBlocks);
    for (int64_t e = blk_ptr[b] + (threadIdx.x & 31); e < blk_ptr[b + 1]; e += 32)
        keys[e] = (g << pbits) | (uint32_t)(col[e] >> kPageShift);
}

__device__ int64_t lower_bound_u32(const uint32_t *a, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((uint64_t)a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// thread per group: walk the group's sorted keys run by run and keep the
// P pages with the most references
__global__ void stage_select_kernel(int64_t ngroups, const uint32_t *__restrict__ ks, int64_t nnz, int pbits, int P,
                                    int32_t min_refs, int32_t *pages) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const uint32_t mask = (1u << pbits) - 1u;
    int64_t i = lower_bound_u32(ks, nnz, (uint64_t)g << pbits);
    const int64_t hi = lower_bound_u32(ks, nnz, (uint64_t)(g + 1) << pbits);
    int32_t tp[kMaxPages], tc[kMaxPages];
    int m = 0;
    while (i < hi) {
        const uint32_t k = ks[i];
        int64_t j = i + 1;
        while (j < hi && ks[j] == k) ++j;
        const int32_t cnt = (int32_t)(j - i);
        i = j;
        if (cnt < min_refs) continue;
        // runs come in increasing page order: a later page displaces a kept
        // one only with strictly more references
        if (m == P && cnt <= tc[P - 1]) continue;
        int q = m < P ? m++ : P - 1;
        while (q > 0 && tc[q - 1] < cnt) {
            tc[q] = tc[q - 1];
            tp[q] = tp[q - 1];
            --q;
        }
        tc[q] = cnt;
        tp[q] = (int32_t)(k & mask);
    }
    for (int t = 0; t < P; ++t) pages[g * P + t] = t < m ? tp[t] : -1;
}

// warp per SELL block: re-encode the columns that fall into a staged page
__global__ void stage_encode_kernel(int64_t nb, const int32_t *__restrict__ blk_ptr, const int32_t *__restrict__ col,
                                    const int32_t *__restrict__ pages, int P, int32_t *col_st) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;
    const int64_t g = b / kGroupBlocks;
    int32_t pg[kMaxPages];
#pragma unroll
    for (int t = 0; t < kMaxPages; ++t) pg[t] = t < P ? __ldg(pages + g * P + t) : -1;
    for (int64_t e = blk_ptr[b] + (threadIdx.x & 31); e < blk_ptr[b + 1]; e += 32) {
        const int32_t c = col[e], page = c >> kPageShift;
        int slot = -1;
#pragma unroll
        for (int t = 0; t < kMaxPages; ++t)
            if (slot < 0 && pg[t] >= 0 && pg[t] == page) slot = t;
        col_st[e] = slot >= 0 ? ~(slot * kPage + (c & (kPage - 1))) : c;
    }
}

int max_pages_for(int dtype) {
    // two CTAs per SM share about 228 KB of shared memory
    const int per_cta = 112 * 1024;
    return std::min(kMaxPages, per_cta / (kPage * (dtype == GBSP_F64 ? 8 : 4)));
}

}  // namespace

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_sell_stage_bytes(gbsp_handle h, int32_t pages_per_group, int64_t *col_bytes,
                                             int64_t *pages_bytes, int64_t *ws_bytes) {
    if (!h || !col_bytes || !pages_bytes || !ws_bytes) return arg_error("gbsp_sell_stage_bytes: NULL argument");
    if (h->kind != KIND_JDS || h->format != GBSP_SELL) return arg_error("gbsp_sell_stage_bytes: needs a SELL handle");
    if (pages_per_group < 1 || pages_per_group > max_pages_for(h->dtype))
        return arg_error("gbsp_sell_stage_bytes: pages_per_group out of range");
    const int64_t ngroups = ceil_div(h->n_blocks, kGroupBlocks);
    *col_bytes = 4 * h->nnz;
    *pages_bytes = 4 * ngroups * pages_per_group;
    *ws_bytes = ((4 * h->nnz + 255) & ~int64_t(255)) + sort_keys_ws_bytes(h->nnz) + 256;
    return GBSP_OK;
}

extern "C" gbsp_status gbsp_sell_stage(gbsp_handle h, int32_t pages_per_group, int32_t min_refs,
                                       int32_t *d_col_staged, int32_t *d_pages, void *d_ws, int64_t ws_bytes,
                                       void *stream) {
    if (!h) return arg_error("gbsp_sell_stage: NULL handle");
    if (h->kind != KIND_JDS || h->format != GBSP_SELL) return arg_error("gbsp_sell_stage: needs a SELL handle");
    if (pages_per_group == 0) {  // remove the staging
        h->stage_col = nullptr;
        h->stage_pages = nullptr;
        h->stage_pages_per_group = 0;
        return GBSP_OK;
    }
    int64_t cb = 0, pb = 0, wb = 0;
    gbsp_status st = gbsp_sell_stage_bytes(h, pages_per_group, &cb, &pb, &wb);
    if (st != GBSP_OK) return st;
    if (min_refs < 1) return arg_error("gbsp_sell_stage: min_refs must be >= 1");
    if ((cb > 0 && !d_col_staged) || !d_pages || !d_ws || ws_bytes < wb)
        return arg_error("gbsp_sell_stage: NULL or undersized buffer");
    const int64_t nb = h->n_blocks, nnz = h->nnz, ngroups = ceil_div(nb, kGroupBlocks);
    const int pbits = bits_of((uint64_t)std::max<int64_t>(h->n_cols - 1, 0) >> kPageShift);
    const int gbits = bits_of((uint64_t)std::max<int64_t>(ngroups - 1, 0));
    if (pbits + gbits > 32) {
        set_error("gbsp_sell_stage: the (group, page) key exceeds 32 bits");
        return GBSP_ERR_UNSUPPORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *keys = static_cast<uint32_t *>(d_ws);
    char *sort_ws = static_cast<char *>(d_ws) + ((4 * nnz + 255) & ~int64_t(255));
    if (nb > 0 && nnz > 0) {
        const unsigned gw = (unsigned)ceil_div(nb * 32, 256);
        stage_keys_kernel<<<gw, 256, 0, s>>>(nb, h->blk_ptr, h->col, pbits, keys);
        GBSP_LAUNCH_CHECK("stage_keys_kernel");
        uint32_t *ks = nullptr;
        st = sort_keys(keys, nnz, std::max(pbits + gbits, 1), sort_ws, s, &ks);
        if (st != GBSP_OK) return st;
        stage_select_kernel<<<(unsigned)ceil_div(ngroups, 128), 128, 0, s>>>(ngroups, ks, nnz, pbits,
                                                                             pages_per_group, min_refs, d_pages);
        GBSP_LAUNCH_CHECK("stage_select_kernel");
        stage_encode_kernel<<<gw, 256, 0, s>>>(nb, h->blk_ptr, h->col, d_pages, pages_per_group, d_col_staged);
        GBSP_LAUNCH_CHECK("stage_encode_kernel");
    } else if (ngroups > 0) {
        GBSP_CUDA(cudaMemsetAsync(d_pages, 0xff, 4 * ngroups * pages_per_group, s));
    }
    GBSP_CUDA(cudaStreamSynchronize(s));
    h->stage_col = d_col_staged;
    h->stage_pages = d_pages;
    h->stage_pages_per_group = pages_per_group;
    return GBSP_OK;
}
