// Format conversion on the device: CRS -> JDS family (Sect. 2 JDS
// construction), RBJDS / SOJDS re-layout, and the transposed CRS structure.
//
// Everything is deterministic: the row sort and the transpose use a stable
// LSD radix sort whose per-tile ranks come from warp match/ballot
// operations in a fixed (round, warp, lane) order; integer atomics only
// count.  So every output array is a bit-exact function of the input.
#include <algorithm>
#include <vector>

#include "accum.cuh"
#include "internal.cuh"

namespace gbsp {

// ----------------------------------------------------------------- scan --
// Exclusive prefix sum of int32 (totals < 2^31): tiles of 2048 items.

constexpr int kScanThreads = 512;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_sums,
                                                        int32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += t;
        }
        if (lane < nw) warp_sums[lane] = s;  // inclusive warp totals
        if (lane == nw - 1) *total = s;
    }
    __syncthreads();
    const int32_t before = wid > 0 ? warp_sums[wid - 1] : 0;
    const int32_t res = before + incl - v;
    __syncthreads();
    return res;
}

__global__ void scan_tile_sums(const int32_t *__restrict__ in, int64_t n, int32_t *sums) {
    __shared__ int32_t ws[32];
    __shared__ int32_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int32_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanPer; ++u)
        if (base + u < n) s += in[base + u];
    block_exclusive_scan(s, ws, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single CTA: exclusive scan of the tile sums in place
__global__ void scan_sums_kernel(int32_t *sums, int64_t n) {
    __shared__ int32_t ws[32];
    __shared__ int32_t tot;
    int32_t carry = 0;
    for (int64_t c = 0; c < n; c += blockDim.x) {
        const int64_t i = c + threadIdx.x;
        const int32_t v = i < n ? sums[i] : 0;
        const int32_t ex = block_exclusive_scan(v, ws, &tot);
        if (i < n) sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

__global__ void scan_apply(const int32_t *in, int64_t n, const int32_t *__restrict__ sums,
                           int32_t *out, int32_t *total_out) {
    __shared__ int32_t ws[32];
    __shared__ int32_t tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int32_t v[kScanPer];
    int32_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        v[u] = base + u < n ? in[base + u] : 0;
        s += v[u];
    }
    int32_t run = sums[blockIdx.x] + block_exclusive_scan(s, ws, &tot);
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        if (base + u < n) out[base + u] = run;
        run += v[u];
    }
    if (total_out && base < n && base + kScanPer >= n) *total_out = run;
}

int64_t scan_ws_bytes(int64_t n) { return (ceil_div(std::max<int64_t>(n, 1), kScanTile) + 1) * 4; }

// out[0..n) = exclusive scan of in[0..n); out[n] = total if total_out given
// (total_out may point at out + n).  in and out may alias.
gbsp_status scan_exclusive(const int32_t *in, int64_t n, int32_t *out, int32_t *total_out,
                                  int32_t *ws, cudaStream_t s) {
    if (n == 0) {
        if (total_out) GBSP_CUDA(cudaMemsetAsync(total_out, 0, 4, s));
        return GBSP_OK;
    }
    const int64_t tiles = ceil_div(n, kScanTile);
    scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, ws);
    scan_sums_kernel<<<1, 1024, 0, s>>>(ws, tiles);
    scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, ws, out, total_out);
    GBSP_LAUNCH_CHECK("scan");
    return GBSP_OK;
}

// ----------------------------------------------------------- radix sort --
// Stable LSD radix sort of (uint32 key, int32 value) pairs, 8 bits a pass.

constexpr int kSortThreads = 256;
constexpr int kSortPer = 8;
constexpr int kSortTile = kSortThreads * kSortPer;
constexpr int kRadix = 256;

__global__ void radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                  int64_t n_tiles, int32_t *hist) {
    __shared__ int32_t cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int u = 0; u < kSortPer; ++u) {
        const int64_t i = base + u * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter with stable ranks.  Items of a tile are visited as round u, warp w,
// lane l (item base + u*256 + w*32 + l), which is their index order, so a
// running per-digit count across (round, warp) gives each item the number of
// equal digits before it in the tile.
__global__ void radix_scatter_kernel(const uint32_t *__restrict__ keys_in,
                                     const int32_t *__restrict__ vals_in, int64_t n, int shift,
                                     int64_t n_tiles, const int32_t *__restrict__ offsets,
                                     uint32_t *__restrict__ keys_out,
                                     int32_t *__restrict__ vals_out) {
    __shared__ int32_t run[kRadix];
    __shared__ int32_t warp_cnt[kSortThreads / 32][kRadix];
    __shared__ int32_t tile_off[kRadix];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    tile_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int u = 0; u < kSortPer; ++u) {
        for (int w = 0; w < kSortThreads / 32; ++w) warp_cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + u * kSortThreads + threadIdx.x;
        const bool ok = i < n;
        const uint32_t key = ok ? keys_in[i] : 0u;
        const int32_t val = ok ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
        const int dig = ok ? (int)((key >> shift) & (kRadix - 1)) : kRadix;  // kRadix: no item
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & lt_mask);
        if (ok && rank == 0) warp_cnt[wid][dig] = __popc(peers);
        __syncthreads();
        {
            // thread d turns warp counts of digit d into running offsets
            const int d = threadIdx.x;
            int32_t r = run[d];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const int32_t c = warp_cnt[w][d];
                warp_cnt[w][d] = r;
                r += c;
            }
            run[d] = r;
        }
        __syncthreads();
        if (ok) {
            const int64_t dst = (int64_t)tile_off[dig] + warp_cnt[wid][dig] + rank;
            keys_out[dst] = key;
            vals_out[dst] = val;
        }
        __syncthreads();
    }
}

struct SortWs {
    uint32_t *keys_b;
    int32_t *vals_a, *vals_b;
    int32_t *hist;
    int32_t *scan_ws;
};

static int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

static int64_t sort_ws_bytes(int64_t n) {
    const int64_t tiles = ceil_div(std::max<int64_t>(n, 1), kSortTile);
    return align256(4 * n) * 3 + align256(4 * kRadix * tiles) + align256(scan_ws_bytes(kRadix * tiles));
}

static SortWs carve_sort_ws(char *&p, int64_t n) {
    const int64_t tiles = ceil_div(std::max<int64_t>(n, 1), kSortTile);
    SortWs w;
    w.keys_b = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * n);
    w.vals_a = reinterpret_cast<int32_t *>(p);
    p += align256(4 * n);
    w.vals_b = reinterpret_cast<int32_t *>(p);
    p += align256(4 * n);
    w.hist = reinterpret_cast<int32_t *>(p);
    p += align256(4 * kRadix * tiles);
    w.scan_ws = reinterpret_cast<int32_t *>(p);
    p += align256(scan_ws_bytes(kRadix * tiles));
    return w;
}

// Sorts keys[0..n) (bits significant bits) carrying values vals0[0..n)
// (the original index when vals0 is NULL; vals0 is only read, and must not
// be one of the workspace's value buffers).
// Result: *keys_out / *vals_out point at the buffer holding the sorted pairs.
static gbsp_status radix_sort_pairs(uint32_t *keys, const int32_t *vals0, int64_t n, int bits, SortWs &w,
                                    cudaStream_t s, uint32_t **keys_out, int32_t **vals_out) {
    const int64_t tiles = ceil_div(std::max<int64_t>(n, 1), kSortTile);
    uint32_t *ka = keys, *kb = w.keys_b;
    const int32_t *va = vals0;
    int32_t *vb = w.vals_a;
    int32_t *vspare = w.vals_b;
    bool va_in_ws = false;
    if (bits <= 0) bits = 1;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(ka, n, shift, tiles, w.hist);
        gbsp_status st = scan_exclusive(w.hist, kRadix * tiles, w.hist, nullptr, w.scan_ws, s);
        if (st != GBSP_OK) return st;
        radix_scatter_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(ka, va, n, shift, tiles,
                                                                      w.hist, kb, vb);
        GBSP_LAUNCH_CHECK("radix_scatter_kernel");
        std::swap(ka, kb);
        // values: the buffer just written becomes the input; the next output
        // is the workspace buffer not being read
        int32_t *written = vb;
        vb = va_in_ws ? const_cast<int32_t *>(va) : vspare;
        va = written;
        va_in_ws = true;
    }
    *keys_out = ka;
    *vals_out = const_cast<int32_t *>(va);
    return GBSP_OK;
}

static gbsp_status radix_sort_index(uint32_t *keys, int64_t n, int bits, SortWs &w,
                                    cudaStream_t s, uint32_t **keys_out, int32_t **vals_out) {
    return radix_sort_pairs(keys, nullptr, n, bits, w, s, keys_out, vals_out);
}

// Sort of bare keys (the values, the original positions, are not needed):
// workspace of sort_keys_ws_bytes(n); *sorted points into keys or the
// workspace.  `keys` is overwritten.
int64_t sort_keys_ws_bytes(int64_t n) { return sort_ws_bytes(n); }

gbsp_status sort_keys(uint32_t *keys, int64_t n, int bits, void *ws, cudaStream_t s, uint32_t **sorted) {
    char *p = static_cast<char *>(ws);
    SortWs w = carve_sort_ws(p, n);
    int32_t *vs = nullptr;
    return radix_sort_index(keys, n, bits, w, s, sorted, &vs);
}

// ------------------------------------------------------------ JDS build --

__global__ void row_len_kernel(int64_t n, const int32_t *__restrict__ row_ptr, int32_t *len,
                               int32_t *max_len) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t l = 0;
    if (i < n) {
        l = row_ptr[i + 1] - row_ptr[i];
        if (len) len[i] = l;
    }
    // warp max then one atomic per warp (integer: order-independent)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, off));
    if ((threadIdx.x & 31) == 0 && l > 0) atomicMax(max_len, l);
}

__global__ void len_key_kernel(int64_t n, const int32_t *__restrict__ len, int32_t max_len,
                               uint32_t *keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = (uint32_t)(max_len - len[i]);  // ascending key = decreasing length
}

__global__ void inverse_perm_kernel(int64_t n, const int32_t *__restrict__ perm, int32_t *iperm) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) iperm[perm[r]] = (int32_t)r;
}

// diagLen(d) = #{rows with length > d}.  With rows sorted by decreasing
// length, sorted row r is the last one present in diagonals
// len_sorted[r+1] .. len_sorted[r]-1, so it writes diagLen = r + 1 there.
__global__ void diag_len_kernel(int64_t n, int64_t n_diag, const int32_t *__restrict__ perm,
                                const int32_t *__restrict__ len, int32_t *diag_len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t lr = (int32_t)min((int64_t)len[perm[r]], n_diag);
    const int32_t ln = r + 1 < n ? len[perm[r + 1]] : 0;
    for (int32_t d = ln; d < lr; ++d) diag_len[d] = (int32_t)(r + 1);
}

// val_jds[jd_ptr[d] + r] = val[row_ptr[perm[r]] + d], col likewise
// (renumbered by iperm under the symmetric permutation).
template <typename T>
__global__ void jds_scatter_kernel(int64_t n, const int32_t *__restrict__ perm,
                                   const int32_t *__restrict__ iperm,
                                   const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, const T *__restrict__ val,
                                   const int32_t *__restrict__ jd_ptr, int64_t n_diag,
                                   int symmetric, int32_t *col_out, T *val_out, int32_t *vmap) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int32_t src = row_ptr[perm[r]];
    // rows longer than the planned N_j (matrix changed after the plan) are cut
    const int32_t len = (int32_t)min((int64_t)(row_ptr[perm[r] + 1] - src), n_diag);
    for (int32_t d = 0; d < len; ++d) {
        const int64_t dst = (int64_t)jd_ptr[d] + r;
        const int32_t c = col[src + d];
        col_out[dst] = symmetric ? iperm[c] : c;
        val_out[dst] = val[src + d];
        if (vmap) vmap[dst] = src + d;
    }
}

// blk_ptr[k] = #entries in rows before the block = sum_d min(diagLen(d), b0).
__global__ void blk_ptr_kernel(int64_t n_rows, int64_t n_diag, int64_t block, int64_t n_blocks,
                               const int32_t *__restrict__ jd_ptr, int32_t *blk_ptr) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n_blocks) return;
    const int64_t b0 = std::min<int64_t>(k * block, n_rows);
    int64_t s = 0;
    for (int64_t d = 0; d < n_diag; ++d) {
        const int64_t dl = jd_ptr[d + 1] - jd_ptr[d];
        if (dl <= 0) break;
        s += dl < b0 ? dl : b0;
    }
    blk_ptr[k] = (int32_t)s;
}

// RBJDS re-layout: entry (d, r) of block k goes to
// blk_ptr[k] + sum_{d'<d}(min(diagLen(d'), b1) - b0) + (r - b0).
template <typename T>
__global__ void rbjds_scatter_kernel(int64_t n_rows, int64_t n_diag, int64_t block,
                                     const int32_t *__restrict__ jd_ptr,
                                     const int32_t *__restrict__ blk_ptr,
                                     const int32_t *__restrict__ col_in,
                                     const T *__restrict__ val_in, const int32_t *__restrict__ map_in,
                                     int32_t *col_out, T *val_out, int32_t *map_out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const int64_t k = r / block, b0 = k * block, b1 = std::min<int64_t>(b0 + block, n_rows);
    int64_t off = blk_ptr[k];
    for (int64_t d = 0; d < n_diag; ++d) {
        const int64_t dl = jd_ptr[d + 1] - jd_ptr[d];
        if (dl <= r) break;
        const int64_t src = (int64_t)jd_ptr[d] + r;
        col_out[off + (r - b0)] = col_in[src];
        val_out[off + (r - b0)] = val_in[src];
        if (map_out) map_out[off + (r - b0)] = map_in[src];
        off += (dl < b1 ? dl : b1) - b0;
    }
}

// SOJDS: one warp per block walks its rows in order.  Row b0 keeps its
// order; for a later row, slot d takes the unplaced entry whose column is
// nearest to prev[d] + 1 (prev[d] = column placed in slot d of the row
// above), ties to the smaller column, then to the earlier slot.  The warp
// searches the row's entries in parallel and reduces (distance, column,
// slot) lexicographically.  Dynamic shared memory: per warp, n_slots x
// (prev col, cur col, cur val, used flag).
template <typename T>
__global__ void sojds_kernel(int64_t n_rows, int64_t n_diag, int64_t block, int64_t n_blocks,
                             const int32_t *__restrict__ jd_ptr,
                             const int32_t *__restrict__ blk_ptr,
                             const int32_t *__restrict__ col_in, const T *__restrict__ val_in,
                             const int32_t *__restrict__ map_in, int32_t *col_out, T *val_out,
                             int32_t *map_out, int32_t max_slots) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // regions, each nw * max_slots long: [values][prev cols][cur cols][used]
    const size_t per = (size_t)max_slots, all = (size_t)nw * per;
    T *cur_val = reinterpret_cast<T *>(smem) + (size_t)wid * per;
    int32_t *ints = reinterpret_cast<int32_t *>(smem + all * sizeof(T));
    int32_t *prev = ints + (size_t)wid * per;
    int32_t *cur_col = ints + all + (size_t)wid * per;
    unsigned char *used = reinterpret_cast<unsigned char *>(ints + 2 * all) + (size_t)wid * per;
    for (int64_t k = (int64_t)blockIdx.x * nw + wid; k < n_blocks; k += (int64_t)gridDim.x * nw) {
        const int64_t b0 = k * block, b1 = std::min<int64_t>(b0 + block, n_rows);
        const int64_t base = blk_ptr[k];
        for (int64_t r = b0; r < b1; ++r) {
            // row length and the block-local slot offsets walk together
            int64_t off = 0;
            int32_t len = 0;
            for (int64_t d = 0; d < n_diag; ++d) {
                const int64_t dl = jd_ptr[d + 1] - jd_ptr[d];
                if (dl <= r) break;
                ++len;
            }
            for (int32_t d = lane; d < len; d += 32) {
                cur_col[d] = col_in[jd_ptr[d] + r];
                cur_val[d] = val_in[jd_ptr[d] + r];
                used[d] = 0;
            }
            __syncwarp();
            off = 0;
            for (int32_t d = 0; d < len; ++d) {
                const int64_t dl = jd_ptr[d + 1] - jd_ptr[d];
                int32_t pick = d;
                if (r != b0) {
                    const int64_t target = (int64_t)prev[d] + 1;
                    int64_t bd = INT64_MAX;
                    int32_t bc = 0, be = INT32_MAX;
                    for (int32_t e = lane; e < len; e += 32) {
                        if (used[e]) continue;
                        const int64_t dist = llabs((int64_t)cur_col[e] - target);
                        if (dist < bd || (dist == bd && cur_col[e] < bc)) {
                            bd = dist;
                            bc = cur_col[e];
                            be = e;
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const int64_t od = __shfl_xor_sync(0xffffffffu, bd, o);
                        const int32_t oc = __shfl_xor_sync(0xffffffffu, bc, o);
                        const int32_t oe = __shfl_xor_sync(0xffffffffu, be, o);
                        if (od < bd || (od == bd && (oc < bc || (oc == bc && oe < be)))) {
                            bd = od;
                            bc = oc;
                            be = oe;
                        }
                    }
                    pick = be;
                }
                const int64_t dst = base + off + (r - b0);
                if (lane == 0) {
                    used[pick] = 1;
                    col_out[dst] = cur_col[pick];
                    val_out[dst] = cur_val[pick];
                    // the picked entry sat in slot `pick` of this row in the input
                    if (map_out) map_out[dst] = map_in[jd_ptr[pick] + r];
                }
                __syncwarp();
                if (lane == 0) prev[d] = cur_col[pick];
                __syncwarp();
                off += (dl < b1 ? dl : b1) - b0;
            }
        }
    }
}

// --------------------------------------------------------------- SELL ----
// Sort key: window index in the high bits, (max_len - len) in the low bits,
// so a stable ascending sort groups rows by window and, inside a window,
// orders them by decreasing length with ties in row order.
__global__ void sell_key_kernel(int64_t n, const int32_t *__restrict__ len, int32_t max_len,
                                int64_t window, int lbits, uint32_t *keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = ((uint32_t)(i / window) << lbits) | (uint32_t)(max_len - len[i]);
}

// Second key of the two-stage SELL sort: the window of the row now at r.
__global__ void window_key_kernel(int64_t n, const int32_t *__restrict__ rows, int64_t window,
                                  uint32_t *keys) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) keys[r] = (uint32_t)(rows[r] / window);
}

__global__ void sell_rlen_kernel(int64_t n, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ len, int32_t *rlen) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) rlen[r] = len[perm[r]];
}

// entries per block of 32 permuted rows (one warp per block)
__global__ void sell_block_nnz_kernel(int64_t n, int64_t nb, const int32_t *__restrict__ rlen,
                                      int32_t *blk_nnz) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t l = r < n ? rlen[r] : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && (r >> 5) < nb) blk_nnz[r >> 5] = l;
}

// Thread per permuted row, warps aligned to 32-row blocks: slot d of the
// block holds the rows with length > d, which are the block's first rows
// (sorted), so the position of row r's slot d is
// blk_ptr[b] + (entries of slots < d in the block) + (r mod 32).
template <typename T>
__global__ void sell_scatter_kernel(int64_t n, const int32_t *__restrict__ perm,
                                    const int32_t *__restrict__ iperm, const int32_t *__restrict__ rlen,
                                    const int32_t *__restrict__ blk_ptr,
                                    const int32_t *__restrict__ row_ptr,
                                    const int32_t *__restrict__ col, const T *__restrict__ val,
                                    int symmetric, int32_t *col_out, T *val_out, int32_t *vmap) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int32_t len = r < n ? rlen[r] : 0;
    const int64_t src = r < n ? (int64_t)row_ptr[perm[r]] : 0;
    int64_t off = (r >> 5) <= (n - 1) / 32 ? blk_ptr[r >> 5] : 0;
    for (int32_t d = 0;; ++d) {
        const unsigned mask = __ballot_sync(0xffffffffu, len > d);
        if (!mask) break;
        if (len > d) {
            const int64_t dst = off + lane;
            const int32_t c = col[src + d];
            col_out[dst] = symmetric ? iperm[c] : c;
            val_out[dst] = val[src + d];
            if (vmap) vmap[dst] = (int32_t)(src + d);
        }
        off += __popc(mask);
    }
}

// -------------------------------------------------------- paired SELL ----
// Thread per sorted position: rank q of a window of m rows is the first row
// of lane q when q < ceil(m/2), else the second row of lane m-1-q; lane
// (window w0, lane) lives in block w0/64 + lane/32 at position lane % 32.
__global__ void psell_pair_kernel(int64_t n, int64_t window, const int32_t *__restrict__ sorted,
                                  int32_t *perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t w0 = i / window * window, m = min(window, n - w0), q = i - w0;
    const int64_t lanes = (m + 1) / 2;
    const bool first = q < lanes;
    const int64_t lane = first ? q : m - 1 - q;
    const int64_t g = w0 / 64 + lane / 32, p = lane % 32;
    const int64_t R = min((int64_t)64, n - 64 * g), L = (R + 1) / 2;
    perm[first ? 64 * g + p : 64 * g + L + p] = sorted[i];
}

// Lane p of block g: its rows and their lengths (0 for a missing row).
struct PsellLane {
    int64_t ra, rb;
    int32_t la, lb;
    bool lane_ok, has_b;
};

__device__ __forceinline__ PsellLane psell_lane(int64_t n, int64_t g, int p, const int32_t *__restrict__ rlen) {
    PsellLane o;
    const int64_t R = min((int64_t)64, n - 64 * g), L = (R + 1) / 2;
    o.lane_ok = p < L;
    o.has_b = o.lane_ok && L + p < R;
    o.ra = 64 * g + p;
    o.rb = 64 * g + L + p;
    o.la = o.lane_ok ? rlen[o.ra] : 0;
    o.lb = o.has_b ? rlen[o.rb] : 0;
    return o;
}

// entries per 64-row block (one warp per block)
__global__ void psell_block_nnz_kernel(int64_t n, int64_t nb, const int32_t *__restrict__ rlen,
                                       int32_t *blk_nnz) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nb) return;  // warp-uniform
    const PsellLane ln = psell_lane(n, g, threadIdx.x & 31, rlen);
    int32_t l = ln.la + ln.lb;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) blk_nnz[g] = l;
}

// One warp per block: slot t holds the lanes whose two rows have more than
// t entries, in lane order (position by ballot prefix); entry t of a lane is
// entry t of its first row, or entry t - la of its second.
template <typename T>
__global__ void psell_scatter_kernel(int64_t n, int64_t nb, const int32_t *__restrict__ perm,
                                     const int32_t *__restrict__ iperm, const int32_t *__restrict__ rlen,
                                     const int32_t *__restrict__ blk_ptr, const int32_t *__restrict__ row_ptr,
                                     const int32_t *__restrict__ col, const T *__restrict__ val, int symmetric,
                                     int32_t *col_out, T *val_out, int32_t *vmap) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nb) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const PsellLane ln = psell_lane(n, g, lane, rlen);
    const int32_t total = ln.la + ln.lb;
    const int32_t width = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)total);
    const int64_t src_a = ln.lane_ok ? (int64_t)row_ptr[perm[ln.ra]] : 0;
    const int64_t src_b = ln.has_b ? (int64_t)row_ptr[perm[ln.rb]] : 0;
    const unsigned lt = (1u << lane) - 1u;
    int64_t off = blk_ptr[g];
    for (int32_t t = 0; t < width; ++t) {
        const bool act = total > t;
        const unsigned mask = __ballot_sync(0xffffffffu, act);
        if (act) {
            const int64_t dst = off + __popc(mask & lt);
            const int64_t src = t < ln.la ? src_a + t : src_b + (t - ln.la);
            const int32_t c = col[src];
            col_out[dst] = symmetric ? iperm[c] : c;
            val_out[dst] = val[src];
            if (vmap) vmap[dst] = (int32_t)src;
        }
        off += __popc(mask);
    }
}

// ------------------------------------------------------------- host side --

static int bits_for(uint64_t maxv) {
    int b = 0;
    while (b < 32 && (maxv >> b) != 0) ++b;
    return b;
}

gbsp_status jds_plan_impl(const Mat &A, const gbsp_jds_opts &o, int32_t *d_scratch,
                          cudaStream_t s, gbsp_jds_sizes *out) {
    GBSP_CUDA(cudaMemsetAsync(d_scratch, 0, sizeof(int32_t), s));
    if (A.n_rows > 0)
        row_len_kernel<<<(unsigned)ceil_div(A.n_rows, 256), 256, 0, s>>>(A.n_rows, A.row_ptr,
                                                                        nullptr, d_scratch);
    GBSP_LAUNCH_CHECK("row_len_kernel");
    int32_t max_len = 0;
    GBSP_CUDA(cudaMemcpyAsync(&max_len, d_scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    const int64_t block = o.block > 0 ? o.block : 256;
    out->n_rows = A.n_rows;
    out->n_cols = A.n_cols;
    out->nnz = A.nnz;
    out->n_diag = max_len;
    const bool blocked = o.format == GBSP_RBJDS || o.format == GBSP_SOJDS;
    out->n_blocks = blocked ? ceil_div(A.n_rows, block) : 0;
    if (o.format == GBSP_SELL || o.format == GBSP_PSELL) {
        const int64_t window = o.window > 0 ? o.window : 1024;
        const int64_t rows_per_block = o.format == GBSP_PSELL ? 64 : 32;
        if (window % rows_per_block) {
            set_error("gbsp_jds_plan: the %s window must be a multiple of %d",
                      o.format == GBSP_PSELL ? "PSELL" : "SELL", (int)rows_per_block);
            return GBSP_ERR_ARG;
        }
        out->n_blocks = ceil_div(A.n_rows, rows_per_block);
        out->workspace_bytes = align256(4 * A.n_rows) * 2 + sort_ws_bytes(A.n_rows) +
                               align256(4 * (out->n_blocks + 1)) + align256(scan_ws_bytes(out->n_blocks + 1)) + 256;
        return GBSP_OK;
    }
    // workspace: lengths, keys, sort buffers, diagLen (+ RBJDS staging)
    int64_t ws = align256(4 * A.n_rows) + align256(4 * A.n_rows) + sort_ws_bytes(A.n_rows) +
                 align256(4 * (max_len + 1)) + align256(scan_ws_bytes(max_len + 1)) + 256;
    if (blocked) ws += 2 * align256(4 * A.nnz) + align256((A.dtype == GBSP_F64 ? 8 : 4) * A.nnz);
    out->workspace_bytes = ws;
    return GBSP_OK;
}

template <typename T>
static void launch_jds_scatter(const Mat &A, const int32_t *perm, const int32_t *iperm,
                               const int32_t *jd_ptr, int64_t n_diag, int symmetric,
                               int32_t *col_out, void *val_out, int32_t *vmap, cudaStream_t s) {
    jds_scatter_kernel<T><<<(unsigned)ceil_div(A.n_rows, 256), 256, 0, s>>>(
        A.n_rows, perm, iperm, A.row_ptr, A.col, static_cast<const T *>(A.val), jd_ptr, n_diag,
        symmetric, col_out, static_cast<T *>(val_out), vmap);
}

template <typename T>
static gbsp_status relayout_blocked(const Mat &J, int64_t block, int format, const int32_t *col_in,
                                    const void *val_in, const int32_t *map_in, int32_t *col_out,
                                    void *val_out, int32_t *map_out, cudaStream_t s) {
    const int64_t nb = ceil_div(J.n_rows, block);
    if (format == GBSP_RBJDS) {
        rbjds_scatter_kernel<T><<<(unsigned)ceil_div(J.n_rows, 256), 256, 0, s>>>(
            J.n_rows, J.n_diag, block, J.jd_ptr, J.blk_ptr, col_in, static_cast<const T *>(val_in), map_in,
            col_out, static_cast<T *>(val_out), map_out);
        GBSP_LAUNCH_CHECK("rbjds_scatter_kernel");
        return GBSP_OK;
    }
    // SOJDS: slots per row <= n_diag; shared memory per warp = n_diag * (T + 9)
    const int64_t slots = std::max<int64_t>(J.n_diag, 1);
    int warps = 4;
    size_t smem = 0;
    for (; warps >= 1; warps >>= 1) {
        smem = (size_t)warps * slots * (sizeof(T) + 4 + 4 + 1) + 64;
        if (smem <= 200 * 1024) break;
    }
    if (warps < 1) {
        set_error("SOJDS: rows longer than %lld entries are not supported", (long long)(200 * 1024 / (sizeof(T) + 9)));
        return GBSP_ERR_UNSUPPORTED;
    }
    GBSP_CUDA(cudaFuncSetAttribute(sojds_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, warps), (int64_t)num_sms() * 8));
    sojds_kernel<T><<<(unsigned)grid, warps * 32, smem, s>>>(J.n_rows, J.n_diag, block, nb, J.jd_ptr,
                                                             J.blk_ptr, col_in,
                                                             static_cast<const T *>(val_in), map_in,
                                                             col_out, static_cast<T *>(val_out), map_out,
                                                             (int32_t)slots);
    GBSP_LAUNCH_CHECK("sojds_kernel");
    return GBSP_OK;
}

static gbsp_status sell_build_impl(const Mat &A, const gbsp_jds_opts &o, const gbsp_jds_buffers &b,
                                   const gbsp_jds_sizes &sz, cudaStream_t s, Mat *J) {
    const int64_t n = A.n_rows;
    const int symmetric = o.perm_mode == GBSP_PERM_SYMMETRIC;
    const int64_t window = o.window > 0 ? o.window : 1024;
    const bool paired = o.format == GBSP_PSELL;
    const int64_t rows_per_block = paired ? 64 : 32;
    const int64_t nb = ceil_div(n, rows_per_block);
    if (window % rows_per_block) return arg_error("gbsp_jds_build: window is not a multiple of the block rows");
    if (sz.n_blocks != nb) return arg_error("gbsp_jds_build: sizes do not come from this plan");
    char *p = static_cast<char *>(b.workspace);
    int32_t *len = reinterpret_cast<int32_t *>(p);
    p += align256(4 * n);
    uint32_t *keys = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * n);
    SortWs sw = carve_sort_ws(p, n);
    int32_t *blk_nnz = reinterpret_cast<int32_t *>(p);
    p += align256(4 * (nb + 1));
    int32_t *scan_ws = reinterpret_cast<int32_t *>(p);
    p += align256(scan_ws_bytes(nb + 1));
    int32_t *max_len_d = reinterpret_cast<int32_t *>(p);
    GBSP_CUDA(cudaMemsetAsync(max_len_d, 0, 4, s));
    if (n > 0) {
        const unsigned gr = (unsigned)ceil_div(n, 256);
        row_len_kernel<<<gr, 256, 0, s>>>(n, A.row_ptr, len, max_len_d);
        const int lbits = bits_for((uint64_t)sz.n_diag);
        const int wbits = bits_for((uint64_t)(n - 1) / window);
        uint32_t *ks = nullptr;
        int32_t *vs = nullptr;
        gbsp_status st;
        if (lbits + wbits <= 32) {
            // one sort on (window, max_len - len)
            sell_key_kernel<<<gr, 256, 0, s>>>(n, len, (int32_t)sz.n_diag, window, lbits, keys);
            GBSP_LAUNCH_CHECK("sell keys");
            st = radix_sort_index(keys, n, lbits + wbits, sw, s, &ks, &vs);
        } else {
            // the pair does not fit 32 bits: stable sort by length, then a
            // stable sort of that order by window (least significant first)
            len_key_kernel<<<gr, 256, 0, s>>>(n, len, (int32_t)sz.n_diag, keys);
            GBSP_LAUNCH_CHECK("sell length keys");
            st = radix_sort_index(keys, n, lbits, sw, s, &ks, &vs);
            if (st != GBSP_OK) return st;
            GBSP_CUDA(cudaMemcpyAsync(b.perm, vs, 4 * n, cudaMemcpyDeviceToDevice, s));
            window_key_kernel<<<gr, 256, 0, s>>>(n, b.perm, window, keys);
            GBSP_LAUNCH_CHECK("sell window keys");
            st = radix_sort_pairs(keys, b.perm, n, wbits, sw, s, &ks, &vs);
        }
        if (st != GBSP_OK) return st;
        if (paired)
            psell_pair_kernel<<<gr, 256, 0, s>>>(n, window, vs, b.perm);
        else
            GBSP_CUDA(cudaMemcpyAsync(b.perm, vs, 4 * n, cudaMemcpyDeviceToDevice, s));
        inverse_perm_kernel<<<gr, 256, 0, s>>>(n, b.perm, b.iperm);
        sell_rlen_kernel<<<gr, 256, 0, s>>>(n, b.perm, len, b.rlen);
        if (paired)
            psell_block_nnz_kernel<<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(n, nb, b.rlen, blk_nnz);
        else
            sell_block_nnz_kernel<<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(n, nb, b.rlen, blk_nnz);
        GBSP_LAUNCH_CHECK("sell perm / lengths");
        st = scan_exclusive(blk_nnz, nb, b.blk_ptr, b.blk_ptr + nb, scan_ws, s);
        if (st != GBSP_OK) return st;
        if (paired && A.dtype == GBSP_F64)
            psell_scatter_kernel<double><<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(
                n, nb, b.perm, b.iperm, b.rlen, b.blk_ptr, A.row_ptr, A.col, static_cast<const double *>(A.val),
                symmetric, b.col, static_cast<double *>(b.val), b.vmap);
        else if (paired)
            psell_scatter_kernel<float><<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(
                n, nb, b.perm, b.iperm, b.rlen, b.blk_ptr, A.row_ptr, A.col, static_cast<const float *>(A.val),
                symmetric, b.col, static_cast<float *>(b.val), b.vmap);
        else if (A.dtype == GBSP_F64)
            sell_scatter_kernel<double><<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(
                n, b.perm, b.iperm, b.rlen, b.blk_ptr, A.row_ptr, A.col, static_cast<const double *>(A.val),
                symmetric, b.col, static_cast<double *>(b.val), b.vmap);
        else
            sell_scatter_kernel<float><<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(
                n, b.perm, b.iperm, b.rlen, b.blk_ptr, A.row_ptr, A.col, static_cast<const float *>(A.val),
                symmetric, b.col, static_cast<float *>(b.val), b.vmap);
        GBSP_LAUNCH_CHECK("sell_scatter_kernel");
    } else {
        GBSP_CUDA(cudaMemsetAsync(b.blk_ptr, 0, 4, s));
    }
    J->kind = KIND_JDS;
    J->n_rows = A.n_rows;
    J->n_cols = A.n_cols;
    J->nnz = A.nnz;
    J->dtype = A.dtype;
    J->device = A.device;
    J->col = b.col;
    J->val = b.val;
    J->format = paired ? GBSP_PSELL : GBSP_SELL;
    J->perm_mode = o.perm_mode;
    J->block = (int32_t)rows_per_block;
    J->built_block = (int32_t)rows_per_block;
    J->unroll = o.unroll > 0 ? o.unroll : 4;
    J->window = (int32_t)window;
    J->n_diag = sz.n_diag;
    J->n_blocks = nb;
    J->jd_ptr = nullptr;
    J->perm = b.perm;
    J->iperm = b.iperm;
    J->blk_ptr = b.blk_ptr;
    J->rlen = b.rlen;
    J->vmap = b.vmap;
    J->kopt = A.kopt;
    J->kopt.rows_per_warp = 1;
    GBSP_CUDA(cudaStreamSynchronize(s));
    return GBSP_OK;
}

gbsp_status jds_build_impl(const Mat &A, const gbsp_jds_opts &o, const gbsp_jds_buffers &b,
                           const gbsp_jds_sizes &sz, cudaStream_t s, Mat *J) {
    if (o.format == GBSP_SELL || o.format == GBSP_PSELL) return sell_build_impl(A, o, b, sz, s, J);
    const int64_t n = A.n_rows;
    const int symmetric = o.perm_mode == GBSP_PERM_SYMMETRIC;
    const bool blocked = o.format == GBSP_RBJDS || o.format == GBSP_SOJDS;
    const int64_t block = o.block > 0 ? o.block : 256;
    const size_t vsz = A.dtype == GBSP_F64 ? 8 : 4;
    char *p = static_cast<char *>(b.workspace);
    int32_t *len = reinterpret_cast<int32_t *>(p);
    p += align256(4 * n);
    uint32_t *keys = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * n);
    SortWs sw = carve_sort_ws(p, n);
    int32_t *diag_len = reinterpret_cast<int32_t *>(p);
    p += align256(4 * (sz.n_diag + 1));
    int32_t *scan_ws = reinterpret_cast<int32_t *>(p);
    p += align256(scan_ws_bytes(sz.n_diag + 1));
    int32_t *max_len_d = reinterpret_cast<int32_t *>(p);
    p += 256;
    int32_t *col_stage = nullptr, *map_stage = nullptr;
    void *val_stage = nullptr;
    if (blocked) {
        col_stage = reinterpret_cast<int32_t *>(p);
        p += align256(4 * A.nnz);
        val_stage = p;
        p += align256(vsz * A.nnz);
        map_stage = reinterpret_cast<int32_t *>(p);
        p += align256(4 * A.nnz);
    }

    const unsigned gr = (unsigned)ceil_div(std::max<int64_t>(n, 1), 256);
    GBSP_CUDA(cudaMemsetAsync(max_len_d, 0, 4, s));
    if (n > 0) {
        // (i) row lengths
        row_len_kernel<<<gr, 256, 0, s>>>(n, A.row_ptr, len, max_len_d);
        // (ii) stable sort by decreasing length
        len_key_kernel<<<gr, 256, 0, s>>>(n, len, (int32_t)sz.n_diag, keys);
        GBSP_LAUNCH_CHECK("row lengths");
        uint32_t *ks = nullptr;
        int32_t *vs = nullptr;
        gbsp_status st = radix_sort_index(keys, n, bits_for((uint64_t)sz.n_diag), sw, s, &ks, &vs);
        if (st != GBSP_OK) return st;
        GBSP_CUDA(cudaMemcpyAsync(b.perm, vs, 4 * n, cudaMemcpyDeviceToDevice, s));
        inverse_perm_kernel<<<gr, 256, 0, s>>>(n, b.perm, b.iperm);
        // (iii) jd_ptr from diagLen(d) = #{len > d}
        diag_len_kernel<<<gr, 256, 0, s>>>(n, sz.n_diag, b.perm, len, diag_len);
        GBSP_LAUNCH_CHECK("perm / diag_len");
    }
    {
        gbsp_status st = scan_exclusive(diag_len, sz.n_diag, b.jd_ptr, b.jd_ptr + sz.n_diag, scan_ws, s);
        if (st != GBSP_OK) return st;
    }
    // (iv), (v) shift left and scatter diagonal by diagonal
    int32_t *col_dst = blocked ? col_stage : b.col;
    void *val_dst = blocked ? val_stage : b.val;
    int32_t *map_dst = b.vmap ? (blocked ? map_stage : b.vmap) : nullptr;
    if (n > 0) {
        if (A.dtype == GBSP_F64)
            launch_jds_scatter<double>(A, b.perm, b.iperm, b.jd_ptr, sz.n_diag, symmetric, col_dst,
                                       val_dst, map_dst, s);
        else
            launch_jds_scatter<float>(A, b.perm, b.iperm, b.jd_ptr, sz.n_diag, symmetric, col_dst,
                                      val_dst, map_dst, s);
        GBSP_LAUNCH_CHECK("jds_scatter_kernel");
    }

    J->kind = KIND_JDS;
    J->n_rows = A.n_rows;
    J->n_cols = A.n_cols;
    J->nnz = A.nnz;
    J->dtype = A.dtype;
    J->device = A.device;
    J->col = b.col;
    J->val = b.val;
    J->format = o.format;
    J->perm_mode = o.perm_mode;
    J->block = (int32_t)block;
    J->built_block = blocked ? (int32_t)block : 0;
    J->unroll = o.unroll > 0 ? o.unroll : 4;
    J->n_diag = sz.n_diag;
    J->n_blocks = blocked ? ceil_div(n, block) : 0;
    J->jd_ptr = b.jd_ptr;
    J->perm = b.perm;
    J->iperm = b.iperm;
    J->blk_ptr = blocked ? b.blk_ptr : nullptr;
    J->vmap = b.vmap;
    J->kopt = A.kopt;
    J->kopt.rows_per_warp = 1;  // JDS walks: rows per thread

    if (blocked && n > 0) {
        blk_ptr_kernel<<<(unsigned)ceil_div(J->n_blocks + 1, 256), 256, 0, s>>>(
            n, J->n_diag, block, J->n_blocks, J->jd_ptr, b.blk_ptr);
        GBSP_LAUNCH_CHECK("blk_ptr_kernel");
        gbsp_status st = A.dtype == GBSP_F64
                             ? relayout_blocked<double>(*J, block, o.format, col_stage, val_stage,
                                                        map_dst, b.col, b.val, b.vmap, s)
                             : relayout_blocked<float>(*J, block, o.format, col_stage, val_stage,
                                                       map_dst, b.col, b.val, b.vmap, s);
        if (st != GBSP_OK) return st;
    } else if (blocked) {
        GBSP_CUDA(cudaMemsetAsync(b.blk_ptr, 0, 4, s));
    }
    // host copy of jd_ptr for per-diagonal launch planning
    J->h_jd_ptr.assign((size_t)sz.n_diag + 1, 0);
    GBSP_CUDA(cudaMemcpyAsync(J->h_jd_ptr.data(), b.jd_ptr, 4 * (sz.n_diag + 1),
                              cudaMemcpyDeviceToHost, s));
    GBSP_CUDA(cudaStreamSynchronize(s));
    return GBSP_OK;
}

// ------------------------------------------------------------ transpose --

__global__ void row_of_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr, int32_t *row_of) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) row_of[k] = (int32_t)r;
}

__global__ void col_count_kernel(int64_t nnz, const int32_t *__restrict__ col, int32_t *count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(count + col[k], 1);
}

__global__ void copy_keys_kernel(int64_t nnz, const int32_t *__restrict__ col, uint32_t *keys) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) keys[k] = (uint32_t)col[k];
}

__global__ void transpose_fill_kernel(int64_t nnz, const int32_t *__restrict__ sorted_idx,
                                      const int32_t *__restrict__ row_of, int32_t *tmap,
                                      int32_t *t_col) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int32_t k = sorted_idx[t];
    tmap[t] = k;
    t_col[t] = row_of[k];
}

template <typename T>
__global__ void gather_values_kernel(int64_t nnz, const int32_t *__restrict__ tmap,
                                     const T *__restrict__ val, T *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) out[t] = val[tmap[t]];
}

// Value re-gathers in row order.  A thread (or, for SELL, a lane) owns one
// stored row and walks its slots, so the source entries it reads, one CRS
// row, are read together and each source sector is fetched once; in entry
// order the lanes of a warp would take one 8-byte value from each of 32
// sectors and come back for the rest of those sectors much later.
template <typename T>
__global__ void csr_rows_gather_kernel(int64_t n_rows, const int32_t *__restrict__ row_ptr,
                                       const int32_t *__restrict__ map, const T *__restrict__ src,
                                       T *__restrict__ dst) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const int32_t e1 = __ldg(row_ptr + r + 1);
    for (int32_t e = __ldg(row_ptr + r); e < e1; ++e) dst[e] = src[__ldg(map + e)];
}

// JDS storage (JDS, NBJDS, NUJDS): thread r walks the diagonals of permuted row r.
template <typename T>
__global__ void jds_rows_gather_kernel(int64_t n, int64_t n_diag, const int32_t *__restrict__ jd_ptr,
                                       const int32_t *__restrict__ map, const T *__restrict__ src,
                                       T *__restrict__ dst) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    for (int64_t d = 0; d < n_diag; ++d) {
        const int32_t p0 = __ldg(jd_ptr + d), p1 = __ldg(jd_ptr + d + 1);
        if (p1 - p0 <= r) break;
        const int64_t pos = p0 + r;
        dst[pos] = src[__ldg(map + pos)];
    }
}

// SELL: one warp per 32-row block, lane = row, slots as in the SELL walk.
template <typename T>
__global__ void sell_rows_gather_kernel(int64_t n, int64_t nb, const int32_t *__restrict__ rlen,
                                        const int32_t *__restrict__ blk_ptr, const int32_t *__restrict__ map,
                                        const T *__restrict__ src, T *__restrict__ dst) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nb) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const int64_t r = b * 32 + lane;
    const int32_t len = r < n ? __ldg(rlen + r) : 0;
    int64_t off = __ldg(blk_ptr + b);
    for (int32_t d = 0;; ++d) {
        const unsigned mask = __ballot_sync(0xffffffffu, len > d);
        if (!mask) break;
        if (len > d) dst[off + lane] = src[__ldg(map + off + lane)];
        off += __popc(mask);
    }
}

gbsp_status jds_values_launch(const Mat &J, const void *src, cudaStream_t s) {
    if (J.nnz == 0) return GBSP_OK;
    const bool jds_storage = J.jd_ptr && (J.format == GBSP_JDS || J.format == GBSP_NBJDS ||
                                          J.format == GBSP_NUJDS || J.format == GBSP_JDS_LITERAL);
    const bool f64 = J.dtype == GBSP_F64;
    void *dst = const_cast<void *>(J.val);
    if (jds_storage) {
        const unsigned g = (unsigned)ceil_div(J.n_rows, 256);
        if (f64)
            jds_rows_gather_kernel<double><<<g, 256, 0, s>>>(J.n_rows, J.n_diag, J.jd_ptr, J.vmap,
                                                             static_cast<const double *>(src), static_cast<double *>(dst));
        else
            jds_rows_gather_kernel<float><<<g, 256, 0, s>>>(J.n_rows, J.n_diag, J.jd_ptr, J.vmap,
                                                            static_cast<const float *>(src), static_cast<float *>(dst));
        GBSP_LAUNCH_CHECK("jds_rows_gather_kernel");
        return GBSP_OK;
    }
    if (J.format == GBSP_SELL && J.rlen && J.blk_ptr) {
        const int64_t nb = ceil_div(J.n_rows, 32);
        const unsigned g = (unsigned)ceil_div(nb * 32, 256);
        if (f64)
            sell_rows_gather_kernel<double><<<g, 256, 0, s>>>(J.n_rows, nb, J.rlen, J.blk_ptr, J.vmap,
                                                              static_cast<const double *>(src), static_cast<double *>(dst));
        else
            sell_rows_gather_kernel<float><<<g, 256, 0, s>>>(J.n_rows, nb, J.rlen, J.blk_ptr, J.vmap,
                                                             static_cast<const float *>(src), static_cast<float *>(dst));
        GBSP_LAUNCH_CHECK("sell_rows_gather_kernel");
        return GBSP_OK;
    }
    return gather_values_launch(J.nnz, J.vmap, src, dst, J.dtype, s);
}

gbsp_status transpose_workspace_impl(const Mat &A, int64_t *bytes) {
    *bytes = align256(4 * A.nnz) * 2 + sort_ws_bytes(A.nnz) + align256(scan_ws_bytes(A.n_cols + 1)) + 256;
    return GBSP_OK;
}

gbsp_status transpose_build_impl(const Mat &A, const gbsp_transpose_buffers &b, int64_t ws_bytes,
                                 cudaStream_t s, Mat *T) {
    int64_t need = 0;
    transpose_workspace_impl(A, &need);
    if (ws_bytes < need) {
        set_error("transpose workspace too small: %lld < %lld", (long long)ws_bytes, (long long)need);
        return GBSP_ERR_NOMEM;
    }
    char *p = static_cast<char *>(b.workspace);
    int32_t *row_of = reinterpret_cast<int32_t *>(p);
    p += align256(4 * A.nnz);
    uint32_t *keys = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * A.nnz);
    SortWs sw = carve_sort_ws(p, A.nnz);
    int32_t *scan_ws = reinterpret_cast<int32_t *>(p);

    GBSP_CUDA(cudaMemsetAsync(b.t_row_ptr, 0, 4 * (A.n_cols + 1), s));
    if (A.nnz > 0) {
        const unsigned gk = (unsigned)ceil_div(A.nnz, 256);
        row_of_kernel<<<(unsigned)ceil_div(A.n_rows, 256), 256, 0, s>>>(A.n_rows, A.row_ptr, row_of);
        col_count_kernel<<<gk, 256, 0, s>>>(A.nnz, A.col, b.t_row_ptr);
        copy_keys_kernel<<<gk, 256, 0, s>>>(A.nnz, A.col, keys);
        GBSP_LAUNCH_CHECK("transpose counts");
        uint32_t *ks = nullptr;
        int32_t *vs = nullptr;
        gbsp_status st = radix_sort_index(keys, A.nnz, bits_for((uint64_t)std::max<int64_t>(A.n_cols - 1, 0)),
                                          sw, s, &ks, &vs);
        if (st != GBSP_OK) return st;
        transpose_fill_kernel<<<gk, 256, 0, s>>>(A.nnz, vs, row_of, b.tmap, b.t_col);
        GBSP_LAUNCH_CHECK("transpose_fill_kernel");
    }
    gbsp_status st = scan_exclusive(b.t_row_ptr, A.n_cols, b.t_row_ptr, b.t_row_ptr + A.n_cols, scan_ws, s);
    if (st != GBSP_OK) return st;

    T->kind = KIND_CRS;
    T->n_rows = A.n_cols;
    T->n_cols = A.n_rows;
    T->nnz = A.nnz;
    T->dtype = A.dtype;
    T->device = A.device;
    T->row_ptr = b.t_row_ptr;
    T->col = b.t_col;
    T->val = b.t_val;
    T->tmap = b.tmap;
    T->transpose_src = &A;
    crs_default_opts(*T);
    T->kopt.accum = A.kopt.accum;
    return transpose_values_impl(*T, s);
}

gbsp_status gather_values_launch(int64_t n, const int32_t *map, const void *src, void *dst, int dtype,
                                 cudaStream_t s) {
    if (n == 0) return GBSP_OK;
    const unsigned g = (unsigned)ceil_div(n, 256);
    if (dtype == GBSP_F64)
        gather_values_kernel<double><<<g, 256, 0, s>>>(n, map, static_cast<const double *>(src),
                                                       static_cast<double *>(dst));
    else
        gather_values_kernel<float><<<g, 256, 0, s>>>(n, map, static_cast<const float *>(src),
                                                      static_cast<float *>(dst));
    GBSP_LAUNCH_CHECK("gather_values_kernel");
    return GBSP_OK;
}

gbsp_status transpose_values_impl(const Mat &T, cudaStream_t s) {
    if (T.nnz == 0) return GBSP_OK;
    const unsigned g = (unsigned)ceil_div(T.n_rows, 256);
    if (T.dtype == GBSP_F64)
        csr_rows_gather_kernel<double><<<g, 256, 0, s>>>(T.n_rows, T.row_ptr, T.tmap,
                                                         static_cast<const double *>(T.transpose_src->val),
                                                         static_cast<double *>(const_cast<void *>(T.val)));
    else
        csr_rows_gather_kernel<float><<<g, 256, 0, s>>>(T.n_rows, T.row_ptr, T.tmap,
                                                        static_cast<const float *>(T.transpose_src->val),
                                                        static_cast<float *>(const_cast<void *>(T.val)));
    GBSP_LAUNCH_CHECK("csr_rows_gather_kernel");
    return GBSP_OK;
}

}  // namespace gbsp
