// Autotuner: times the candidate kernels of one handle on the device and
// keeps the fastest.  The analogue of the paper's block-size and schedule
// sweeps (Sect. 4.2 and 4): on GB300 the knobs are lanes per row, rows in
// flight per lane group, the tile of the TILED kernel, the right-hand-side
// tile, and for the JDS family the walk (JDS / NUJDS unroll / NBJDS block).
// Results are cached per matrix signature so that a batch of similar
// matrices is tuned once.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace gbsp {

struct Cand {
    gbsp_kernel_opts k;
    int format, block, unroll;
};

typedef std::tuple<int, int, int64_t, int64_t, int64_t, int, int, int, int, int> TuneKey;

static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<Cand, float>> g_tune_cache;

static TuneKey key_of(const Mat &A, int k) {
    return TuneKey(A.kind, A.kind == KIND_JDS ? (A.built_block > 0 ? A.format : -1) : -1, A.n_rows, A.n_cols,
                   A.nnz, k, A.dtype, A.kopt.accum, A.tile_rows != nullptr ? A.tile : 0, A.device);
}

static void apply(Mat &A, const Cand &c) {
    const int accum = A.kopt.accum;
    A.kopt = c.k;
    A.kopt.accum = accum;
    if (A.kind == KIND_JDS) {
        A.format = c.format;
        if (c.block > 0) A.block = c.block;
        if (c.unroll > 0) A.unroll = c.unroll;
    }
}

static gbsp_status time_one(Mat &A, const VecArgs &v, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                            float *ms) {
    auto launch = [&]() { return A.kind == KIND_CRS ? crs_launch(A, v, s) : jds_launch(A, v, s); };
    gbsp_status st = launch();  // warm-up
    if (st != GBSP_OK) return st;
    std::vector<float> t;
    for (int rep = 0; rep < 3; ++rep) {
        GBSP_CUDA(cudaEventRecord(e0, s));
        st = launch();
        if (st != GBSP_OK) return st;
        GBSP_CUDA(cudaEventRecord(e1, s));
        GBSP_CUDA(cudaEventSynchronize(e1));
        float x = 0;
        GBSP_CUDA(cudaEventElapsedTime(&x, e0, e1));
        t.push_back(x);
    }
    std::sort(t.begin(), t.end());
    *ms = t[1];
    return GBSP_OK;
}

static std::vector<Cand> candidates(const Mat &A, int k) {
    std::vector<Cand> out;
    Cand base{};
    base.k = A.kopt;
    base.format = A.format;
    base.block = A.block;
    base.unroll = A.unroll;
    if (A.kind == KIND_CRS) {
        if (k == 1) {
            for (int l : {2, 4, 8, 16, 32})
                for (int r : {1, 2, 4}) {
                    Cand c = base;
                    c.k.kernel = GBSP_KERNEL_VECTOR;
                    c.k.lanes = l;
                    c.k.rows_per_warp = r;
                    out.push_back(c);
                }
            for (auto lr : {std::make_pair(1, 8), std::make_pair(2, 4), std::make_pair(2, 8),
                            std::make_pair(4, 4), std::make_pair(4, 8), std::make_pair(8, 8)}) {
                Cand c = base;
                c.k.kernel = GBSP_KERNEL_RUNS;
                c.k.lanes = lr.first;
                c.k.rows_per_warp = lr.second;
                out.push_back(c);
            }
            if (A.tile_rows) {
                Cand c = base;
                c.k.kernel = GBSP_KERNEL_TILED;
                out.push_back(c);
            }
        } else {
            for (int t : {4, 8, 16}) {
                Cand c = base;
                c.k.kernel = GBSP_KERNEL_VECTOR;
                c.k.rhs_tile = t;
                out.push_back(c);
            }
        }
    } else if (A.built_block > 0) {
        if (k == 1 && (A.format == GBSP_SELL || A.format == GBSP_PSELL)) {
            for (int u : {1, 2, 4}) {
                Cand c = base;
                c.unroll = u;
                out.push_back(c);
            }
        } else if (k == 1) {
            out.push_back(base);
        } else {
            for (int t : {4, 8, 16}) {
                Cand c = base;
                c.k.rhs_tile = t;
                out.push_back(c);
            }
        }
    } else {
        if (k == 1) {
            Cand c = base;
            c.format = GBSP_JDS;
            c.k.rows_per_warp = 1;
            out.push_back(c);
            for (int u : {2, 4, 8})
                for (int r : {1, 2, 4}) {
                    if (u == 8 && r == 4) continue;
                    c = base;
                    c.format = GBSP_NUJDS;
                    c.unroll = u;
                    c.k.rows_per_warp = r;
                    out.push_back(c);
                }
            for (int b : {256, 1024, 2048}) {
                c = base;
                c.k.rows_per_warp = 1;
                c.format = GBSP_NBJDS;
                c.block = b;
                out.push_back(c);
            }
        } else {
            for (int t : {4, 8, 16}) {
                Cand c = base;
                c.format = GBSP_JDS;
                c.k.rhs_tile = t;
                out.push_back(c);
            }
        }
    }
    return out;
}

}  // namespace gbsp

using namespace gbsp;

extern "C" gbsp_status gbsp_autotune(gbsp_handle h, int32_t k, const void *d_X, void *d_Y, void *stream,
                                     gbsp_kernel_opts *best, float *best_ms) {
    if (!h || k < 1) return arg_error("gbsp_autotune: bad arguments");
    if (h->kind == KIND_DIA) {
        set_error("gbsp_autotune: a DIA handle has one kernel");
        return GBSP_ERR_UNSUPPORTED;
    }
    if (h->n_rows > 0 && (!d_X || !d_Y)) return arg_error("gbsp_autotune: NULL scratch vectors");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TuneKey key = key_of(*h, k);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply(*h, it->second.first);
            if (best) gbsp_get_kernel(h, best);
            if (best_ms) *best_ms = it->second.second;
            return GBSP_OK;
        }
    }
    VecArgs v{};
    v.x = d_X;
    v.y = d_Y;
    v.ldx = k;
    v.ldy = k;
    v.k = k;
    cudaEvent_t e0, e1;
    GBSP_CUDA(cudaEventCreate(&e0));
    GBSP_CUDA(cudaEventCreate(&e1));
    Cand top{};
    float top_ms = -1.f;
    gbsp_status st = GBSP_OK;
    for (const Cand &c : candidates(*h, k)) {
        apply(*h, c);
        float ms = 0;
        st = time_one(*h, v, s, e0, e1, &ms);
        if (st != GBSP_OK) break;
        if (top_ms < 0 || ms < top_ms) {
            top = c;
            top_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBSP_OK) return st;
    if (top_ms >= 0) apply(*h, top);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = std::make_pair(top, top_ms);
    }
    if (best) gbsp_get_kernel(h, best);
    if (best_ms) *best_ms = top_ms;
    return GBSP_OK;
}
