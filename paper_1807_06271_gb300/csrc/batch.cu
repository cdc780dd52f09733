// Many pairs per call: every pair's pipeline runs on its own branch of one
// CUDA graph, captured on first use and replayed while the same handles and
// buffers come back; and the autotuner that picks the aggregation kernel's
// resident blocks per SM for a given image shape and parameter set.
#include <algorithm>
#include <mutex>
#include <vector>

#include "sgm_handle.cuh"

namespace {

struct BatchKey {
    std::vector<const void *> v;  // handles, buffers and tuning of every pair
    bool operator==(const BatchKey &o) const { return v == o.v; }
};

struct BatchGraph {
    BatchKey key;
    int device;
    cudaGraphExec_t exec;
    unsigned long long last_use;
};

constexpr size_t kMaxGraphs = 8;
std::mutex g_mu;
std::vector<BatchGraph> g_graphs;
unsigned long long g_clock = 0;

struct TuneKey {
    int W, H, D, mask, cw, ch, P2, cost;
    bool operator==(const TuneKey &o) const {
        return W == o.W && H == o.H && D == o.D && mask == o.mask && cw == o.cw && ch == o.ch && P2 == o.P2 &&
               cost == o.cost;
    }
};
std::vector<std::pair<TuneKey, sgm::Tuning>> g_tuned;

TuneKey tune_key(const sgm_handle_s *h) {
    return {h->W, h->H, h->D, h->p.path_mask, h->p.census_w, h->p.census_h, h->p.P2, h->p.cost};
}

void drop(BatchGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
}

// Direct launches on forked side streams (no graph).
int run_forked(int n, const sgm_handle *hs, const uint8_t *const *left, const uint8_t *const *right,
               uint8_t *const *disp, uint16_t *const *umap, uint16_t *const *vmap, cudaStream_t s) {
    int rc = SGM_OK;
    int forked = 0;
    for (int i = 0; i < n && rc == SGM_OK; i++, forked++) {
        sgm_handle_s *h = hs[i];
        if (cudaEventRecord(h->fork_ev, s) != cudaSuccess ||
            cudaStreamWaitEvent(h->side, h->fork_ev, 0) != cudaSuccess) {
            rc = SGM_ERR_CUDA;
            break;
        }
        rc = sgm::compute_pair(h, left[i], right[i], disp[i], umap ? umap[i] : nullptr,
                               vmap ? vmap[i] : nullptr, h->side);
    }
    // join every side stream that was forked, whatever happened
    for (int i = 0; i < forked; i++) {
        sgm_handle_s *h = hs[i];
        if (cudaEventRecord(h->join_ev, h->side) != cudaSuccess ||
            cudaStreamWaitEvent(s, h->join_ev, 0) != cudaSuccess)
            rc = rc == SGM_OK ? SGM_ERR_CUDA : rc;
    }
    return rc;
}

}  // namespace

void sgm::batch_forget(sgm_handle_s *h) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &g : g_graphs)
        if (std::find(g.key.v.begin(), g.key.v.end(), (const void *)h) != g.key.v.end()) drop(g);
    g_graphs.erase(std::remove_if(g_graphs.begin(), g_graphs.end(),
                                  [](const BatchGraph &g) { return g.exec == nullptr; }),
                   g_graphs.end());
}

sgm::Tuning sgm::tuned_for(const sgm_handle_s *h) {
    std::lock_guard<std::mutex> lock(g_mu);
    const TuneKey k = tune_key(h);
    for (auto &e : g_tuned)
        if (e.first == k) return e.second;
    return Tuning{0, SGM_SCHEDULE_PLANES, 4, 1};
}

extern "C" int sgm_batch_compute(int n, const sgm_handle *hs, const uint8_t *const *left,
                                 const uint8_t *const *right, uint8_t *const *disp,
                                 uint16_t *const *umap, uint16_t *const *vmap, void *stream) {
    if (n < 0 || (n > 0 && (!hs || !left || !right || !disp))) return SGM_ERR_INVALID_ARG;
    if (n == 0) return SGM_OK;
    bool timing = false;
    for (int i = 0; i < n; i++) {
        if (!hs[i] || !left[i] || !right[i] || !disp[i]) return SGM_ERR_INVALID_ARG;
        if (umap && vmap && ((!umap[i]) != (!vmap[i]))) return SGM_ERR_INVALID_ARG;
        if (hs[i]->device != hs[0]->device) return SGM_ERR_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (hs[j] == hs[i]) return SGM_ERR_INVALID_ARG;
        timing = timing || hs[i]->timing;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SGM_ERR_CUDA;
    const int dev = hs[0]->device;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = SGM_OK;
    if (timing) {
        // stage timing records events between kernels: launch directly
        rc = run_forked(n, hs, left, right, disp, umap, vmap, s);
    } else {
        BatchKey key;
        key.v.reserve(9 * n);
        for (int i = 0; i < n; i++) {
            key.v.push_back(hs[i]);
            key.v.push_back(left[i]);
            key.v.push_back(right[i]);
            key.v.push_back(disp[i]);
            key.v.push_back(umap && vmap ? (const void *)umap[i] : nullptr);
            key.v.push_back(umap && vmap ? (const void *)vmap[i] : nullptr);
            key.v.push_back((const void *)(intptr_t)hs[i]->agg_blocks_per_sm);
            key.v.push_back((const void *)(intptr_t)(hs[i]->schedule * 64 + hs[i]->sweep_rows));
            key.v.push_back((const void *)(intptr_t)hs[i]->agg_cpl);
        }
        std::lock_guard<std::mutex> lock(g_mu);
        BatchGraph *hit = nullptr;
        for (auto &g : g_graphs)
            if (g.device == dev && g.key == key) hit = &g;
        if (!hit) {
            // capture every pair's pipeline, forked from one capture stream
            cudaStream_t cap = nullptr;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) rc = SGM_ERR_CUDA;
            if (rc == SGM_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                rc = SGM_ERR_CUDA;
            if (rc == SGM_OK) {
                const int brc = run_forked(n, hs, left, right, disp, umap, vmap, cap);
                const cudaError_t e = cudaStreamEndCapture(cap, &graph);
                if (brc != SGM_OK) rc = brc;
                else if (e != cudaSuccess) rc = SGM_ERR_CUDA;
            }
            if (rc == SGM_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = SGM_ERR_CUDA;
            if (graph) cudaGraphDestroy(graph);
            if (cap) cudaStreamDestroy(cap);
            if (rc != SGM_OK) {
                if (exec) cudaGraphExecDestroy(exec);
                cudaGetLastError();
            } else {
                if (g_graphs.size() >= kMaxGraphs) {  // evict the least recently used graph
                    auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                                [](const BatchGraph &a, const BatchGraph &b) {
                                                    return a.last_use < b.last_use;
                                                });
                    drop(*lru);
                    g_graphs.erase(lru);
                }
                g_graphs.push_back({key, dev, exec, 0});
                hit = &g_graphs.back();
            }
        }
        if (rc == SGM_OK) {
            hit->last_use = ++g_clock;
            if (cudaGraphLaunch(hit->exec, s) != cudaSuccess) rc = SGM_ERR_CUDA;
        }
    }
    if (prev != dev) cudaSetDevice(prev);
    return rc;
}

extern "C" int sgm_autotune(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                            void *stream, int *best_blocks_per_sm) {
    if (!h || !left || !right || !disp) return SGM_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SGM_ERR_CUDA;
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SGM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SGM_ERR_CUDA;
    const int saved = h->agg_blocks_per_sm, saved_timing = h->timing, saved_cpl = h->agg_cpl;
    const int saved_schedule = h->schedule, saved_rows = h->sweep_rows;
    h->timing = 0;
    // candidates: the plane schedule at each resident-block count and each
    // number of chunks per lane, then the fused sweep at each rows-per-CTA
    // count it can run with
    struct Cand {
        int schedule, param, cpl;
    };
    std::vector<Cand> cands;
    const int cmax = sgm::chunks_per_lane_max(h->D, h->wide != 0);
    for (int cpl : {1, 2, sgm::kMixedCpl, 4})
        if ((cpl == sgm::kMixedCpl ? 2 : cpl) <= cmax)
            for (int c : {1, 2, 3, 4, 6}) cands.push_back({SGM_SCHEDULE_PLANES, c, cpl});
    for (int r : {2, 4, 8})
        if (sgm::sweep_feasible(h, r) == SGM_OK) cands.push_back({SGM_SCHEDULE_SWEEP, r, saved_cpl});
    int best_bps = saved, best_cpl = saved_cpl;
    Cand best{saved_schedule, saved_schedule == SGM_SCHEDULE_SWEEP ? saved_rows : saved, saved_cpl};
    float best_ms = 1e30f, best_planes_ms = 1e30f;
    for (const Cand &c : cands) {
        if (rc != SGM_OK) break;
        h->schedule = c.schedule;
        if (c.schedule == SGM_SCHEDULE_SWEEP) {
            h->sweep_rows = c.param;
        } else {
            h->agg_blocks_per_sm = c.param;
            h->agg_cpl = c.cpl;
        }
        for (int w = 0; w < 2 && rc == SGM_OK; w++)
            rc = sgm::compute_pair(h, left, right, disp, nullptr, nullptr, s);
        if (rc != SGM_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = SGM_ERR_CUDA;
        for (int r = 0; r < 5 && rc == SGM_OK; r++)
            rc = sgm::compute_pair(h, left, right, disp, nullptr, nullptr, s);
        float ms = 0.f;
        if (rc == SGM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = SGM_ERR_CUDA;
        if (rc == SGM_OK && c.schedule == SGM_SCHEDULE_PLANES && ms < best_planes_ms) {
            best_planes_ms = ms;
            best_bps = c.param;
            best_cpl = c.cpl;
        }
        if (rc == SGM_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    h->timing = saved_timing;
    if (rc == SGM_OK) {
        h->agg_blocks_per_sm = best_bps;
        h->agg_cpl = best_cpl;
        h->schedule = best.schedule;
        h->sweep_rows = best.schedule == SGM_SCHEDULE_SWEEP ? best.param : saved_rows;
    } else {
        h->agg_blocks_per_sm = saved;
        h->agg_cpl = saved_cpl;
        h->schedule = saved_schedule;
        h->sweep_rows = saved_rows;
    }
    sgm::batch_forget(h);
    if (rc == SGM_OK) {
        std::lock_guard<std::mutex> lock(g_mu);
        const TuneKey k = tune_key(h);
        const sgm::Tuning t{best_bps, h->schedule, h->sweep_rows, best_cpl};
        bool found = false;
        for (auto &e : g_tuned)
            if (e.first == k) {
                e.second = t;
                found = true;
            }
        if (!found) g_tuned.push_back({k, t});
        if (best_blocks_per_sm) *best_blocks_per_sm = best_bps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    if (prev != h->device) cudaSetDevice(prev);
    return rc;
}
