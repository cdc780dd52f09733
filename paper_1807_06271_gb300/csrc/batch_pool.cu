// The batch engine: many stereo pairs of uneven size and disparity range
// (each the method of Sec. 3.1) from one pooled scratch allocation, with the
// path aggregation of all pairs in one persistent launch.
//
// Per call the engine runs, as one CUDA graph (captured on the first call and
// replayed while the same buffers and tuning come back):
//   per pair, on its own branch: census, matching cost;
//   per group of pairs: one persistent aggregation launch whose work list
//     holds every (pair, direction, scanline group) job of the group, the
//     long-axis scanlines of all its pairs first;
//   per pair, on its own branch: WTA + right WTA + LR check, median, U/V.
// With more than one group the groups' branches run side by side, so one
// group's HBM-bound WTA passes overlap another group's aggregation.  A group
// of one pair runs the single-pair chain instead (its own aggregation kernel
// on the pair's stream, the work-queue state cleared by the cost kernel), so
// that with one group per pair the engine does what a graph of handles does,
// from the pool.  The
// tuner (sgm_batch_autotune) picks the number of groups (up to one per pair,
// which is one aggregation launch per pair) and the aggregation kernel's
// resident blocks per SM.
#include <stdlib.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sgm_handle.cuh"

using namespace sgm;

namespace {

struct PairSlot {
    int W, H, D, Dp;
    size_t codes, cost, planes, disp_lr;  // offsets in the pool
    cudaStream_t side;
    cudaEvent_t ready, done;  // costs ready / pair finished (graph capture)
};

struct Group {
    std::vector<int> pairs;
    size_t table, prefix, job_state;  // offsets in the pool
    cudaStream_t stream;
    cudaEvent_t aggregated;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct sgm_batch_s {
    int n;
    sgm_params p;
    int device;
    int nbits, code_bytes, wide, npaths;
    std::vector<PairSlot> pairs;
    std::vector<Group> groups;
    int ngroups, blocks_per_sm;
    int cpl;      // chunks per lane of the batched aggregation (1 or 4)
    int cpl_max;  // 4 when every pair allows it, else 1
    unsigned char *pool;
    size_t pool_bytes;  // the whole pool
    size_t tables_at;   // where the group tables start (after the pairs' scratch)
    cudaEvent_t origin;
    // the captured graph and what it was captured for
    cudaGraphExec_t exec;
    std::vector<const void *> key;
};

namespace {

void free_streams(sgm_batch_s *b) {
    for (PairSlot &ps : b->pairs) {
        if (ps.side) cudaStreamDestroy(ps.side);
        if (ps.ready) cudaEventDestroy(ps.ready);
        if (ps.done) cudaEventDestroy(ps.done);
        ps.side = nullptr;
        ps.ready = ps.done = nullptr;
    }
    for (Group &g : b->groups) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.aggregated) cudaEventDestroy(g.aggregated);
    }
    b->groups.clear();
}

void free_batch(sgm_batch_s *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_streams(b);
    if (b->origin) cudaEventDestroy(b->origin);
    if (b->pool) cudaFree(b->pool);
    delete b;
}

// Deals the pairs, largest work first, round-robin into `ng` groups and lays
// out each group's job table, prefix sums and work-queue state in the pool
// region that starts at `at` (returns the end).  With upload, copies the
// tables to the device.
int layout_groups(sgm_batch_s *b, int ng, bool upload, size_t at, size_t *end) {
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const PairSlot &x = b->pairs[a], &y = b->pairs[c];
        return (long long)x.W * x.H * x.Dp > (long long)y.W * y.H * y.Dp;
    });
    std::vector<Group> gs(ng);
    for (int i = 0; i < b->n; i++) gs[i % ng].pairs.push_back(order[i]);
    for (Group &g : gs) {
        const int np = (int)g.pairs.size();
        g.table = at;
        at = align256(at + sizeof(BatchAggPair) * (size_t)np);
        g.prefix = at;
        at = align256(at + sizeof(int) * 2 * (size_t)(np + 1));
        g.job_state = at;
        at = align256(at + kJobStateBytes);
        if (!upload) continue;
        // pairs in the queues: longest scanlines first
        std::stable_sort(g.pairs.begin(), g.pairs.end(), [&](int a, int c) {
            const PairSlot &x = b->pairs[a], &y = b->pairs[c];
            return std::max(x.W, x.H) > std::max(y.W, y.H);
        });
        std::vector<BatchAggPair> table(np);
        std::vector<int> prefix(2 * (size_t)(np + 1), 0);
        for (int k = 0; k < np; k++) {
            const PairSlot &ps = b->pairs[g.pairs[k]];
            BatchAggPair &t = table[k];
            t.cost = b->pool + ps.cost;
            t.planes = b->pool + ps.planes;
            t.W = ps.W;
            t.H = ps.H;
            t.D = ps.D;
            t.lps = lanes_per_scanline(ps.D) / b->cpl;
            t.ragged = ps.D != 8 * lanes_per_scanline(ps.D);
            t.nplanes = b->npaths;
            t.jobs = make_path_jobs(ps.W, ps.H, ps.D, b->p.path_mask, b->cpl);
            prefix[k + 1] = prefix[k] + t.jobs.nlong;
            prefix[np + 1 + k + 1] = prefix[np + 1 + k] + (t.jobs.jbegin[t.jobs.n] - t.jobs.nlong);
        }
        if (cudaMemcpy(b->pool + g.table, table.data(), sizeof(BatchAggPair) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->pool + g.prefix, prefix.data(), sizeof(int) * prefix.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            return SGM_ERR_CUDA;
        }
    }
    if (upload) b->groups = std::move(gs);
    *end = at;
    return SGM_OK;
}

// Streams and events of the pairs and groups (first use of a grouping).
int make_streams(sgm_batch_s *b) {
    for (PairSlot &ps : b->pairs) {
        if (ps.side) continue;
        if (cudaStreamCreateWithFlags(&ps.side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ps.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ps.done, cudaEventDisableTiming) != cudaSuccess)
            return SGM_ERR_CUDA;
    }
    for (Group &g : b->groups) {
        if (g.pairs.size() == 1) continue;  // runs on its pair's stream
        if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.aggregated, cudaEventDisableTiming) != cudaSuccess)
            return SGM_ERR_CUDA;
    }
    return SGM_OK;
}

// The batch's work on stream s (directly, or into a capture of s).
int enqueue(sgm_batch_s *b, const uint8_t *const *left, const uint8_t *const *right, uint8_t *const *disp,
            uint16_t *const *umap, uint16_t *const *vmap, cudaStream_t s) {
    if (cudaEventRecord(b->origin, s) != cudaSuccess) return SGM_ERR_CUDA;
    const RectMaps no_maps{nullptr, nullptr, nullptr, nullptr};
    // census and matching cost of pair i on its own stream; a non-null
    // job_state is cleared by the cost kernel
    auto costs = [&](int i, unsigned *job_state) -> cudaError_t {
        PairSlot &ps = b->pairs[i];
        if (cudaStreamWaitEvent(ps.side, b->origin, 0) != cudaSuccess) return cudaErrorUnknown;
        if (b->wide)
            return launch_sad_cost(left[i], right[i], ps.W, ps.W, ps.H, ps.D, b->p.census_w, b->p.census_h, no_maps,
                                   reinterpret_cast<uint16_t *>(b->pool + ps.cost), job_state, ps.side);
        cudaError_t e = launch_census(left[i], right[i], ps.W, ps.W, ps.H, b->p.census_w, b->p.census_h,
                                      b->code_bytes, b->pool + ps.codes, no_maps, ps.side);
        if (e == cudaSuccess)
            e = launch_cost(b->pool + ps.codes, b->code_bytes, ps.W, ps.H, ps.D, b->nbits, b->pool + ps.cost,
                            job_state, nullptr, SGM_COST_KERNEL_AUTO, ps.side);
        return e;
    };
    // WTA + LR check, median and U/V of pair i on its own stream, then join s
    auto finish = [&](int i) -> int {
        PairSlot &ps = b->pairs[i];
        uint8_t *lr = b->pool + ps.disp_lr;
        cudaError_t e = launch_wta(b->pool + ps.planes, b->npaths, ps.W, ps.H, ps.D, b->wide != 0,
                                   b->p.lr_tolerance, lr, nullptr, nullptr, nullptr, ps.side);
        if (e == cudaSuccess)
            e = b->p.median_k <= 1 ? cudaMemcpyAsync(disp[i], lr, (size_t)ps.W * ps.H, cudaMemcpyDeviceToDevice, ps.side)
                                   : launch_median(lr, disp[i], ps.W, ps.H, b->p.median_k, ps.side);
        if (e == cudaSuccess && umap && vmap && umap[i] && vmap[i])
            e = launch_uvmap(disp[i], ps.W, ps.H, ps.D, umap[i], vmap[i], ps.side);
        if (e != cudaSuccess || cudaEventRecord(ps.done, ps.side) != cudaSuccess ||
            cudaStreamWaitEvent(s, ps.done, 0) != cudaSuccess)
            return SGM_ERR_CUDA;
        return SGM_OK;
    };
    for (Group &g : b->groups) {
        unsigned *job_state = reinterpret_cast<unsigned *>(b->pool + g.job_state);
        if (g.pairs.size() == 1) {
            // One pair: the single-pair chain on the pair's stream, with its
            // own specialised aggregation kernel; the cost kernel clears the
            // work-queue state, so every launch keeps the programmatic
            // (overlapped) dependency on the one before it.
            const int i = g.pairs[0];
            PairSlot &ps = b->pairs[i];
            const PathJobs jobs = make_path_jobs(ps.W, ps.H, ps.D, b->p.path_mask, b->cpl);
            if (costs(i, job_state) != cudaSuccess ||
                launch_aggregate(b->pool + ps.cost, ps.W, ps.H, ps.D, b->p.P1, b->p.P2, b->wide != 0, jobs,
                                 b->pool + ps.planes, b->npaths, job_state, b->blocks_per_sm, b->cpl,
                                 ps.side) != cudaSuccess)
                return SGM_ERR_CUDA;
            const int rc = finish(i);
            if (rc != SGM_OK) return rc;
            continue;
        }
        if (cudaStreamWaitEvent(g.stream, b->origin, 0) != cudaSuccess) return SGM_ERR_CUDA;
        for (int i : g.pairs) {
            PairSlot &ps = b->pairs[i];
            if (costs(i, nullptr) != cudaSuccess || cudaEventRecord(ps.ready, ps.side) != cudaSuccess ||
                cudaStreamWaitEvent(g.stream, ps.ready, 0) != cudaSuccess)
                return SGM_ERR_CUDA;
        }
        if (cudaMemsetAsync(job_state, 0, kJobStateBytes, g.stream) != cudaSuccess ||
            launch_aggregate_batch(reinterpret_cast<const BatchAggPair *>(b->pool + g.table), (int)g.pairs.size(),
                                   reinterpret_cast<const int *>(b->pool + g.prefix), b->p.P1, b->p.P2, b->wide != 0,
                                   b->cpl, job_state, b->blocks_per_sm, g.stream) != cudaSuccess ||
            cudaEventRecord(g.aggregated, g.stream) != cudaSuccess)
            return SGM_ERR_CUDA;
        for (int i : g.pairs) {
            if (cudaStreamWaitEvent(b->pairs[i].side, g.aggregated, 0) != cudaSuccess) return SGM_ERR_CUDA;
            const int rc = finish(i);
            if (rc != SGM_OK) return rc;
        }
    }
    return SGM_OK;
}

int check_buffers(const sgm_batch_s *b, const uint8_t *const *left, const uint8_t *const *right,
                  uint8_t *const *disp, uint16_t *const *umap, uint16_t *const *vmap) {
    if (!left || !right || !disp) return SGM_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; i++) {
        if (!left[i] || !right[i] || !disp[i]) return SGM_ERR_INVALID_ARG;
        if (umap && vmap && ((!umap[i]) != (!vmap[i]))) return SGM_ERR_INVALID_ARG;
    }
    if ((!umap) != (!vmap)) return SGM_ERR_INVALID_ARG;
    return SGM_OK;
}

// Rebuilds the grouping (the device must be idle for b: the tables are
// overwritten in place).
int regroup(sgm_batch_s *b, int groups) {
    if (groups == b->ngroups && !b->groups.empty()) return SGM_OK;
    free_streams(b);
    size_t end = 0;
    const int rc = layout_groups(b, groups, true, b->tables_at, &end);
    if (rc != SGM_OK) return rc;
    b->ngroups = groups;
    return make_streams(b);
}

struct DeviceSwitch {
    int prev = -1;
    bool ok = true;
    explicit DeviceSwitch(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess || (prev != dev && cudaSetDevice(dev) != cudaSuccess)) {
            ok = false;
            cudaGetLastError();
        }
    }
    ~DeviceSwitch() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr int kMaxGroups = 64;

}  // namespace

extern "C" {

int sgm_batch_create(int n, const int *W, const int *H, const int *D, const sgm_params *params, sgm_batch *out) {
    if (!out) return SGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !W || !H || !D || !params) return SGM_ERR_INVALID_ARG;
    if (params->row_pitch != 0) return SGM_ERR_INVALID_ARG;  // pairs of different widths: dense rows only
    for (int i = 0; i < n; i++) {
        const int rc = validate_params(W[i], H[i], D[i], params);
        if (rc != SGM_OK) return rc;
    }
    sgm_batch_s *b = new (std::nothrow) sgm_batch_s();
    if (!b) return SGM_ERR_OOM;
    b->n = n;
    b->p = *params;
    b->wide = params->cost == SGM_COST_SAD;
    b->nbits = b->wide ? params->census_w * params->census_h * 255 : params->census_w * params->census_h - 1;
    b->code_bytes = b->wide ? 0 : (b->nbits <= 32 ? 4 : 8);
    b->npaths = __builtin_popcount((unsigned)params->path_mask);
    b->ngroups = n;
    b->blocks_per_sm = 3;
    b->cpl = 1;
    b->cpl_max = 4;
    for (int i = 0; i < n; i++)
        if (chunks_per_lane_max(D[i], b->wide != 0) < 4) b->cpl_max = 1;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    // the pool: every pair's codes, cost volume, planes and LR map, then the
    // job tables of the largest grouping (kMaxGroups groups)
    b->pairs.resize(n);
    size_t at = 0;
    for (int i = 0; i < n; i++) {
        PairSlot &ps = b->pairs[i];
        ps = PairSlot{};
        ps.W = W[i];
        ps.H = H[i];
        ps.D = D[i];
        ps.Dp = padded_disparities(D[i]);
        const ScratchSizes sz = scratch_sizes(W[i], H[i], D[i], params);
        ps.codes = at;
        at = align256(at + sz.codes);
        ps.cost = at;
        at = align256(at + sz.cost);
        ps.planes = at;
        at = align256(at + sz.planes);
        ps.disp_lr = at;
        at = align256(at + sz.disp_lr);
    }
    b->tables_at = at;
    size_t tables_end = at;
    for (int g = 1;; g *= 2) {  // every allowed grouping: powers of two up to kMaxGroups, and n
        const int ng = g <= kMaxGroups ? std::min(g, n) : n;
        size_t end = 0;
        layout_groups(b, ng, false, b->tables_at, &end);
        tables_end = std::max(tables_end, end);
        if (g > kMaxGroups) break;
    }
    b->pool_bytes = tables_end;
    void *pool = nullptr;
    if (cudaMalloc(&pool, b->pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return SGM_ERR_OOM;
    }
    b->pool = (unsigned char *)pool;
    b->ngroups = 0;
    int rc = cudaEventCreateWithFlags(&b->origin, cudaEventDisableTiming) == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
    if (rc == SGM_OK) rc = regroup(b, n);
    if (rc != SGM_OK) {
        cudaGetLastError();
        free_batch(b);
        return rc;
    }
    *out = b;
    return SGM_OK;
}

int sgm_batch_destroy(sgm_batch b) {
    if (!b) return SGM_ERR_INVALID_ARG;
    DeviceSwitch on(b->device);
    cudaDeviceSynchronize();
    free_batch(b);
    return SGM_OK;
}

int sgm_batch_device_bytes(sgm_batch b, size_t *bytes) {
    if (!b || !bytes) return SGM_ERR_INVALID_ARG;
    *bytes = b->pool_bytes;
    return SGM_OK;
}

int sgm_batch_set_tuning(sgm_batch b, int groups, int blocks_per_sm, int chunks_per_lane) {
    if (!b || groups < 1 || blocks_per_sm < 1 || blocks_per_sm > 16) return SGM_ERR_INVALID_ARG;
    if (groups != b->n && (groups > kMaxGroups || (groups & (groups - 1)))) return SGM_ERR_INVALID_ARG;
    if (chunks_per_lane != 1 && chunks_per_lane != 4) return SGM_ERR_INVALID_ARG;
    if (chunks_per_lane > b->cpl_max) return SGM_ERR_UNSUPPORTED;
    DeviceSwitch on(b->device);
    if (!on.ok) return SGM_ERR_CUDA;
    const int ng = std::min(groups, b->n);
    if (ng != b->ngroups || chunks_per_lane != b->cpl) {
        // the tables are rewritten in place: nothing of b may still run
        if (cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return SGM_ERR_CUDA;
        }
        b->cpl = chunks_per_lane;
        b->ngroups = 0;  // force the rebuild
        const int rc = regroup(b, ng);
        if (rc != SGM_OK) return rc;
    }
    b->blocks_per_sm = blocks_per_sm;  // a changed tuning is captured anew by the next run
    return SGM_OK;
}

int sgm_batch_get_tuning(sgm_batch b, int *groups, int *blocks_per_sm, int *chunks_per_lane) {
    if (!b) return SGM_ERR_INVALID_ARG;
    if (groups) *groups = b->ngroups;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    if (chunks_per_lane) *chunks_per_lane = b->cpl;
    return SGM_OK;
}

int sgm_batch_run(sgm_batch b, const uint8_t *const *left, const uint8_t *const *right, uint8_t *const *disp,
                  uint16_t *const *umap, uint16_t *const *vmap, void *stream) {
    if (!b) return SGM_ERR_INVALID_ARG;
    int rc = check_buffers(b, left, right, disp, umap, vmap);
    if (rc != SGM_OK) return rc;
    DeviceSwitch on(b->device);
    if (!on.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const void *> key;
    key.reserve(5 * (size_t)b->n + 2);
    for (int i = 0; i < b->n; i++) {
        key.push_back(left[i]);
        key.push_back(right[i]);
        key.push_back(disp[i]);
        key.push_back(umap && vmap ? (const void *)umap[i] : nullptr);
        key.push_back(umap && vmap ? (const void *)vmap[i] : nullptr);
    }
    key.push_back((const void *)(intptr_t)b->ngroups);
    key.push_back((const void *)(intptr_t)b->blocks_per_sm);
    key.push_back((const void *)(intptr_t)b->cpl);
    if (!b->exec || key != b->key) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->key.clear();
        cudaStream_t cap = nullptr;
        cudaGraph_t graph = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) rc = SGM_ERR_CUDA;
        if (rc == SGM_OK && cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            rc = SGM_ERR_CUDA;
        if (rc == SGM_OK) {
            const int erc = enqueue(b, left, right, disp, umap, vmap, cap);
            const cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (erc != SGM_OK) rc = erc;
            else if (e != cudaSuccess) rc = SGM_ERR_CUDA;
        }
        if (rc == SGM_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = SGM_ERR_CUDA;
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (rc != SGM_OK) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            cudaGetLastError();
            return rc;
        }
        b->key = key;
    }
    return cudaGraphLaunch(b->exec, s) == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int sgm_batch_autotune(sgm_batch b, const uint8_t *const *left, const uint8_t *const *right, uint8_t *const *disp,
                       uint16_t *const *umap, uint16_t *const *vmap, void *stream, int *best_groups,
                       int *best_blocks_per_sm, int *best_chunks_per_lane) {
    if (!b) return SGM_ERR_INVALID_ARG;
    int rc = check_buffers(b, left, right, disp, umap, vmap);
    if (rc != SGM_OK) return rc;
    DeviceSwitch on(b->device);
    if (!on.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SGM_ERR_CUDA;
    int bg = b->ngroups, bb = b->blocks_per_sm, bc = b->cpl;
    float best = 1e30f;
    for (int cpl : {1, 4}) {
        if (cpl > b->cpl_max) break;
        // 1, 2, 4, ... groups below one per pair, then one group per pair
        std::vector<int> gs;
        for (int g = 1; g < b->n && g <= kMaxGroups; g *= 2) gs.push_back(g);
        gs.push_back(b->n);
        for (int g : gs) {
            if (rc != SGM_OK) break;
            for (int bps : {2, 3, 4}) {
                rc = sgm_batch_set_tuning(b, g, bps, cpl);
                for (int w = 0; w < 2 && rc == SGM_OK; w++) rc = sgm_batch_run(b, left, right, disp, umap, vmap, stream);
                if (rc != SGM_OK) break;
                float ms = 0.f;
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = SGM_ERR_CUDA;
                for (int r = 0; r < 3 && rc == SGM_OK; r++) rc = sgm_batch_run(b, left, right, disp, umap, vmap, stream);
                if (rc == SGM_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = SGM_ERR_CUDA;
                if (rc == SGM_OK && ms < best) {
                    best = ms;
                    bg = g;
                    bb = bps;
                    bc = cpl;
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc == SGM_OK) rc = sgm_batch_set_tuning(b, bg, bb, bc);
    if (rc == SGM_OK) {
        if (best_groups) *best_groups = b->ngroups;
        if (best_blocks_per_sm) *best_blocks_per_sm = b->blocks_per_sm;
        if (best_chunks_per_lane) *best_chunks_per_lane = b->cpl;
    }
    cudaGetLastError();
    return rc;
}

}  // extern "C"
