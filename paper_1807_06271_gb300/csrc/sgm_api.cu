// The C ABI of libsgm: handle life cycle, argument checks, scratch ownership,
// the stage sequence of one pair and CUDA-event stage timing.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sgm_handle.cuh"

using namespace sgm;

namespace {

constexpr int kTimingRing = 1024;

const char *const kStageNames[kNumStages] = {"census", "cost", "aggregate", "wta_lr", "median", "uvmap", "sweep"};
// NVTX push/pop range around each stage's launches (host side; a tool attached
// to the process can select kernels by range, e.g. ncu --nvtx --nvtx-include
// "sgm:aggregate/").  Stage ranges are not nested in a per-pair range, so they
// match at the top level of an application that opens none itself.
const char *const kStageRanges[kNumStages] = {"sgm:census", "sgm:cost", "sgm:aggregate",
                                              "sgm:wta_lr", "sgm:median", "sgm:uvmap", "sgm:sweep"};

int validate(int W, int H, int D, const sgm_params *p) {
    if (!p || W < 1 || H < 1 || D < 1) return SGM_ERR_INVALID_ARG;
    if (p->census_w < 1 || p->census_h < 1 || !(p->census_w & 1) || !(p->census_h & 1))
        return SGM_ERR_INVALID_ARG;
    if (p->path_mask <= 0 || p->path_mask > 0xFF) return SGM_ERR_INVALID_ARG;
    if (p->P1 < 0 || p->P2 < p->P1) return SGM_ERR_INVALID_ARG;
    if (p->row_pitch != 0 && p->row_pitch < W) return SGM_ERR_INVALID_ARG;
    if (p->median_k < 0 || (p->median_k > 1 && !(p->median_k & 1))) return SGM_ERR_INVALID_ARG;
    if (p->cost != SGM_COST_CENSUS && p->cost != SGM_COST_SAD) return SGM_ERR_INVALID_ARG;
    const int npaths = __builtin_popcount((unsigned)p->path_mask);
    if (p->cost == SGM_COST_CENSUS) {
        const int nbits = p->census_w * p->census_h - 1;
        if (nbits > 64) return SGM_ERR_UNSUPPORTED;
        if (nbits + p->P2 > 255) return SGM_ERR_UNSUPPORTED;  // L_r must fit a byte
    } else {
        if (p->census_w > kMaxSadWindow || p->census_h > kMaxSadWindow) return SGM_ERR_UNSUPPORTED;
        // 16-bit path costs: below the 0x7FFF padding marker, and their sum over
        // the paths within 16 bits
        const long long top = (long long)p->census_w * p->census_h * 255 + p->P2;
        if (top > 0x7FFE || top * npaths > 0xFFFF) return SGM_ERR_UNSUPPORTED;
    }
    if (D > kMaxD || W > kMaxW || H > 65535) return SGM_ERR_UNSUPPORTED;
    if (p->median_k > 7) return SGM_ERR_UNSUPPORTED;
    // kernels index the per-path planes with 32-bit counts of lane chunks (one
    // lane's disparities of one pixel); the cost ring's index runs up to 16
    // steps of W + 1 pixels past a scanline's end
    const long long chunks = ((long long)W * H * npaths + 64ll * (W + 1)) * lanes_per_scanline(D);
    if (chunks >= (1ll << 31)) return SGM_ERR_UNSUPPORTED;
    return SGM_OK;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---- stage timing --------------------------------------------------------

void harvest(sgm_handle_s *h, TimingRecord &rec) {
    float ms = 0.f;
    if (cudaEventSynchronize(rec.stop) == cudaSuccess &&
        cudaEventElapsedTime(&ms, rec.start, rec.stop) == cudaSuccess) {
        h->acc_ms[rec.stage] += ms;
        h->acc_n[rec.stage] += 1;
    }
}

TimingRecord *stage_begin(sgm_handle_s *h, int stage, cudaStream_t s) {
    nvtxRangePushA(kStageRanges[stage]);
    if (!h->timing || !h->recs) return nullptr;
    TimingRecord *rec;
    if (h->rec_count == kTimingRing) {  // ring full: fold the oldest record first
        rec = &h->recs[h->rec_head];
        harvest(h, *rec);
        h->rec_head = (h->rec_head + 1) % kTimingRing;
        h->rec_count--;
    }
    rec = &h->recs[(h->rec_head + h->rec_count) % kTimingRing];
    rec->stage = stage;
    cudaEventRecord(rec->start, s);
    return rec;
}

void stage_end(sgm_handle_s *h, TimingRecord *rec, cudaStream_t s) {
    nvtxRangePop();
    if (!rec) return;
    cudaEventRecord(rec->stop, s);
    h->rec_count++;
}

// ---- the pipeline -----------------------------------------------------------

int run_census(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, cudaStream_t s) {
    if (h->wide) return SGM_ERR_UNSUPPORTED;  // the SAD cost has no census codes
    const int pitch = h->p.row_pitch ? h->p.row_pitch : h->W;
    TimingRecord *t = stage_begin(h, kStageCensus, s);
    cudaError_t e = launch_census(left, right, pitch, h->W, h->H, h->p.census_w, h->p.census_h,
                                  h->code_bytes, h->codes, h->rect, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int run_cost(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, cudaStream_t s) {
    TimingRecord *t = stage_begin(h, kStageCost, s);
    cudaError_t e;
    if (h->wide) {
        const int pitch = h->p.row_pitch ? h->p.row_pitch : h->W;
        e = launch_sad_cost(left, right, pitch, h->W, h->H, h->D, h->p.census_w, h->p.census_h, h->rect,
                            reinterpret_cast<uint16_t *>(h->cost), h->job_counter, s);
    } else {
        e = launch_cost(h->codes, h->code_bytes, h->W, h->H, h->D, h->nbits, h->cost, h->job_counter, h->dev_status,
                        h->cost_kernel, s);
    }
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

// The matching-cost volume of one pair: census codes then Hamming costs, or SAD.
int run_matching(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, cudaStream_t s) {
    int rc = h->wide ? SGM_OK : run_census(h, left, right, s);
    if (rc == SGM_OK) rc = run_cost(h, left, right, s);
    return rc;
}

// All enabled directions into h->planes, or direction only_r alone into plane 0.
int run_aggregate(sgm_handle_s *h, int only_r, cudaStream_t s) {
    const int mask = only_r >= 0 ? (1 << only_r) : h->p.path_mask;
    const PathJobs jobs = h->agg_cpl == kMixedCpl ? make_path_jobs_mixed(h->W, h->H, h->D, mask, 1, 2)
                                                  : make_path_jobs(h->W, h->H, h->D, mask, h->agg_cpl);
    TimingRecord *t = stage_begin(h, kStageAggregate, s);
    cudaError_t e = launch_aggregate(h->cost, h->W, h->H, h->D, h->p.P1, h->p.P2, h->wide != 0, jobs, h->planes,
                                     only_r >= 0 ? 1 : h->npaths, h->job_counter, h->agg_blocks_per_sm, h->agg_cpl, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int run_wta(sgm_handle_s *h, uint8_t *dbg_left, uint8_t *dbg_right, uint16_t *dbg_sum,
            cudaStream_t s) {
    TimingRecord *t = stage_begin(h, kStageWta, s);
    cudaError_t e = launch_wta(h->planes, h->npaths, h->W, h->H, h->D, h->wide != 0,
                               h->p.lr_tolerance, h->disp_lr, dbg_left, dbg_right, dbg_sum, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int run_median(sgm_handle_s *h, uint8_t *disp, cudaStream_t s) {
    TimingRecord *t = stage_begin(h, kStageMedian, s);
    cudaError_t e;
    if (h->p.median_k <= 1)
        e = cudaMemcpyAsync(disp, h->disp_lr, (size_t)h->W * h->H, cudaMemcpyDeviceToDevice, s);
    else
        e = launch_median(h->disp_lr, disp, h->W, h->H, h->p.median_k, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

// The fused streaming sweep (cost, paths, both winners, LR check) into h->disp_lr.
int run_sweep(sgm_handle_s *h, uint8_t *dbg_left, uint8_t *dbg_right, cudaStream_t s) {
    TimingRecord *t = stage_begin(h, kStageSweep, s);
    cudaError_t e = launch_sweep(h->codes, h->code_bytes, h->W, h->H, h->D, h->nbits, h->p.P1, h->p.P2,
                                 h->p.path_mask, h->p.lr_tolerance, h->disp_lr, dbg_left, dbg_right,
                                 h->sweep_scratch, h->dev_status, h->sweep_rows, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int compute_on(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
               cudaStream_t s) {
    int rc;
    if (h->schedule == SGM_SCHEDULE_SWEEP) {
        rc = run_census(h, left, right, s);
        if (rc == SGM_OK) rc = run_sweep(h, nullptr, nullptr, s);
    } else {
        rc = run_matching(h, left, right, s);
        if (rc == SGM_OK) rc = run_aggregate(h, -1, s);
        if (rc == SGM_OK) rc = run_wta(h, nullptr, nullptr, nullptr, s);
    }
    if (rc == SGM_OK) rc = run_median(h, disp, s);
    return rc;
}

int uv_on(sgm_handle_s *h, const uint8_t *disp, uint16_t *umap, uint16_t *vmap, cudaStream_t s) {
    TimingRecord *t = stage_begin(h, kStageUv, s);
    cudaError_t e = launch_uvmap(disp, h->W, h->H, h->D, umap, vmap, s);
    stage_end(h, t, s);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

void free_handle(sgm_handle_s *h) {
    if (!h) return;
    for (int i = 0; i < h->nallocs; i++) cudaFree(h->allocs[i].base);
    for (IoSlot &sl : h->io) {
        if (sl.in_ready) cudaEventDestroy(sl.in_ready);
        if (sl.computed) cudaEventDestroy(sl.computed);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->recs) {
        for (int i = 0; i < kTimingRing; i++) {
            cudaEventDestroy(h->recs[i].start);
            cudaEventDestroy(h->recs[i].stop);
        }
        free(h->recs);
    }
    free(h);
}

// Test hooks (process-wide): the n-th device allocation from now fails
// (sgm_debug_fail_alloc), and handles created while canaries are on guard
// their allocations (sgm_debug_canaries).
std::atomic<int> g_fail_alloc_in{0};
std::atomic<int> g_canaries{0};

// A device buffer of `bytes` for handle h, recorded in h->allocs.
template <typename T>
int dev_alloc(sgm_handle_s *h, T **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (g_fail_alloc_in.load() > 0 && g_fail_alloc_in.fetch_sub(1) == 1) return SGM_ERR_OOM;
    if (h->nallocs == kMaxAllocs) return SGM_ERR_CUDA;
    const size_t pad = h->canaries ? kCanaryBytes : 0;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, bytes + 2 * pad);
    if (e == cudaSuccess && pad &&
        (cudaMemset(base, kCanaryByte, pad) != cudaSuccess ||
         cudaMemset((unsigned char *)base + pad + bytes, kCanaryByte, pad) != cudaSuccess)) {
        cudaFree(base);
        e = cudaErrorUnknown;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SGM_ERR_OOM : SGM_ERR_CUDA;
    }
    h->allocs[h->nallocs++] = DevAlloc{base, bytes};
    *p = reinterpret_cast<T *>((unsigned char *)base + pad);
    return SGM_OK;
}

// Frees the allocations made after the first `keep` (a failed multi-buffer setup).
void dev_release_after(sgm_handle_s *h, int keep) {
    while (h->nallocs > keep) cudaFree(h->allocs[--h->nallocs].base);
}

}  // namespace

// One pair (and its maps when umap/vmap are non-null) on stream s; used by
// the batched entry points in batch.cu.
int sgm::compute_pair(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                      uint16_t *umap, uint16_t *vmap, cudaStream_t s) {
    int rc = compute_on(h, left, right, disp, s);
    if (rc == SGM_OK && umap && vmap) rc = uv_on(h, disp, umap, vmap, s);
    return rc;
}

// Same host-side argument checks as sgm_create, for entry points without a handle.
int sgm::validate_params(int W, int H, int D, const sgm_params *p) { return validate(W, H, D, p); }

sgm::ScratchSizes sgm::scratch_sizes(int W, int H, int D, const sgm_params *p) {
    const bool wide = p->cost == SGM_COST_SAD;
    const int nbits = p->census_w * p->census_h - 1;
    const size_t code_bytes = wide ? 0 : (nbits <= 32 ? 4 : 8);
    const size_t eb = wide ? 2 : 1;  // bytes per cost / path cost
    const size_t npx = (size_t)W * H, Dp = (size_t)padded_disparities(D);
    const size_t npaths = (size_t)__builtin_popcount((unsigned)p->path_mask);
    ScratchSizes s;
    s.codes = 2 * npx * code_bytes;
    s.cost = npx * Dp * eb;
    s.job_state = kJobStateBytes + sizeof(unsigned);
    s.planes = npaths * npx * Dp * eb;
    s.disp_lr = npx;
    s.sweep = sweep_supported(D, p->path_mask, (int)code_bytes) ? sweep_scratch_bytes(W, H, D, kSweepMinRows) : 0;
    s.staging_slot = 3 * npx + 2 * (size_t)D * W + 2 * (size_t)H * D;
    return s;
}

int sgm::sweep_feasible(const sgm_handle_s *h, int rows) {
    if (!h->sweep_scratch || !sweep_supported(h->D, h->p.path_mask, h->code_bytes)) return SGM_ERR_UNSUPPORTED;
    if (rows < kSweepMinRows || rows > 8) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    return sweep_fits(h->H, h->D, h->code_bytes, rows) ? SGM_OK : SGM_ERR_UNSUPPORTED;
}

extern "C" {

const char *sgm_status_string(int status) {
    switch (status) {
        case SGM_OK: return "ok";
        case SGM_ERR_INVALID_ARG: return "invalid argument";
        case SGM_ERR_UNSUPPORTED: return "unsupported parameters";
        case SGM_ERR_OOM: return "out of memory";
        case SGM_ERR_CUDA: return "CUDA error";
        case SGM_ERR_TIMEOUT: return "device wait timed out";
        case SGM_ERR_OVERRUN: return "a kernel wrote outside its buffer";
        default: return "unknown status";
    }
}

const char *sgm_stage_name(int i) { return (i >= 0 && i < kNumStages) ? kStageNames[i] : nullptr; }

int sgm_create(int W, int H, int D, const sgm_params *params, sgm_handle *out) {
    if (!out) return SGM_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(W, H, D, params);
    if (rc != SGM_OK) return rc;
    sgm_handle_s *h = (sgm_handle_s *)calloc(1, sizeof(sgm_handle_s));
    if (!h) return SGM_ERR_OOM;
    h->W = W;
    h->H = H;
    h->D = D;
    h->p = *params;
    h->wide = params->cost == SGM_COST_SAD;
    h->nbits = h->wide ? params->census_w * params->census_h * 255 : params->census_w * params->census_h - 1;
    h->code_bytes = h->wide ? 0 : (h->nbits <= 32 ? 4 : 8);
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        free(h);
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    for (int r = 0; r < kMaxPaths; r++)
        if ((params->path_mask >> r) & 1) h->path_of_plane[h->npaths++] = r;
    h->Dp = padded_disparities(D);
    h->agg_blocks_per_sm = 3;  // 12 resident warps per SM (fastest on 1242 x 375, D = 128)
    h->agg_cpl = 1;  // one 8-disparity chunk per lane: fastest for single pairs on every measured shape
    h->schedule = SGM_SCHEDULE_PLANES;
    h->sweep_rows = 4;
    const Tuning tuned = tuned_for(h);
    if (tuned.blocks_per_sm > 0) {
        h->agg_blocks_per_sm = tuned.blocks_per_sm;
        h->agg_cpl = tuned.cpl;
        h->schedule = tuned.schedule;
        h->sweep_rows = tuned.sweep_rows;
    }
    if (const char *env = getenv("SGM_AGG_BLOCKS_PER_SM")) {  // tuning override
        const int v = atoi(env);
        if (v >= 1 && v <= 16) h->agg_blocks_per_sm = v;
    }
    const ScratchSizes sz = scratch_sizes(W, H, D, params);
    h->canaries = g_canaries.load();
    rc = h->wide ? SGM_OK : dev_alloc(h, &h->codes, sz.codes);
    if (rc == SGM_OK) rc = dev_alloc(h, &h->cost, sz.cost);
    if (rc == SGM_OK) rc = dev_alloc(h, &h->job_counter, sz.job_state);
    if (rc == SGM_OK) {
        h->dev_status = h->job_counter + kJobStateBytes / sizeof(unsigned);
        if (cudaMemset(h->dev_status, 0, sizeof(unsigned)) != cudaSuccess) rc = SGM_ERR_CUDA;
    }
    if (rc == SGM_OK) rc = dev_alloc(h, &h->planes, sz.planes);
    if (rc == SGM_OK) rc = dev_alloc(h, &h->disp_lr, sz.disp_lr);
    if (rc == SGM_OK && sz.sweep) rc = dev_alloc(h, &h->sweep_scratch, sz.sweep);
    if (rc == SGM_OK && h->schedule == SGM_SCHEDULE_SWEEP && sweep_feasible(h, h->sweep_rows) != SGM_OK)
        h->schedule = SGM_SCHEDULE_PLANES;
    if (rc == SGM_OK && cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    if (rc == SGM_OK && (cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess))
        rc = SGM_ERR_CUDA;
    if (rc != SGM_OK) {
        cudaGetLastError();
        free_handle(h);
        return rc;
    }
    *out = h;
    return SGM_OK;
}

int sgm_destroy(sgm_handle h) {
    if (!h) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    batch_forget(h);
    free_handle(h);
    return SGM_OK;
}

int sgm_scratch_bytes(int W, int H, int D, const sgm_params *params, size_t *handle_bytes,
                      size_t *host_staging_bytes, size_t *static_bytes) {
    const int rc = validate(W, H, D, params);
    if (rc != SGM_OK) return rc;
    const ScratchSizes sz = scratch_sizes(W, H, D, params);
    if (handle_bytes) *handle_bytes = sz.handle();
    if (host_staging_bytes) *host_staging_bytes = 2 * sz.staging_slot;
    if (static_bytes) *static_bytes = static_scratch_bytes(sz);
    return SGM_OK;
}

int sgm_get_shape(sgm_handle h, int *W, int *H, int *D, int *census_bits) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (W) *W = h->W;
    if (H) *H = h->H;
    if (D) *D = h->D;
    if (census_bits) *census_bits = h->nbits;
    return SGM_OK;
}

int sgm_compute(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                void *stream) {
    if (!h || !left || !right || !disp) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    return compute_on(h, left, right, disp, (cudaStream_t)stream);
}

int uvmap_compute(sgm_handle h, const uint8_t *disp, uint16_t *umap, uint16_t *vmap, void *stream) {
    if (!h || !disp || !umap || !vmap) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    return uv_on(h, disp, umap, vmap, (cudaStream_t)stream);
}

namespace {

// Device buffers and events of staging slot i (first use only).
int ensure_slot(sgm_handle_s *h, int i) {
    IoSlot &sl = h->io[i];
    if (sl.left) return SGM_OK;
    const size_t npx = (size_t)h->W * h->H;
    const int keep = h->nallocs;
    int rc = dev_alloc(h, &sl.left, npx);
    if (rc == SGM_OK) rc = dev_alloc(h, &sl.right, npx);
    if (rc == SGM_OK) rc = dev_alloc(h, &sl.disp, npx);
    if (rc == SGM_OK) rc = dev_alloc(h, &sl.umap, (size_t)h->D * h->W * sizeof(uint16_t));
    if (rc == SGM_OK) rc = dev_alloc(h, &sl.vmap, (size_t)h->H * h->D * sizeof(uint16_t));
    if (rc == SGM_OK && (cudaEventCreateWithFlags(&sl.in_ready, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&sl.computed, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess))
        rc = SGM_ERR_CUDA;
    if (rc != SGM_OK) {
        dev_release_after(h, keep);
        if (sl.in_ready) cudaEventDestroy(sl.in_ready);
        if (sl.computed) cudaEventDestroy(sl.computed);
        if (sl.done) cudaEventDestroy(sl.done);
        sl = IoSlot{};
        cudaGetLastError();
    }
    return rc;
}

// The pipeline on slot sl's device inputs, into its device outputs (dense images).
int compute_slot(sgm_handle_s *h, IoSlot &sl, bool maps, cudaStream_t s) {
    const int saved_pitch = h->p.row_pitch;
    h->p.row_pitch = 0;
    int rc = compute_on(h, sl.left, sl.right, sl.disp, s);
    h->p.row_pitch = saved_pitch;
    if (rc == SGM_OK && maps) rc = uv_on(h, sl.disp, sl.umap, sl.vmap, s);
    return rc;
}

int copy_out(sgm_handle_s *h, const IoSlot &sl, uint8_t *disp, uint16_t *umap, uint16_t *vmap,
             cudaStream_t s) {
    const size_t npx = (size_t)h->W * h->H;
    if (cudaMemcpyAsync(disp, sl.disp, npx, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SGM_ERR_CUDA;
    if (umap && (cudaMemcpyAsync(umap, sl.umap, (size_t)h->D * h->W * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(vmap, sl.vmap, (size_t)h->H * h->D * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess))
        return SGM_ERR_CUDA;
    return SGM_OK;
}

}  // namespace

int sgm_compute_host(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                     uint16_t *umap, uint16_t *vmap, void *stream) {
    if (!h || !left || !right || !disp || (!umap) != (!vmap)) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    int rc = ensure_slot(h, 0);
    if (rc != SGM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    IoSlot &sl = h->io[0];
    const size_t npx = (size_t)h->W * h->H;
    // frames still in flight through sgm_compute_host_async use the slots too
    for (IoSlot &o : h->io)
        if (o.done && cudaStreamWaitEvent(s, o.done, 0) != cudaSuccess) rc = SGM_ERR_CUDA;
    if (rc == SGM_OK && (cudaMemcpyAsync(sl.left, left, npx, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                         cudaMemcpyAsync(sl.right, right, npx, cudaMemcpyHostToDevice, s) != cudaSuccess))
        rc = SGM_ERR_CUDA;
    if (rc == SGM_OK) rc = compute_slot(h, sl, umap != nullptr, s);
    if (rc == SGM_OK) rc = copy_out(h, sl, disp, umap, vmap, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == SGM_OK) rc = SGM_ERR_CUDA;
    return rc;
}

int sgm_compute_host_async(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                           uint16_t *umap, uint16_t *vmap, void *stream, unsigned long long *ticket) {
    if (!h || !left || !right || !disp || !ticket || (!umap) != (!vmap)) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    int rc = ensure_slot(h, 0);
    if (rc == SGM_OK) rc = ensure_slot(h, 1);
    if (rc == SGM_OK && !h->h2d && cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    if (rc == SGM_OK && !h->d2h && cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    if (rc != SGM_OK) {
        cudaGetLastError();
        return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long t = h->tickets;
    IoSlot &sl = h->io[t & 1];
    const size_t npx = (size_t)h->W * h->H;
    // inputs: once the slot's previous frame (t - 2) has been copied back
    if (cudaStreamWaitEvent(h->h2d, sl.done, 0) != cudaSuccess ||
        cudaMemcpyAsync(sl.left, left, npx, cudaMemcpyHostToDevice, h->h2d) != cudaSuccess ||
        cudaMemcpyAsync(sl.right, right, npx, cudaMemcpyHostToDevice, h->h2d) != cudaSuccess ||
        cudaEventRecord(sl.in_ready, h->h2d) != cudaSuccess)
        return SGM_ERR_CUDA;
    // the pipeline on the caller's stream, once the inputs are there
    if (cudaStreamWaitEvent(s, sl.in_ready, 0) != cudaSuccess) return SGM_ERR_CUDA;
    rc = compute_slot(h, sl, umap != nullptr, s);
    if (rc != SGM_OK) return rc;
    if (cudaEventRecord(sl.computed, s) != cudaSuccess) return SGM_ERR_CUDA;
    // results: back to the host on the second copy stream
    if (cudaStreamWaitEvent(h->d2h, sl.computed, 0) != cudaSuccess) return SGM_ERR_CUDA;
    rc = copy_out(h, sl, disp, umap, vmap, h->d2h);
    if (rc != SGM_OK) return rc;
    if (cudaEventRecord(sl.done, h->d2h) != cudaSuccess) return SGM_ERR_CUDA;
    *ticket = t;
    h->tickets = t + 1;
    return SGM_OK;
}

int sgm_host_wait(sgm_handle h, unsigned long long ticket) {
    if (!h || ticket >= h->tickets) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    // the slot's done event was recorded by this frame or by a later one on
    // the same copy stream; either way this frame's copies have finished
    return cudaEventSynchronize(h->io[ticket & 1].done) == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}

int sgm_debug_census(sgm_handle h, const uint8_t *left, const uint8_t *right, uint64_t *codes_left,
                     uint64_t *codes_right, void *stream) {
    if (!h || !left || !right || !codes_left || !codes_right) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_census(h, left, right, s);
    if (rc != SGM_OK) return rc;
    const size_t npx = (size_t)h->W * h->H;
    if (h->code_bytes == 8) {
        if (cudaMemcpyAsync(codes_left, h->codes, npx * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(codes_right, (uint8_t *)h->codes + npx * 8, npx * 8,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SGM_ERR_CUDA;
    } else {
        // widen 32-bit codes: zero the outputs, then copy into the low halves
        if (cudaMemsetAsync(codes_left, 0, npx * 8, s) != cudaSuccess ||
            cudaMemsetAsync(codes_right, 0, npx * 8, s) != cudaSuccess ||
            cudaMemcpy2DAsync(codes_left, 8, h->codes, 4, 4, npx, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpy2DAsync(codes_right, 8, (uint8_t *)h->codes + npx * 4, 4, 4, npx,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SGM_ERR_CUDA;
    }
    return SGM_OK;
}

// SGM_OK when kernel (SGM_COST_KERNEL_*) can compute h's matching cost.
static int check_cost_kernel(const sgm_handle_s *h, int kernel) {
    if (kernel < SGM_COST_KERNEL_AUTO || kernel > SGM_COST_KERNEL_TENSOR_CORES) return SGM_ERR_INVALID_ARG;
    if (h->wide && kernel != SGM_COST_KERNEL_AUTO) return SGM_ERR_UNSUPPORTED;
    if (kernel == SGM_COST_KERNEL_TENSOR_CORES && !cost_mma_supported(h->D)) return SGM_ERR_UNSUPPORTED;
    return SGM_OK;
}

int sgm_set_cost_kernel(sgm_handle h, int kernel) {
    if (!h) return SGM_ERR_INVALID_ARG;
    const int rc = check_cost_kernel(h, kernel);
    if (rc == SGM_OK) h->cost_kernel = kernel;
    return rc;
}

int sgm_device_status(sgm_handle h) {
    if (!h) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    unsigned v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&v, h->dev_status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess ||
        (v && cudaMemset(h->dev_status, 0, sizeof v) != cudaSuccess)) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    return v ? SGM_ERR_TIMEOUT : SGM_OK;
}

int sgm_debug_fail_alloc(int n) {
    if (n < 0) return SGM_ERR_INVALID_ARG;
    g_fail_alloc_in.store(n);
    return SGM_OK;
}

int sgm_debug_canaries(int on) {
    g_canaries.store(on ? 1 : 0);
    return SGM_OK;
}

int sgm_debug_check_canaries(sgm_handle h) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (!h->canaries) return SGM_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    std::vector<unsigned char> pad(kCanaryBytes);
    for (int i = 0; i < h->nallocs; i++) {
        const unsigned char *b = (const unsigned char *)h->allocs[i].base;
        for (const unsigned char *src : {b, b + kCanaryBytes + h->allocs[i].bytes}) {
            if (cudaMemcpy(pad.data(), src, kCanaryBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return SGM_ERR_CUDA;
            }
            for (unsigned char c : pad)
                if (c != kCanaryByte) return SGM_ERR_OVERRUN;
        }
    }
    return SGM_OK;
}

int sgm_debug_poke_canary(sgm_handle h, int i) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (!h->canaries) return SGM_ERR_UNSUPPORTED;
    if (i < 0 || i >= h->nallocs) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    unsigned char *after = (unsigned char *)h->allocs[i].base + kCanaryBytes + h->allocs[i].bytes;
    if (cudaMemset(after, (unsigned char)~kCanaryByte, 1) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    return SGM_OK;
}

int sgm_debug_cost(sgm_handle h, const uint8_t *left, const uint8_t *right, int kernel, uint16_t *C,
                   void *stream) {
    if (!h || !left || !right || !C) return SGM_ERR_INVALID_ARG;
    int rc = check_cost_kernel(h, kernel);
    if (rc != SGM_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int keep = h->cost_kernel;
    h->cost_kernel = kernel;
    rc = run_matching(h, left, right, s);
    h->cost_kernel = keep;
    if (rc == SGM_OK && launch_unpermute(h->cost, h->W, h->H, h->D, h->wide != 0, C, s) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    return rc;
}

int sgm_debug_guard_hits(unsigned long long *hits, int reset) {
    if (!hits) return SGM_ERR_INVALID_ARG;
#ifdef SGM_GUARDED
    unsigned long long total = 0;
    for (unsigned long long v : {guard_hits_census(reset != 0), guard_hits_aggregate(reset != 0),
                                 guard_hits_wta(reset != 0), guard_hits_post(reset != 0)}) {
        if (v == ~0ull) {
            cudaGetLastError();
            return SGM_ERR_CUDA;
        }
        total += v;
    }
    *hits = total;
    return SGM_OK;
#else
    (void)reset;
    *hits = 0;
    return SGM_ERR_UNSUPPORTED;
#endif
}

int sgm_debug_stalled_wait(sgm_handle h, const uint8_t *left, const uint8_t *right, void *stream) {
    if (!h || !left || !right) return SGM_ERR_INVALID_ARG;
    if (h->schedule == SGM_SCHEDULE_SWEEP) {
        // the fused sweep: row 1 waits for a pixel row 0 never publishes
        if (h->H < 2 || h->sweep_rows < 2 || !(h->p.path_mask & 0x54)) return SGM_ERR_UNSUPPORTED;
        DeviceGuard g(h->device);
        if (!g.ok) return SGM_ERR_CUDA;
        cudaStream_t s = (cudaStream_t)stream;
        int rc = run_census(h, left, right, s);
        if (rc == SGM_OK &&
            launch_sweep(h->codes, h->code_bytes, h->W, h->H, h->D, h->nbits, h->p.P1, h->p.P2, h->p.path_mask,
                         h->p.lr_tolerance, h->disp_lr, nullptr, nullptr, h->sweep_scratch, h->dev_status,
                         h->sweep_rows, s, 1) != cudaSuccess)
            rc = SGM_ERR_CUDA;
        return rc;
    }
    int rc = check_cost_kernel(h, SGM_COST_KERNEL_TENSOR_CORES);
    if (rc != SGM_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    rc = run_census(h, left, right, s);
    if (rc == SGM_OK && launch_cost_mma(h->codes, h->code_bytes, h->W, h->H, h->D, h->nbits, h->cost, h->job_counter,
                                        h->dev_status, s, 1) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    return rc;
}

int sgm_debug_path(sgm_handle h, int r, const uint8_t *left, const uint8_t *right, uint16_t *L,
                   void *stream) {
    if (!h || !left || !right || !L || r < 0 || r >= kMaxPaths) return SGM_ERR_INVALID_ARG;
    if (!((h->p.path_mask >> r) & 1)) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_matching(h, left, right, s);
    if (rc == SGM_OK) rc = run_aggregate(h, r, s);
    if (rc == SGM_OK && launch_unpermute(h->planes, h->W, h->H, h->D, h->wide != 0, L, s) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    return rc;
}

int sgm_debug_sum(sgm_handle h, const uint8_t *left, const uint8_t *right, uint16_t *S, void *stream) {
    if (!h || !left || !right || !S) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_matching(h, left, right, s);
    if (rc == SGM_OK) rc = run_aggregate(h, -1, s);
    if (rc == SGM_OK) rc = run_wta(h, nullptr, nullptr, S, s);
    return rc;
}

int sgm_debug_raw(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp_left,
                  uint8_t *disp_right, uint8_t *disp_lr, void *stream) {
    if (!h || !left || !right) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (h->schedule == SGM_SCHEDULE_SWEEP) {
        rc = run_census(h, left, right, s);
        if (rc == SGM_OK) rc = run_sweep(h, disp_left, disp_right, s);
    } else {
        rc = run_matching(h, left, right, s);
        if (rc == SGM_OK) rc = run_aggregate(h, -1, s);
        if (rc == SGM_OK) rc = run_wta(h, disp_left, disp_right, nullptr, s);
    }
    if (rc == SGM_OK && disp_lr &&
        cudaMemcpyAsync(disp_lr, h->disp_lr, (size_t)h->W * h->H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = SGM_ERR_CUDA;
    return rc;
}

int sgm_set_rectification(sgm_handle h, const uint16_t *left_x, const uint16_t *left_y,
                          const uint16_t *right_x, const uint16_t *right_y) {
    if (!h) return SGM_ERR_INVALID_ARG;
    const int set = (left_x != nullptr) + (left_y != nullptr) + (right_x != nullptr) + (right_y != nullptr);
    if (set != 0 && set != 4) return SGM_ERR_INVALID_ARG;
    h->rect = {left_x, left_y, right_x, right_y};
    batch_forget(h);  // captured graphs hold the previous census launch
    return SGM_OK;
}

int sgm_set_schedule(sgm_handle h, int schedule, int rows_per_cta) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (schedule == SGM_SCHEDULE_AUTO) {
        const Tuning t = tuned_for(h);
        schedule = t.blocks_per_sm > 0 ? t.schedule : SGM_SCHEDULE_PLANES;
        rows_per_cta = t.blocks_per_sm > 0 ? t.sweep_rows : h->sweep_rows;
        if (schedule == SGM_SCHEDULE_SWEEP && sweep_feasible(h, rows_per_cta) != SGM_OK) schedule = SGM_SCHEDULE_PLANES;
    } else if (schedule == SGM_SCHEDULE_SWEEP) {
        const int rc = sweep_feasible(h, rows_per_cta);
        if (rc != SGM_OK) return rc;
    } else if (schedule != SGM_SCHEDULE_PLANES) {
        return SGM_ERR_INVALID_ARG;
    }
    h->schedule = schedule;
    if (schedule == SGM_SCHEDULE_SWEEP) h->sweep_rows = rows_per_cta;
    batch_forget(h);  // captured graphs hold the previous schedule's launches
    return SGM_OK;
}

int sgm_set_aggregation(sgm_handle h, int blocks_per_sm, int chunks_per_lane) {
    if (!h || blocks_per_sm < 1 || blocks_per_sm > 16) return SGM_ERR_INVALID_ARG;
    if (chunks_per_lane != 1 && chunks_per_lane != 2 && chunks_per_lane != 4 && chunks_per_lane != kMixedCpl)
        return SGM_ERR_INVALID_ARG;
    if ((chunks_per_lane == kMixedCpl ? 2 : chunks_per_lane) > chunks_per_lane_max(h->D, h->wide != 0))
        return SGM_ERR_UNSUPPORTED;
    h->agg_blocks_per_sm = blocks_per_sm;
    h->agg_cpl = chunks_per_lane;
    batch_forget(h);  // captured graphs hold the previous launch shape
    return SGM_OK;
}

int sgm_get_aggregation(sgm_handle h, int *blocks_per_sm, int *chunks_per_lane) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (blocks_per_sm) *blocks_per_sm = h->agg_blocks_per_sm;
    if (chunks_per_lane) *chunks_per_lane = h->agg_cpl;
    return SGM_OK;
}

int sgm_get_schedule(sgm_handle h, int *schedule, int *rows_per_cta) {
    if (!h) return SGM_ERR_INVALID_ARG;
    if (schedule) *schedule = h->schedule;
    if (rows_per_cta) *rows_per_cta = h->sweep_rows;
    return SGM_OK;
}

int sgm_set_timing(sgm_handle h, int enable) {
    if (!h) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (enable && !h->recs) {
        TimingRecord *recs = (TimingRecord *)calloc(kTimingRing, sizeof(TimingRecord));
        if (!recs) return SGM_ERR_OOM;
        for (int i = 0; i < kTimingRing; i++) {
            if (cudaEventCreate(&recs[i].start) != cudaSuccess ||
                cudaEventCreate(&recs[i].stop) != cudaSuccess) {
                for (int j = 0; j <= i; j++) {
                    if (recs[j].start) cudaEventDestroy(recs[j].start);
                    if (recs[j].stop) cudaEventDestroy(recs[j].stop);
                }
                free(recs);
                cudaGetLastError();
                return SGM_ERR_CUDA;
            }
        }
        h->recs = recs;
        h->rec_head = h->rec_count = 0;
    }
    h->timing = enable ? 1 : 0;
    return SGM_OK;
}

int sgm_get_stage_times(sgm_handle h, float *ms, int *count, int n, int *n_stages) {
    if (!h || n < 0) return SGM_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    while (h->rec_count > 0) {
        harvest(h, h->recs[h->rec_head]);
        h->rec_head = (h->rec_head + 1) % kTimingRing;
        h->rec_count--;
    }
    for (int i = 0; i < n && i < kNumStages; i++) {
        if (ms) ms[i] = (float)h->acc_ms[i];
        if (count) count[i] = h->acc_n[i];
    }
    for (int i = 0; i < kNumStages; i++) {
        h->acc_ms[i] = 0;
        h->acc_n[i] = 0;
    }
    if (n_stages) *n_stages = kNumStages;
    return SGM_OK;
}

}  // extern "C"
