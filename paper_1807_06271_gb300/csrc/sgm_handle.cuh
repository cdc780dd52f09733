// The handle of the C ABI and the host-side pieces shared by the entry points
// (sgm_api.cu, batch.cu, and the map post-processing entry point in
// uvpost.cu).  Kernel-only sources include sgm_internal.cuh alone.
#pragma once

#include "sgm_internal.cuh"

namespace sgm {

// Device staging of one frame for the host-pointer entry points.  done is
// recorded after the frame's results have been copied back; in_ready after its
// inputs have arrived; computed after its pipeline has run.
struct IoSlot {
    uint8_t *left, *right, *disp;
    uint16_t *umap, *vmap;
    cudaEvent_t in_ready, computed, done;
};

enum Stage { kStageCensus = 0, kStageCost, kStageAggregate, kStageWta, kStageMedian, kStageUv, kStageSweep, kNumStages };

struct TimingRecord {
    int stage;
    cudaEvent_t start, stop;
};

// One device allocation of a handle.  With canaries on, kCanaryBytes of
// kCanaryByte sit before and after the bytes the handle uses (base is the
// cudaMalloc pointer; the handle's pointer is base + kCanaryBytes).
struct DevAlloc {
    void *base;
    size_t bytes;
};
constexpr int kMaxAllocs = 16;
constexpr size_t kCanaryBytes = 256;  // keeps the buffers 256-byte aligned
constexpr unsigned char kCanaryByte = 0xA5;

}  // namespace sgm

struct sgm_handle_s {
    int W, H, D;
    sgm_params p;
    int nbits;       // largest matching cost: census bits, or window * 255 for SAD
    int code_bytes;  // census: 4 (nbits <= 32) or 8; SAD: 0 (no codes)
    int wide;        // 1: 16-bit costs and path costs (SAD), 0: 8-bit (census)
    int device;
    int npaths;
    int path_of_plane[sgm::kMaxPaths];

    int Dp;          // padded disparities per pixel (8 * lanes per scanline)

    // every device allocation of the handle (scratch and staging), freed by sgm_destroy
    sgm::DevAlloc allocs[sgm::kMaxAllocs];
    int nallocs;
    int canaries;  // allocations carry guard bytes on both sides (sgm_debug_canaries)

    // scratch, owned
    void *codes;        // [2][H][W] census codes (left, right); null for SAD
    uint8_t *cost;      // [H][W][Dp] matching cost, lane-chunk order (bytes, or uint16 when wide)
    uint8_t *planes;    // [H][W][npaths][Dp] per-path aggregated costs, same order
    uint8_t *disp_lr;   // [H][W] after the LR check, before the median
    unsigned *job_counter;  // work-queue state of the aggregation kernel (kJobStateBytes), then dev_status
    unsigned *dev_status;   // bit 0: a bounded device wait gave up (one word after the work-queue state)
    int cost_kernel;        // SGM_COST_KERNEL_* of the census cost
    int agg_blocks_per_sm;  // resident 4-warp blocks per SM of the aggregation kernel
    int agg_cpl;            // 8-disparity chunks per lane of the aggregation kernel (1, 2 or 4)
    int schedule;           // SGM_SCHEDULE_PLANES or SGM_SCHEDULE_SWEEP (resolved, never AUTO)
    int sweep_rows;         // rows (warps) per CTA of the fused sweep
    void *sweep_scratch;    // global rings, counters and right map of the fused sweep (null when unsupported)
    sgm::RectMaps rect;     // caller-owned rectification maps, or all null

    // device staging of the host-pointer entry points, allocated on first use:
    // slot 0 for sgm_compute_host, both slots in turn for sgm_compute_host_async
    sgm::IoSlot io[2];
    cudaStream_t h2d, d2h;       // copy streams of sgm_compute_host_async
    unsigned long long tickets;  // frames submitted through sgm_compute_host_async

    // internal stream for sgm_batch_compute
    cudaStream_t side;
    cudaEvent_t fork_ev, join_ev;

    // stage timing
    int timing;
    int rec_head, rec_count;
    sgm::TimingRecord *recs;
    double acc_ms[sgm::kNumStages];
    int acc_n[sgm::kNumStages];
};

namespace sgm {

// Bytes of each device buffer of one pair.  sgm_create allocates each as its
// own buffer, sgm_compute_static packs them into its fixed array, and
// sgm_scratch_bytes reports them, all from this one computation.
struct ScratchSizes {
    size_t codes;         // census codes of both images (0 for SAD)
    size_t cost;          // cost volume
    size_t job_state;     // aggregation work-queue state plus the device status word
    size_t planes;        // one plane per enabled path
    size_t disp_lr;       // map after the LR check
    size_t sweep;         // fused streaming sweep (0 when the path set or D rules it out)
    size_t staging_slot;  // one host-path staging slot: left, right, disp, U, V
    size_t handle() const { return codes + cost + job_state + planes + disp_lr + sweep; }
};
// Call only with parameters that passed validate_params.
ScratchSizes scratch_sizes(int W, int H, int D, const sgm_params *p);

// Where sgm_compute_static places each buffer in its fixed array: codes,
// cost volume, planes, work-queue state and LR map in turn, each at a
// 256-byte boundary; end is the number of bytes used.
struct StaticLayout {
    size_t codes, cost, planes, job_state, disp_lr, end;
};
StaticLayout static_layout(const ScratchSizes &sz);
inline size_t static_scratch_bytes(const ScratchSizes &sz) { return static_layout(sz).end; }

// One pair (and its U/V maps when umap and vmap are non-null) on stream s.
int compute_pair(sgm_handle_s *h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                 uint16_t *umap, uint16_t *vmap, cudaStream_t s);
// Drops cached batch graphs that use h (called before h is freed).
void batch_forget(sgm_handle_s *h);
// What sgm_autotune chose for h's shape: aggregation blocks per SM (0: not
// tuned) and chunks per lane, and the schedule with its rows per CTA.
struct Tuning {
    int blocks_per_sm, schedule, sweep_rows, cpl;
};
Tuning tuned_for(const sgm_handle_s *h);
// Rows per CTA the fused sweep's scratch is sized for (the smallest it runs with).
constexpr int kSweepMinRows = 2;
// SGM_OK when h can run the fused sweep with `rows` rows per CTA on its device.
int sweep_feasible(const sgm_handle_s *h, int rows);

}  // namespace sgm
