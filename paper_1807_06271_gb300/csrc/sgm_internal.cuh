// Internal declarations of libsgm: handle layout and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgm.h"

namespace sgm {

constexpr int kMaxPaths = 8;
constexpr int kMaxD = 255;
constexpr int kMaxW = 8192;  // the right-WTA keeps one 32-bit key per column in shared memory

// Path directions (dx, dy), bit r of a path mask enables entry r.
__host__ __device__ constexpr int dir_dx(int r) {
    return r == 0 ? 1 : r == 1 ? -1 : r == 2 ? 0 : r == 3 ? 0 : r == 4 ? 1 : r == 5 ? -1 : r == 6 ? -1 : 1;
}
__host__ __device__ constexpr int dir_dy(int r) {
    return r == 0 ? 0 : r == 1 ? 0 : r == 2 ? 1 : r == 3 ? -1 : r == 4 ? 1 : r == 5 ? -1 : r == 6 ? 1 : -1;
}

// Number of scanlines of direction r in a W x H image.
inline long scanlines_of(int r, int W, int H) {
    int dx = dir_dx(r), dy = dir_dy(r);
    if (dy == 0) return H;
    if (dx == 0) return W;
    return (long)W + H - 1;
}

// Flattened list of scanlines over the enabled paths: warp g of the
// aggregation launch works on scanline g - begin[k] of path entry k.
struct PathJobs {
    int n;                    // number of path entries
    int dx[kMaxPaths], dy[kMaxPaths];
    int plane[kMaxPaths];     // output plane of entry k
    int begin[kMaxPaths + 1]; // prefix sums of scanline counts
};

enum Stage { kStageCensus = 0, kStageAggregate, kStageWta, kStageMedian, kStageUv, kNumStages };

struct TimingRecord {
    int stage;
    cudaEvent_t start, stop;
};

}  // namespace sgm

struct sgm_handle_s {
    int W, H, D;
    sgm_params p;
    int nbits;       // census bits
    int code_bytes;  // 4 (nbits <= 32) or 8
    int device;
    int npaths;
    int path_of_plane[sgm::kMaxPaths];

    // scratch, owned
    void *codes;        // [2][H][W] census codes (left, right)
    uint8_t *planes;    // [npaths][H][W][D] per-path aggregated costs
    uint8_t *disp_lr;   // [H][W] after the LR check, before the median

    // device staging for sgm_compute_host, allocated on first use
    uint8_t *io_left, *io_right, *io_disp;
    uint16_t *io_umap, *io_vmap;

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

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_census(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int cw, int ch, int code_bytes, void *codes, cudaStream_t s);
cudaError_t launch_aggregate(const void *codes, int code_bytes, int W, int H, int D, int nbits,
                             int P1, int P2, const PathJobs &jobs, uint8_t *planes,
                             size_t plane_elems, cudaStream_t s);
cudaError_t launch_wta(const uint8_t *planes, int nplanes, size_t plane_elems, int W, int H, int D,
                       int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                       uint16_t *dbg_sum, cudaStream_t s);
cudaError_t launch_median(const uint8_t *in, uint8_t *out, int W, int H, int k, cudaStream_t s);
// Host-side argument checks shared by every entry point (SGM_OK or an error status).
int validate_params(int W, int H, int D, const sgm_params *p);

cudaError_t launch_uvmap(const uint8_t *disp, int W, int H, int D, uint16_t *umap, uint16_t *vmap,
                         cudaStream_t s);

}  // namespace sgm
