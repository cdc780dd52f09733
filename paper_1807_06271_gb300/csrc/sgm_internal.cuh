// Internal declarations of libsgm: handle layout and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgm.h"

namespace sgm {

constexpr int kMaxPaths = 8;
constexpr int kMaxD = 255;
constexpr int kMaxW = 8192;  // the right-WTA keeps one 32-bit key per column in shared memory
constexpr int kMaxSadWindow = 15;  // largest SAD support window side (shared-memory rows of the cost kernel)

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

// Rectification maps of the left and right image (device, W x H each; all
// null when the images are already rectified).
// Programmatic dependent launch.  Every kernel of the pipeline is launched
// with programmatic stream serialisation, so the launch of kernel k+1 overlaps
// the end of kernel k; each kernel's first statement waits until its stream
// predecessor has completed and its memory is visible, before it reads or
// writes anything.  Kernels launched the ordinary way pass the wait at once.
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

struct RectMaps {
    const uint16_t *lx, *ly, *rx, *ry;
};

// Pixel (gx, gy) of the rectified image: the source image read through the
// maps (Sec. 3.1.1), 0 where a map entry leaves the source.
// Guarded builds (compiled with -DSGM_GUARDED: a test variant of the
// library, never the default).  The plane path's kernels (census, the
// CUDA-core cost, the aggregation, the WTA, the median and the U/V maps)
// check each global index they compute, and each shared index that depends
// on the image, against its buffer's extent before the access.  An index out
// of range skips the access and is counted in the translation unit's
// counter; sgm_debug_guard_hits sums the counters.  In the default build
// in_range is constant true and the checks compile away.
#ifdef SGM_GUARDED
static __device__ unsigned long long g_guard_hits;  // one per translation unit
__device__ __forceinline__ bool in_range(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_guard_hits, 1ull);
    return false;
}
#define SGM_GUARD_COUNTER(name)                                                   \
    unsigned long long name(bool reset) {                                         \
        unsigned long long v = 0, z = 0;                                          \
        if (cudaMemcpyFromSymbol(&v, g_guard_hits, sizeof(v)) != cudaSuccess)     \
            v = ~0ull;                                                            \
        if (reset && cudaMemcpyToSymbol(g_guard_hits, &z, sizeof(z)) != cudaSuccess) \
            v = ~0ull;                                                            \
        return v;                                                                 \
    }
#else
__device__ __forceinline__ constexpr bool in_range(long long, long long) { return true; }
#define SGM_GUARD_COUNTER(name) \
    unsigned long long name(bool) { return 0; }
#endif
// Each guarded translation unit's counter (~0 when it cannot be read).
unsigned long long guard_hits_census(bool reset);
unsigned long long guard_hits_aggregate(bool reset);
unsigned long long guard_hits_wta(bool reset);
unsigned long long guard_hits_post(bool reset);

template <bool RECT>
__device__ __forceinline__ uint8_t rect_pixel(const uint8_t *__restrict__ img, int pitch, int W,
                                              int H, int gx, int gy, const uint16_t *__restrict__ mx,
                                              const uint16_t *__restrict__ my) {
    if constexpr (!RECT) {
        const long long i = (long long)gy * pitch + gx;
        return in_range(i, (long long)pitch * H) ? img[i] : 0;
    } else {
        const long long m = (long long)gy * W + gx;
        if (!in_range(m, (long long)W * H)) return 0;
        const int sx = mx[m], sy = my[m];
        return (sx < W && sy < H) ? img[(size_t)sy * pitch + sx] : 0;
    }
}

// Disparity layout.  The D disparities of a pixel are held by LPS lanes
// ("lanes per scanline", a power of two) with DPL = 8 disparities each, so a
// pixel owns Dp = DPL * LPS slots in the cost volume and in every path plane;
// slots d >= D are padding.  A lane's chunk (disparities DPL*i .. DPL*i + DPL-1)
// is stored so that the aggregation kernel gets the packed 16-bit pairs
// (d+k, d+k+h), h = DPL/2, it works on with at most one mask or byte-permute:
//   8-bit costs (census): DPL/4 32-bit words, word w holding the bytes
//     d+2w  d+2w+1  d+2w+h  d+2w+1+h  (mask 0x00FF00FF, or permute, per pair);
//   16-bit costs (SAD, "wide"): DPL/2 32-bit words, word k holding the
//     uint16 pair (d+k, d+k+h) itself.
// The kernels are written for any DPL that is a multiple of 4; 16 per lane was
// measured slower on the 1242 x 375, D = 128 workload (fewer, fatter warps
// lengthen the horizontal scanlines, which set the aggregation's duration), so
// 8 is used for every D.
inline int disparities_per_lane(int) { return 8; }
inline int lanes_per_scanline(int D) {
    const int dpl = disparities_per_lane(D);
    int need = (D + dpl - 1) / dpl, l = 1;
    while (l < need) l *= 2;
    return l;
}
inline int padded_disparities(int D) { return disparities_per_lane(D) * lanes_per_scanline(D); }
__host__ __device__ constexpr int chunk_byte(int dpl, int j) {  // byte of disparity dpl*i + j
    return j < dpl / 2 ? 4 * (j / 2) + (j % 2) : 4 * ((j - dpl / 2) / 2) + 2 + ((j - dpl / 2) % 2);
}

// Work list of the aggregation kernel: entry k is one enabled direction whose
// nlines scanlines are cut into jobs of G = 32 / LPS neighbouring scanlines
// (one warp each).  Job j belongs to entry k when jbegin[k] <= j < jbegin[k+1].
struct PathJobs {
    int n;                     // number of entries
    int dx[kMaxPaths], dy[kMaxPaths];
    int plane[kMaxPaths];      // output plane of entry k
    int nlines[kMaxPaths];
    int cpl[kMaxPaths];        // 8-disparity chunks per lane of entry k's jobs
    int jbegin[kMaxPaths + 1];
    int nlong;                 // jobs [0, nlong) belong to the long-axis directions
    uint32_t unit;             // always 1; see the kernel's multiply-adds
};

// Work-queue state of the aggregation kernel (cleared before every launch):
// word 0 hands out the long-axis jobs, word 1 the others, and words
// kJobClaimBase + slot are claim flags, one per (SM, warp scheduler).
constexpr int kJobClaimBase = 32, kJobClaimSlots = 1024;
constexpr size_t kJobStateBytes = (size_t)(kJobClaimBase + kJobClaimSlots) * sizeof(unsigned);

// Builds the work list for the directions in `mask` (planes numbered in
// increasing direction order), longest scanlines first, for lanes holding
// `cpl` 8-disparity chunks each: G = 32 / (lanes_per_scanline(D) / cpl).
PathJobs make_path_jobs(int W, int H, int D, int mask, int cpl);
// The same with the long-axis directions (rows when W >= H) at cpl_long chunks
// per lane and the others at cpl_other.
PathJobs make_path_jobs_mixed(int W, int H, int D, int mask, int cpl_long, int cpl_other);
// The most chunks per lane the aggregation takes for D (1 for 16-bit costs, up to 4).
int chunks_per_lane_max(int D, bool wide);
// Chunks-per-lane code of the mixed layout: long-axis scanlines at 1, the others at 2.
constexpr int kMixedCpl = SGM_AGG_CHUNKS_MIXED;

// One pair of a batched aggregation launch (device-resident table entry).
struct BatchAggPair {
    const void *cost;  // the pair's cost volume
    void *planes;      // its path planes
    int W, H, D;
    int lps;           // lanes per scanline: the pixel's chunks / chunks per lane
    int ragged;        // D < 8 * lps
    int nplanes;
    PathJobs jobs;
};

}  // namespace sgm

namespace sgm {

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_census(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int cw, int ch, int code_bytes, void *codes, const RectMaps &maps,
                          cudaStream_t s);
// The cost kernels also clear job_state (kJobStateBytes, may be null), the
// work-queue state of the aggregation kernel that follows them on the stream.
// Hamming costs of the census codes come from one of two kernels (kernel:
// SGM_COST_KERNEL_*): POPC on the CUDA cores (any D) or +-1 inner products on
// the tensor cores (Dp <= 128), which ORs 1 into *status (may be null) when its
// bounded wait for the MMA gives up.
cudaError_t launch_cost(const void *codes, int code_bytes, int W, int H, int D, int nbits,
                        uint8_t *cost, unsigned *job_state, unsigned *status, int kernel, cudaStream_t s);
bool cost_mma_supported(int D);
// stall_test != 0: the kernel's first wait is on an mbarrier nothing arrives at,
// with a 2 ms limit, so that it takes its timeout path (for tests of it).
cudaError_t launch_cost_mma(const void *codes, int code_bytes, int W, int H, int D, int nbits, uint8_t *cost,
                            unsigned *job_state, unsigned *status, cudaStream_t s, int stall_test = 0);
// The kernel SGM_COST_KERNEL_AUTO selects for D.
int cost_kernel_for(int D);
// SAD over a ww x wh window (clamped reads; rectified through maps when set) into a
// 16-bit cost volume [H][W][Dp] in the wide lane-chunk order.
cudaError_t launch_sad_cost(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                            int D, int ww, int wh, const RectMaps &maps, uint16_t *cost,
                            unsigned *job_state, cudaStream_t s);
// Planes are pixel-interleaved: [H][W][nplanes][Dp], entry k of `jobs` writing
// plane jobs.plane[k].  job_counter (kJobStateBytes) must have been cleared by
// the cost kernel launched before it on s.
// wide: 16-bit costs and planes (SAD), else 8-bit.  cpl: 8-disparity chunks
// per lane (1, 2 or 4, at most chunks_per_lane_max; jobs built with the same).
cudaError_t launch_aggregate(const uint8_t *cost, int W, int H, int D, int P1, int P2, bool wide,
                             const PathJobs &jobs, uint8_t *planes, int nplanes,
                             unsigned *job_counter, int blocks_per_sm, int cpl, cudaStream_t s);
// All pairs' aggregation in one persistent launch (pairs: device table of
// npairs entries; prefix: device [2][npairs + 1], the running counts of the
// pairs' long-axis jobs and of their other jobs).  job_counter as above, for
// this launch alone.  P1/P2 and the cost width are shared by the pairs.
// cpl: 1 or 4 (4 only for 8-bit costs and pairs whose D allows it).
cudaError_t launch_aggregate_batch(const BatchAggPair *pairs, int npairs, const int *prefix, int P1, int P2,
                                   bool wide, int cpl, unsigned *job_counter, int blocks_per_sm, cudaStream_t s);
// Copies a single plane ([H][W][Dp], lane-chunk order) to L ([H][W][D] uint16, natural order).
cudaError_t launch_unpermute(const uint8_t *plane, int W, int H, int D, bool wide, uint16_t *L,
                             cudaStream_t s);
cudaError_t launch_wta(const uint8_t *planes, int nplanes, int W, int H, int D, bool wide,
                       int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                       uint16_t *dbg_sum, cudaStream_t s);
cudaError_t launch_median(const uint8_t *in, uint8_t *out, int W, int H, int k, cudaStream_t s);
// Host-side argument checks shared by every entry point (SGM_OK or an error status).
int validate_params(int W, int H, int D, const sgm_params *p);

cudaError_t launch_uvmap(const uint8_t *disp, int W, int H, int D, uint16_t *umap, uint16_t *vmap,
                         cudaStream_t s);

// The paper's streaming set in one top-down sweep with the cost, the paths,
// both winners and the LR check fused (sweep.cu): census codes (code_bytes 4
// or 8) of both images in, the checked map disp_lr out (dbg_left/dbg_right,
// optional, receive the raw maps).  Supported for D <= 128 and path masks
// within 0x55.  scratch: sweep_scratch_bytes(W, H, D, rows_per_cta) bytes.
// A bounded wait that gives up ORs 2 into *status (may be null).
// Returns cudaErrorCooperativeLaunchTooLarge when the grid cannot be resident at once.
bool sweep_supported(int D, int mask, int code_bytes);
bool sweep_fits(int H, int D, int code_bytes, int rows_per_cta);
size_t sweep_scratch_bytes(int W, int H, int D, int rows_per_cta);
// stall_test != 0: row 1 waits for a pixel row 0 never publishes, with a 2 ms
// limit, so that the bounded waits take their timeout path (for tests of it).
cudaError_t launch_sweep(const void *codes, int code_bytes, int W, int H, int D, int nbits, int P1, int P2,
                         int mask, int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                         void *scratch, unsigned *status, int rows_per_cta, cudaStream_t s, int stall_test = 0);

}  // namespace sgm
