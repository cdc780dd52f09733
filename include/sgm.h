/*
 * libsgm — semi-global-matching stereo and U-/V-disparity maps on GB300 (sm_103a).
 *
 * Method: Ruf, Monka, Kollmann, Grinberg, "Real-time on-board obstacle
 * avoidance for UAVs based on embedded stereo vision" (ISPRS TC I, 2018),
 * Sec. 3.1 (disparity estimation) and Sec. 3.2 (U-/V-maps).
 *
 * Conventions shared by every entry point
 *   - Images are 8-bit grey, rectified, row-major.  A left/right image row is
 *     `row_pitch` bytes apart (sgm_params; 0 means W).  Every other array is
 *     dense row-major with no padding.
 *   - Disparities are 8-bit; 0xFF (SGM_INVALID) marks a pixel removed by the
 *     left-right check.  d runs over [0, D).
 *   - "device" pointers are CUDA global-memory pointers on the handle's device
 *     (for example torch tensor data pointers); "host" pointers are ordinary
 *     (preferably pinned) CPU memory.  The caller owns every pointer it passes;
 *     the handle owns its scratch memory and keeps it between calls.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device-pointer calls are asynchronous: results are valid once the stream
 *     has been synchronised.  Calls on one handle must not overlap in time on
 *     different streams (they share the handle's scratch).
 *   - Every call returns an SGM_* status; nothing throws across the ABI.
 *     Arguments are validated on the host before any work is queued.
 */
#ifndef SGM_H
#define SGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SGM_OK 0
#define SGM_ERR_INVALID_ARG 1 /* null/inconsistent argument                       */
#define SGM_ERR_UNSUPPORTED 2 /* valid but outside what the kernels implement     */
#define SGM_ERR_OOM 3         /* device or pinned-host allocation failed          */
#define SGM_ERR_CUDA 4        /* a CUDA runtime call or kernel launch failed      */
#define SGM_ERR_TIMEOUT 5     /* a bounded device-side wait gave up               */
#define SGM_ERR_OVERRUN 6     /* a guard byte next to a buffer changed (canaries) */

#define SGM_INVALID 0xFF

/* Path sets (bit r enables direction r).  Directions, as (dx, dy) steps from a
 * pixel's predecessor to the pixel:
 *   0 (1,0) left->right      1 (-1,0) right->left
 *   2 (0,1) top->bottom      3 (0,-1) bottom->top
 *   4 (1,1) TL->BR           5 (-1,-1) BR->TL
 *   6 (-1,1) TR->BL          7 (1,-1) BL->TR                                    */
#define SGM_PATHS_4 0x0F       /* horizontal and vertical, both ways                 */
#define SGM_PATHS_8 0xFF       /* all eight (Sec. 3.1.3, Fig. 3a)                    */
#define SGM_PATHS_STREAM4 0x55 /* 0, 45, 90, 135 degrees: the paper's streaming set
                                  (Sec. 3.1.3, Fig. 2 and Fig. 3b)                   */

/* Matching costs (Sec. 3.1.2).  Both use the census_w x census_h window of
 * sgm_params as their support region (5x5 in Sec. 4.1). */
#define SGM_COST_CENSUS 0 /* Hamming distance of census codes: bit 1 iff the
                             neighbour is darker than the centre, raster order,
                             centre skipped, neighbours outside the image 0     */
#define SGM_COST_SAD 1    /* sum of absolute differences over the window, both
                             images read with clamped (replicated) coordinates;
                             the paper pairs it with P1 = 200, P2 = 800         */

/* Kernels for the Hamming costs of SGM_COST_CENSUS (Eq. 1); both give the
 * same cost volume bit for bit.  With the census bits as entries +1 (bit
 * clear) and -1 (bit set), the inner product of two codes is
 * nbits - 2 * Hamming distance, so a row segment's costs are a band of a
 * matrix product of the left and right codes. */
#define SGM_COST_KERNEL_AUTO 0         /* the faster one on GB300: CUDA cores            */
#define SGM_COST_KERNEL_CUDA_CORES 1   /* POPC of the XOR of the two codes, any D        */
#define SGM_COST_KERNEL_TENSOR_CORES 2 /* the band on tcgen05 (e4m3 +-1 entries, f32
                                          sums in tensor memory); 17 <= D <= 128    */

typedef struct sgm_handle_s *sgm_handle;

typedef struct sgm_params {
    int census_w, census_h; /* support window of the matching cost, both odd
                               (Sec. 3.1.2; 5x5 in Sec. 4.1).  Census:
                               census_w*census_h-1 <= 64 bits                   */
    int path_mask;          /* SGM_PATHS_* or any non-empty subset of 0xFF          */
    int P1, P2;             /* penalties of Eq. 2, 0 <= P1 <= P2.  Census:
                               bits + P2 <= 255 (8-bit path costs).  SAD
                               (window sides <= 15): with cmax =
                               census_w*census_h*255, cmax + P2 <= 32766 and
                               (cmax + P2) * (number of paths) <= 65535
                               (16-bit path costs whose sum fits 16 bits)     */
    int lr_tolerance;       /* Sec. 3.1.4; < 0 switches the check off                */
    int median_k;           /* Sec. 3.1.5; 0 or 1 = off, else odd, <= 7             */
    int row_pitch;          /* bytes between image rows; 0 = W                       */
    int cost;               /* SGM_COST_CENSUS (0, the default) or SGM_COST_SAD      */
} sgm_params;

/* Create a handle for W x H images and D disparities (1 <= D <= 255) and
 * allocate all scratch memory on the current CUDA device.  Out of memory ->
 * SGM_ERR_OOM; unsupported parameters -> SGM_ERR_UNSUPPORTED; *out stays NULL
 * on failure.  The handle is bound to the device current at creation. */
int sgm_create(int W, int H, int D, const sgm_params *params, sgm_handle *out);

/* Free the handle and its scratch (synchronises the device first). */
int sgm_destroy(sgm_handle h);

/* Dense disparity of one rectified pair (Sec. 3.1): census transform and
 * Hamming cost, or SAD (Sec. 3.1.2, Eq. 1), aggregation along the enabled paths with
 * P1/P2 (Sec. 3.1.3, Eq. 2), winner-takes-all, right disparity from the same
 * aggregated volume and left-right check (Sec. 3.1.4), k x k median
 * (Sec. 3.1.5).  left/right: device, H rows of row_pitch bytes.  disp: device,
 * H x W bytes, SGM_INVALID where the LR check failed. */
int sgm_compute(sgm_handle h, const uint8_t *left, const uint8_t *right,
                uint8_t *disp, void *stream);

/* U-map and V-map of a disparity map (Sec. 3.2): umap[d*W + x] counts the
 * pixels of column x with disparity d (D x W); vmap[y*D + d] counts the pixels
 * of row y with disparity d (H x D).  SGM_INVALID pixels are not counted.
 * disp, umap, vmap: device.  Every output element is written. */
int uvmap_compute(sgm_handle h, const uint8_t *disp, uint16_t *umap,
                  uint16_t *vmap, void *stream);

/* Post-processing of the maps before obstacle extraction (Sec. 3.2; the
 * paper names the steps but not their parameters):
 *   binary(i,j) = map(i,j) >= threshold inside the region of interest
 *                 [roi[0], roi[1]) x [roi[2], roi[3]) (rows x columns of the
 *                 map), 0 outside it;
 *   dilated     = max of binary over a (2 dilate_r + 1)^2 square;
 *   out         = 3x3 binomial Gaussian [1 2 1; 2 4 2; 1 2 1]/16 of
 *                 255 * dilated, (sum + 8) / 16;
 * cells outside the map count as 0.  The U-map is D x W (rows d, columns x),
 * the V-map H x D (rows y, columns d). */
typedef struct sgm_uv_post {
    int u_threshold, v_threshold;
    int u_roi[4]; /* d0, d1, x0, x1 */
    int v_roi[4]; /* y0, y1, d0, d1 */
    int dilate_r; /* 0..7 */
} sgm_uv_post;

/* umap/vmap: device maps from uvmap_compute; uout (D x W) and vout (H x D):
 * device uint8 outputs, either may be NULL to skip that map. */
int uvmap_postprocess(sgm_handle h, const uint16_t *umap, const uint16_t *vmap,
                      const sgm_uv_post *params, uint8_t *uout, uint8_t *vout, void *stream);

/* sgm_compute followed by uvmap_compute with HOST buffers: copies left/right
 * (H x W each, dense) to handle-owned device buffers, runs both, copies disp
 * (H x W) and, when non-NULL, umap (D x W) and vmap (H x D) back, and waits
 * for the stream.  Pinned host memory makes the copies asynchronous. */
int sgm_compute_host(sgm_handle h, const uint8_t *left, const uint8_t *right,
                     uint8_t *disp, uint16_t *umap, uint16_t *vmap, void *stream);

/* Pipelined form of sgm_compute_host for a stream of frames (the paper's
 * camera loop, Sec. 3): queues the copy of left/right (host, H x W each,
 * dense) into one of two handle-owned device slots on an internal copy
 * stream, the pipeline on `stream` once they have arrived, and the copy of
 * disp (and of umap/vmap when non-NULL, as in sgm_compute_host) back to the
 * host on a second internal copy stream; returns without waiting and stores
 * the frame's number in *ticket.  Frame t+1's upload and frame t-1's download
 * overlap frame t's pipeline.  Until sgm_host_wait(h, *ticket) returns, the
 * frame's left/right must stay unchanged and disp/umap/vmap must not be read.
 * Use pinned host memory (pageable memory makes the copies synchronous).
 * Calls on one handle must use one `stream`. */
int sgm_compute_host_async(sgm_handle h, const uint8_t *left, const uint8_t *right,
                           uint8_t *disp, uint16_t *umap, uint16_t *vmap, void *stream,
                           unsigned long long *ticket);

/* Wait until frame `ticket` of sgm_compute_host_async has been copied back
 * (its inputs are then free as well).  A ticket not yet issued is
 * SGM_ERR_INVALID_ARG. */
int sgm_host_wait(sgm_handle h, unsigned long long ticket);

/* Many pairs in one go (the method of Sec. 3.1 per pair): n handles (each
 * with its own size and parameters), device pointers left[i], right[i],
 * disp[i] and optional umap[i]/vmap[i] (umap/vmap NULL, or NULL entries, skip
 * the maps of a pair).  Every pair's pipeline runs on its own branch of one
 * CUDA graph, forked from and joined back to `stream`; the graph is captured
 * on the first call and replayed while the same handles and buffers (and
 * tuning) come back, up to 8 distinct batches per process (least recently
 * used dropped first).  Destroying a handle drops the graphs that use it.
 * With stage timing enabled on any handle the pairs are launched directly on
 * forked streams instead.  Handles must be distinct. */
int sgm_batch_compute(int n, const sgm_handle *hs, const uint8_t *const *left,
                      const uint8_t *const *right, uint8_t *const *disp,
                      uint16_t *const *umap, uint16_t *const *vmap, void *stream);

/* ---- batch engine ----------------------------------------------------------
 * Many pairs of uneven size and disparity range, each the method of Sec. 3.1
 * with the same sgm_params, from one pooled device allocation.  A run is one
 * CUDA graph: each pair's census and matching cost on a branch of its own,
 * then per group of pairs one persistent aggregation launch whose work list
 * holds every (pair, direction, scanline group) job of the group (the
 * long-axis scanlines of all its pairs first), then each pair's WTA, right
 * WTA and LR check, median and U/V maps on its branch.  Groups run side by
 * side, so one group's WTA passes (bound by HBM) overlap another group's
 * aggregation (bound by integer issue).  The paper has no counterpart. */
typedef struct sgm_batch_s *sgm_batch;

/* A batch of n pairs: pair i has W[i] x H[i] images and D[i] disparities.
 * params are checked for every pair as by sgm_create; row_pitch must be 0
 * (dense rows).  Allocates the pool (see sgm_batch_device_bytes) on the
 * current device, one CUDA stream per pair, and starts with one group per
 * pair and 3 resident aggregation blocks per SM. */
int sgm_batch_create(int n, const int *W, const int *H, const int *D, const sgm_params *params,
                     sgm_batch *out);

/* Frees the batch (synchronises its device first). */
int sgm_batch_destroy(sgm_batch b);

/* Runs every pair: left[i]/right[i] device images (H[i] x W[i]), disp[i]
 * device H[i] x W[i] output; umap/vmap NULL (no maps), or arrays of device
 * D[i] x W[i] and H[i] x D[i] outputs (a NULL pair of entries skips that
 * pair's maps).  The graph is captured on the first call and replayed while
 * the same buffers and tuning come back.  Asynchronous on `stream`.  Calls on
 * one batch must not overlap in time. */
int sgm_batch_run(sgm_batch b, const uint8_t *const *left, const uint8_t *const *right,
                  uint8_t *const *disp, uint16_t *const *umap, uint16_t *const *vmap, void *stream);

/* Number of groups (a power of two up to 64, capped at the number of pairs,
 * or n: one group per pair; pairs are dealt to groups largest first).  A
 * group of one pair runs the single-pair chain on the pair's stream (its own
 * aggregation launch, overlapped with its cost kernel); larger groups share
 * one persistent aggregation launch.  Then the aggregation kernel's
 * resident blocks per SM (1..16) and its 8-disparity chunks per lane (1, or
 * 4 when every pair's D spans at least 4 chunks and the cost is census; see
 * sgm_set_aggregation) of later runs.  Synchronises the device when the
 * grouping or the chunks per lane change. */
int sgm_batch_set_tuning(sgm_batch b, int groups, int blocks_per_sm, int chunks_per_lane);
int sgm_batch_get_tuning(sgm_batch b, int *groups, int *blocks_per_sm, int *chunks_per_lane);

/* Times runs on these buffers with 1, 2, 4, ... groups and one group per
 * pair at 2, 3 and 4 blocks per SM, each with 1 and (where allowed) 4 chunks per
 * lane, and keeps the fastest; any output may be NULL.  Synchronises. */
int sgm_batch_autotune(sgm_batch b, const uint8_t *const *left, const uint8_t *const *right,
                       uint8_t *const *disp, uint16_t *const *umap, uint16_t *const *vmap,
                       void *stream, int *best_groups, int *best_blocks_per_sm, int *best_chunks_per_lane);

/* Bytes of the batch's device pool: every pair's census codes, cost volume,
 * path planes and LR map, plus the job tables and work-queue state. */
int sgm_batch_device_bytes(sgm_batch b, size_t *bytes);

/* Shape of the aggregation kernel of later calls on h (the paper has no
 * counterpart): resident 4-warp blocks per SM (1..16) and 8-disparity chunks
 * per lane: 1, 2 or 4 for every direction, or SGM_AGG_CHUNKS_MIXED (the
 * long-axis scanlines, rows when W >= H, at 1 and the other directions at 2).
 * SGM_ERR_UNSUPPORTED above what D allows (D must span at least that many
 * chunks; the 16-bit costs of SGM_COST_SAD take 1).  With c chunks per lane a
 * scanline's D disparities occupy D / (8 c) lanes (rounded up to a power of
 * two), so a warp walks more scanlines at once with fewer instructions per
 * disparity estimate, but each step of a scanline takes longer.  Results do
 * not depend on either setting.  A new handle starts with 3 blocks per SM and
 * 1 chunk per lane, or with what sgm_autotune chose for its shape. */
#define SGM_AGG_CHUNKS_MIXED 3
int sgm_set_aggregation(sgm_handle h, int blocks_per_sm, int chunks_per_lane);
int sgm_get_aggregation(sgm_handle h, int *blocks_per_sm, int *chunks_per_lane);

/* Path schedules: how the aggregation of Eq. 2 is organised on the GPU.
 *   PLANES: every enabled direction is cut into independent scanlines that
 *     run concurrently over a materialised cost volume and write one plane
 *     per direction; a second kernel sums the planes and takes both winners
 *     and the LR check.  Any path set, D and cost.
 *   SWEEP: the paper's streaming organisation (Sec. 3.1.3, Fig. 2): one
 *     top-down pass in which the 0, 45, 90 and 135 degree paths of a row
 *     continue from the row above, with the matching cost, S, both winners
 *     and the LR check fused, so neither costs nor S reach memory.  Census
 *     cost, D <= 128, path masks within SGM_PATHS_STREAM4 (0x55); one warp per
 *     image row, rows_per_cta rows (2..8) per thread block, all blocks
 *     resident at once.
 *   AUTO: what sgm_autotune chose for this shape, else PLANES.
 * Both give the same disparities bit for bit. */
#define SGM_SCHEDULE_AUTO 0
#define SGM_SCHEDULE_PLANES 1
#define SGM_SCHEDULE_SWEEP 2

/* Selects the schedule of later calls on h (rows_per_cta is used by SWEEP
 * only).  SGM_ERR_UNSUPPORTED when h's parameters rule the sweep out or its
 * blocks cannot all be resident on the device; SGM_ERR_INVALID_ARG for an
 * unknown schedule or rows_per_cta outside 2..8.  h is unchanged on error. */
int sgm_set_schedule(sgm_handle h, int schedule, int rows_per_cta);

/* The schedule in use (SGM_SCHEDULE_PLANES or SGM_SCHEDULE_SWEEP, never AUTO)
 * and the sweep's rows per thread block; either pointer may be NULL. */
int sgm_get_schedule(sgm_handle h, int *schedule, int *rows_per_cta);

/* Autotuner: times the pipeline on this pair (device pointers as for
 * sgm_compute; disp is overwritten) with the PLANES schedule at 1, 2, 3, 4
 * and 6 resident aggregation blocks per SM, each with 1, 2 and 4 chunks per
 * lane and the mixed layout where D allows (sgm_set_aggregation), and, where
 * h can run it, the SWEEP
 * schedule at 2, 4 and 8 rows per block; keeps the fastest for h and for
 * handles created later in this process with the same W, H, D, path mask,
 * cost, window and P2.  *best_blocks_per_sm (may be NULL) receives the best
 * PLANES setting; sgm_get_schedule tells which schedule won.  Synchronises
 * `stream`. */
int sgm_autotune(sgm_handle h, const uint8_t *left, const uint8_t *right, uint8_t *disp,
                 void *stream, int *best_blocks_per_sm);

/* Short English text for a status code (static storage). */
const char *sgm_status_string(int status);

/* Sizes the handle was created with; any pointer may be NULL. */
int sgm_get_shape(sgm_handle h, int *W, int *H, int *D, int *census_bits);

/* Device memory, in bytes, that the library uses for W x H images with D
 * disparities and `params` (checked as by sgm_create; the paper has no
 * counterpart).  *handle_bytes: what sgm_create allocates (census codes, cost
 * volume, one plane per enabled path, LR map, work-queue state), without the
 * guard bytes of sgm_debug_canaries.  *host_staging_bytes: what the
 * host-buffer entry points add on their first use (two staging slots of
 * left, right, disp, U and V).  *static_bytes: the part of the fixed array
 * that sgm_compute_static would use (it runs only when this is at most
 * SGM_STATIC_SCRATCH_BYTES).  Any output pointer may be NULL.  No device call. */
int sgm_scratch_bytes(int W, int H, int D, const sgm_params *params, size_t *handle_bytes,
                      size_t *host_staging_bytes, size_t *static_bytes);

/* Rectification (Sec. 3.1.1): later calls on h read the left and right
 * images through integer maps, I_rect(x, y) = I(map_x(x, y), map_y(x, y)),
 * inside the census kernel's tile load.  Each map is a device W x H uint16
 * array owned by the caller, which keeps it alive and unchanged while h uses
 * it; a pixel whose map entry is >= W (x) or >= H (y) reads as 0.  Pass four
 * NULLs to switch rectification off (the default); 1 to 3 NULLs is
 * SGM_ERR_INVALID_ARG.  sgm_compute_static never rectifies. */
int sgm_set_rectification(sgm_handle h, const uint16_t *left_x, const uint16_t *left_y,
                          const uint16_t *right_x, const uint16_t *right_y);

/* ---- per-stage parity access (same kernels as sgm_compute) --------------- */

/* Census codes (Sec. 3.1.2), one uint64 per pixel, H x W each (device).
 * SGM_ERR_UNSUPPORTED for a handle with the SAD cost (it has no codes). */
int sgm_debug_census(sgm_handle h, const uint8_t *left, const uint8_t *right,
                     uint64_t *codes_left, uint64_t *codes_right, void *stream);

/* Aggregated cost L_r of direction r alone (Eq. 2), H x W x D uint16
 * (device), d fastest.  r must be enabled in the handle's path mask. */
int sgm_debug_path(sgm_handle h, int r, const uint8_t *left, const uint8_t *right,
                   uint16_t *L, void *stream);

/* Sum over the enabled paths S = C_aggr (Sec. 3.1.3), H x W x D uint16 (device). */
int sgm_debug_sum(sgm_handle h, const uint8_t *left, const uint8_t *right,
                  uint16_t *S, void *stream);

/* Matching cost C (Eq. 1, or the SAD of Sec. 3.1.2) computed by the given
 * kernel (SGM_COST_KERNEL_*), H x W x D uint16 (device), d fastest; entries
 * with x - d < 0 hold the largest cost (census bits, or window * 255).
 * SGM_ERR_UNSUPPORTED when the kernel cannot serve the handle: tensor cores
 * with D <= 16 or D > 128, or any kernel but AUTO on an SGM_COST_SAD handle. */
int sgm_debug_cost(sgm_handle h, const uint8_t *left, const uint8_t *right, int kernel,
                   uint16_t *C, void *stream);

/* Left WTA, right WTA and the map after the LR check, before the median
 * (Sec. 3.1.3-3.1.4), H x W bytes each (device); any may be NULL. */
int sgm_debug_raw(sgm_handle h, const uint8_t *left, const uint8_t *right,
                  uint8_t *disp_left, uint8_t *disp_right, uint8_t *disp_lr,
                  void *stream);

/* Cost kernel (SGM_COST_KERNEL_*) of later calls on h; AUTO when the handle
 * is created.  SGM_ERR_UNSUPPORTED as for sgm_debug_cost (h unchanged). */
int sgm_set_cost_kernel(sgm_handle h, int kernel);

/* Waits for the device, then returns SGM_ERR_TIMEOUT if a kernel of h gave up
 * a bounded device-side wait since the previous call (the tensor-core cost
 * kernel waits about one second at most for its matrix product, and then
 * writes no costs for that segment; the fused sweep waits about one second at
 * most for the row above it, and then leaves that call's disparity map
 * unfinished), else SGM_OK.  Clears the record. */
int sgm_device_status(sgm_handle h);

/* Test of the bounded device waits: runs the census and the tensor-core cost
 * kernel in a mode whose first wait is on an mbarrier that nothing arrives
 * at, so it gives up after 2 ms and records the timeout.  The matrix
 * products still complete and the handle stays usable; the cost volume of
 * this call is not valid.  On a handle using SGM_SCHEDULE_SWEEP it runs the
 * census and the fused sweep with row 1 waiting for a pixel the row above
 * never publishes: that wait gives up after 2 ms, every other row's wait
 * then ends at once, and this call's disparity map is not valid.  A
 * following sgm_device_status(h) returns SGM_ERR_TIMEOUT.
 * SGM_ERR_UNSUPPORTED where the tensor-core kernel cannot serve the handle
 * (see sgm_debug_cost), or, for the sweep, when the image has one row, the
 * sweep runs one row per block, or no enabled path comes from the row above. */
int sgm_debug_stalled_wait(sgm_handle h, const uint8_t *left, const uint8_t *right, void *stream);

/* Guarded builds only (the library compiled with -DSGM_GUARDED, which
 * paper_1807_06271_gb300.build makes as libsgm_guarded.so for tests; the
 * paper has no counterpart).  In them the census, CUDA-core cost,
 * aggregation, WTA, median and U/V kernels check every global index they
 * compute, and every image-dependent shared-memory index, against the
 * buffer's extent, skip an access out of range and count it.  Writes to
 * *hits the count on the current device since the last reset (synchronise
 * the device first), and resets it when reset != 0.  SGM_ERR_UNSUPPORTED in
 * the default build; SGM_ERR_CUDA if a counter cannot be read. */
int sgm_debug_guard_hits(unsigned long long *hits, int reset);

/* ---- fault-detection hooks (tests) ---------------------------------------- */

/* Process-wide: the n-th device allocation the library makes from now on
 * fails as if the device were out of memory (n = 0: none).  The call that
 * hits it returns SGM_ERR_OOM and releases what it had allocated. */
int sgm_debug_fail_alloc(int n);

/* Process-wide: handles created while on (1) place 256 guard bytes of 0xA5
 * before and after each of their device buffers (scratch and staging). */
int sgm_debug_canaries(int on);

/* Waits for the device, then checks every guard byte of h: SGM_OK, or
 * SGM_ERR_OVERRUN if one changed (a kernel wrote outside its buffer).
 * SGM_ERR_UNSUPPORTED for a handle created without canaries. */
int sgm_debug_check_canaries(sgm_handle h);

/* Changes the first guard byte after device buffer i of h (in allocation
 * order), from the host: the test of sgm_debug_check_canaries itself.
 * SGM_ERR_UNSUPPORTED without canaries, SGM_ERR_INVALID_ARG for a bad i. */
int sgm_debug_poke_canary(sgm_handle h, int i);

/* ---- stage timing (CUDA events on the caller's stream) ------------------- */

/* Record a start/stop event pair around every kernel of later calls. */
int sgm_set_timing(sgm_handle h, int enable);

/* Wait for the recorded work, then return for each stage i < n the summed
 * kernel time in ms (ms[i]) and the number of launches (count[i]) since the
 * previous read, and reset.  Either array may be NULL.  *n_stages receives
 * the number of stages. */
int sgm_get_stage_times(sgm_handle h, float *ms, int *count, int n, int *n_stages);

/* Name of stage i ("census", "aggregate", ...), NULL when out of range. */
const char *sgm_stage_name(int i);

/* ---- measurement ----------------------------------------------------------- */

/* Operation mixes of sgm_probe_int_rate (the paper has no counterpart; these
 * give the measured integer peak that the kernels' roofline is taken against). */
#define SGM_PROBE_INT32_ADD_MIN 0  /* add.u32 and min.u32 in turn                  */
#define SGM_PROBE_U16X2_MIN_ADD 1  /* min.u16x2 and add.u32 in turn: the packed
                                      arithmetic of the aggregation (two 16-bit
                                      operations per lane and instruction)          */
#define SGM_PROBE_POPC_XOR 2       /* xor.b32 then popc.b32: the Hamming cost       */

/* Times one launch of a probe kernel on the current device: 8 blocks of 256
 * threads per SM, each thread running 8 independent chains of `iters` steps
 * of the chosen two-operation mix (iters >= 8; about 20000 gives a launch of
 * a few ms).  *lane_ops_per_s receives the instructions executed per second,
 * counted per lane (a packed 16-bit instruction counts once); *ms (may be
 * NULL) the launch's event time.  Synchronises the device; allocates and
 * frees 256 bytes. */
int sgm_probe_int_rate(int kind, int iters, double *lane_ops_per_s, float *ms);

/* ---- no-allocation variant ------------------------------------------------ */

/* Size in bytes of the device array that holds the scratch of
 * sgm_compute_static.  Every GPU that loads the library reserves it when the
 * library's device code is loaded there and keeps it until the process exits. */
#define SGM_STATIC_SCRATCH_BYTES (32u << 20)

/* The disparity path of sgm_compute for one pair, with no handle and no
 * device allocation.  The paper has no counterpart: this entry point is for
 * callers that cannot call cudaMalloc, such as a camera loop with a hard
 * per-frame deadline (an allocation may block or fail mid-flight), a host
 * framework that owns all device memory through its own allocator, or code
 * that must avoid the device synchronisation cudaFree implies.
 *   Arguments and checks as sgm_create + sgm_compute: left/right are device
 *   images of H rows of row_pitch bytes, disp is a device H x W byte map.
 *   All three must be device (or managed) memory of one device, else
 *   SGM_ERR_INVALID_ARG; the call runs on that device whichever is current,
 *   and `stream` must belong to it.
 *   Scratch: census codes (2*W*H*4 bytes when census_w*census_h-1 <= 32, else
 *   2*W*H*8; none for SGM_COST_SAD), a cost volume and one plane per enabled
 *   path of W*H*Dp*e bytes each (Dp = D rounded up to 8 times a power of two:
 *   8, 16, 32, 64, 128 or 256; e = 1 for census, 2 for SAD), the aggregation's
 *   work-queue state and status word (4228 bytes) and a W*H byte map, each
 *   starting at a 256-byte boundary (sgm_scratch_bytes gives the total).  A
 *   call that needs more than SGM_STATIC_SCRATCH_BYTES returns
 *   SGM_ERR_UNSUPPORTED before any GPU work (320x240 with D=64 and 4 paths
 *   needs about 25 MiB).
 *   The first call on a device looks up the array's device address with that
 *   device current, and so does the first call after the device's context was
 *   made again (cudaDeviceReset); make those calls before any stream capture.
 *   All calls on a device share the one array and leave their data in it
 *   (nothing there needs to start at zero).  Calls whose work overlaps on the
 *   GPU (other streams, other host threads) race and corrupt each other's
 *   results: serialise them, e.g. on one stream.
 *   Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
int sgm_compute_static(int W, int H, int D, const sgm_params *params,
                       const uint8_t *left, const uint8_t *right, uint8_t *disp,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SGM_H */
