// Winner-takes-all on S = sum of the path planes (Sec. 3.1.3), the right
// disparity taken from the same S (Sec. 3.1.4) and the left-right check.
//
// One CTA per image row.  A warp handles one pixel at a time with the
// disparities across its lanes: it sums the path planes into S(x, d), forms
// the key (S << 8) | d, reduces the left winner with one redux (ties go to
// the smallest d because d sits in the low bits) and folds every key into
// the right-disparity slot x - d with a shared-memory atomicMin, which gives
// D_right(x') = argmin_d S(x' + d, d) with the same tie rule.  After a CTA
// barrier the row's LR check runs from shared memory.
#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kThreads = 256;

template <int DPL>
__global__ void __launch_bounds__(kThreads)
    wta_kernel(const uint8_t *__restrict__ planes, int nplanes, size_t plane_elems, int W, int H,
               int D, int tol, uint8_t *__restrict__ disp_lr, uint8_t *__restrict__ dbg_left,
               uint8_t *__restrict__ dbg_right, uint16_t *__restrict__ dbg_sum) {
    extern __shared__ uint32_t smem[];
    uint32_t *key_right = smem;                            // W keys
    uint8_t *dl_row = reinterpret_cast<uint8_t *>(smem + W);  // W bytes
    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kThreads / 32;
    for (int i = threadIdx.x; i < W; i += kThreads) key_right[i] = 0xFFFFFFFFu;
    __syncthreads();
    const int d0 = lane * DPL;
    const bool packed = (DPL == 4) && ((D & 3) == 0);
    for (int x = warp; x < W; x += nwarps) {
        const size_t pix = (size_t)y * W + x;
        uint32_t s[DPL];
#pragma unroll
        for (int j = 0; j < DPL; j++) s[j] = 0;
        if (packed) {
            if (d0 < D) {
                for (int p = 0; p < nplanes; p++) {
                    const uint32_t v =
                        *reinterpret_cast<const uint32_t *>(planes + p * plane_elems + pix * D + d0);
#pragma unroll
                    for (int j = 0; j < DPL; j++) s[j] += (v >> (8 * (j & 3))) & 0xFFu;
                }
            }
        } else {
            for (int p = 0; p < nplanes; p++)
#pragma unroll
                for (int j = 0; j < DPL; j++)
                    if (d0 + j < D) s[j] += planes[p * plane_elems + pix * D + d0 + j];
        }
        uint32_t best = 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            const int d = d0 + j;
            if (d < D) {
                const uint32_t key = (s[j] << 8) | (uint32_t)d;
                best = min(best, key);
                if (x - d >= 0) atomicMin(&key_right[x - d], key);
                if (dbg_sum) dbg_sum[pix * D + d] = (uint16_t)s[j];
            }
        }
        best = __reduce_min_sync(0xffffffffu, best);
        if (lane == 0) dl_row[x] = (uint8_t)(best & 0xFFu);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += kThreads) {
        const int dl = dl_row[x];
        uint8_t v = (uint8_t)dl;
        if (tol >= 0) {
            const int xr = x - dl;
            if (xr < 0) {
                v = SGM_INVALID;
            } else {
                const int dr = (int)(key_right[xr] & 0xFFu);
                const int diff = dl > dr ? dl - dr : dr - dl;
                if (diff > tol) v = SGM_INVALID;
            }
        }
        const size_t pix = (size_t)y * W + x;
        disp_lr[pix] = v;
        if (dbg_left) dbg_left[pix] = (uint8_t)dl;
        if (dbg_right) dbg_right[pix] = (uint8_t)(key_right[x] & 0xFFu);
    }
}

}  // namespace

cudaError_t launch_wta(const uint8_t *planes, int nplanes, size_t plane_elems, int W, int H, int D,
                       int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                       uint16_t *dbg_sum, cudaStream_t s) {
    const size_t smem = (size_t)W * sizeof(uint32_t) + (size_t)((W + 3) & ~3);
    if (D <= 32)
        wta_kernel<1><<<H, kThreads, smem, s>>>(planes, nplanes, plane_elems, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum);
    else if (D <= 64)
        wta_kernel<2><<<H, kThreads, smem, s>>>(planes, nplanes, plane_elems, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum);
    else if (D <= 128)
        wta_kernel<4><<<H, kThreads, smem, s>>>(planes, nplanes, plane_elems, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum);
    else
        wta_kernel<8><<<H, kThreads, smem, s>>>(planes, nplanes, plane_elems, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum);
    return cudaGetLastError();
}

}  // namespace sgm
