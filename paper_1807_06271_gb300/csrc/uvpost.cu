// U-/V-map post-processing (Sec. 3.2): threshold the count maps into binary
// maps inside a region of interest, dilate them with a square, and smooth
// them with a 3x3 binomial Gaussian.  One CTA per 32 x 8 output tile: the
// map tile plus a (r + 1)-cell halo is thresholded into shared memory, the
// dilation is taken over a 1-cell halo, and the Gaussian over the tile.
// Cells outside the map count as 0 in both filters.
#include "sgm_handle.cuh"

namespace sgm {
namespace {

constexpr int kTX = 32, kTY = 8, kMaxR = 7;

__global__ void __launch_bounds__(kTX *kTY)
    uvpost_kernel(const uint16_t *__restrict__ map, int rows, int cols, int threshold, int r0, int r1,
                  int c0, int c1, int rad, uint8_t *__restrict__ out) {
    wait_for_predecessor();
    constexpr int BH = kTY + 2 * (kMaxR + 1), BW = kTX + 2 * (kMaxR + 1);
    __shared__ uint8_t bin[BH][BW];               // thresholded, halo rad + 1
    __shared__ uint8_t dil[kTY + 2][kTX + 2];     // dilated, halo 1
    const int h = rad + 1;
    const int oy = blockIdx.y * kTY, ox = blockIdx.x * kTX;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int bh = kTY + 2 * h, bw = kTX + 2 * h;
    for (int i = tid; i < bh * bw; i += kTX * kTY) {
        const int ty = i / bw, tx = i - ty * bw;
        const int y = oy - h + ty, x = ox - h + tx;
        uint8_t b = 0;
        if (y >= 0 && y < rows && x >= 0 && x < cols && y >= r0 && y < r1 && x >= c0 && x < c1)
            b = map[(size_t)y * cols + x] >= threshold;
        bin[ty][tx] = b;
    }
    __syncthreads();
    for (int i = tid; i < (kTY + 2) * (kTX + 2); i += kTX * kTY) {
        const int ty = i / (kTX + 2), tx = i - ty * (kTX + 2);
        const int y = oy - 1 + ty, x = ox - 1 + tx;
        uint8_t v = 0;
        if (y >= 0 && y < rows && x >= 0 && x < cols) {
            for (int u = 0; u <= 2 * rad && !v; u++)
                for (int w = 0; w <= 2 * rad; w++)
                    if (bin[ty + u][tx + w]) {
                        v = 1;
                        break;
                    }
        }
        dil[ty][tx] = v;
    }
    __syncthreads();
    const int y = oy + threadIdx.y, x = ox + threadIdx.x;
    if (y >= rows || x >= cols) return;
    const int k[3] = {1, 2, 1};
    int acc = 0;
#pragma unroll
    for (int u = 0; u < 3; u++)
#pragma unroll
        for (int w = 0; w < 3; w++) acc += k[u] * k[w] * dil[threadIdx.y + u][threadIdx.x + w];
    out[(size_t)y * cols + x] = (uint8_t)((acc * 255 + 8) / 16);
}

cudaError_t launch_uvpost(const uint16_t *map, int rows, int cols, int threshold, const int *roi,
                          int rad, uint8_t *out, cudaStream_t s) {
    const dim3 grid((cols + kTX - 1) / kTX, (rows + kTY - 1) / kTY);
    uvpost_kernel<<<grid, dim3(kTX, kTY), 0, s>>>(map, rows, cols, threshold, roi[0], roi[1], roi[2],
                                                  roi[3], rad, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace sgm

extern "C" int uvmap_postprocess(sgm_handle h, const uint16_t *umap, const uint16_t *vmap,
                                 const sgm_uv_post *p, uint8_t *uout, uint8_t *vout, void *stream) {
    if (!h || !p || (!uout && !vout) || (uout && !umap) || (vout && !vmap)) return SGM_ERR_INVALID_ARG;
    if (p->dilate_r < 0 || p->dilate_r > sgm::kMaxR || p->u_threshold < 0 || p->v_threshold < 0)
        return SGM_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SGM_ERR_CUDA;
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return SGM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (uout) e = sgm::launch_uvpost(umap, h->D, h->W, p->u_threshold, p->u_roi, p->dilate_r, uout, s);
    if (e == cudaSuccess && vout)
        e = sgm::launch_uvpost(vmap, h->H, h->D, p->v_threshold, p->v_roi, p->dilate_r, vout, s);
    if (prev != h->device) cudaSetDevice(prev);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}
