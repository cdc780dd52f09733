// U-/V-map post-processing (Sec. 3.2): threshold the count maps into binary
// maps inside a region of interest, dilate them with a square, and smooth
// them with a 3x3 binomial Gaussian.  One launch covers both maps: the first
// CTAs take 32 x 8 output tiles of the U-map, the rest tiles of the V-map.
// A CTA thresholds its tile plus a (r + 1)-cell halo into shared memory,
// dilates separably (an OR over 2r + 1 cells along each row, then along each
// column, for the tile and a 1-cell halo) and applies the Gaussian over the
// tile.  Cells outside the map count as 0 in both filters.
#include "sgm_handle.cuh"

namespace sgm {
namespace {

constexpr int kTX = 32, kTY = 8, kMaxR = 7;

// One map to post-process (out == nullptr: none).
struct PostMap {
    const uint16_t *map;
    int rows, cols, threshold, r0, r1, c0, c1;
    uint8_t *out;
};

__host__ __device__ inline int tiles_x(const PostMap &m) { return m.out ? (m.cols + kTX - 1) / kTX : 0; }
__host__ __device__ inline int tiles_of(const PostMap &m) { return m.out ? tiles_x(m) * ((m.rows + kTY - 1) / kTY) : 0; }

__global__ void __launch_bounds__(kTX *kTY) uvpost_kernel(PostMap ma, PostMap mb, int rad) {
    wait_for_predecessor();
    constexpr int BH = kTY + 2 * (kMaxR + 1), BW = kTX + 2 * (kMaxR + 1);
    __shared__ uint8_t bin[BH][BW];               // thresholded, halo rad + 1
    __shared__ uint8_t rowor[BH][kTX + 2];        // OR over 2 rad + 1 cells of each bin row
    __shared__ uint8_t dil[kTY + 2][kTX + 2];     // dilated, halo 1
    const int na = tiles_of(ma);
    const bool second = (int)blockIdx.x >= na;
    const PostMap &m = second ? mb : ma;
    const int t = second ? (int)blockIdx.x - na : (int)blockIdx.x;
    const int oy = (t / tiles_x(m)) * kTY, ox = (t % tiles_x(m)) * kTX;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    const int h = rad + 1, bh = kTY + 2 * h, bw = kTX + 2 * h;
    for (int i = tid; i < bh * bw; i += kTX * kTY) {
        const int ty = i / bw, tx = i - ty * bw;
        const int y = oy - h + ty, x = ox - h + tx;
        uint8_t b = 0;
        if (y >= 0 && y < m.rows && x >= 0 && x < m.cols && y >= m.r0 && y < m.r1 && x >= m.c0 && x < m.c1)
            b = m.map[(size_t)y * m.cols + x] >= m.threshold;
        bin[ty][tx] = b;
    }
    __syncthreads();
    // rowor[ty][tx] covers map cells (oy - h + ty, ox - 1 + tx - rad .. ox - 1 + tx + rad)
    for (int i = tid; i < bh * (kTX + 2); i += kTX * kTY) {
        const int ty = i / (kTX + 2), tx = i - ty * (kTX + 2);
        uint8_t v = 0;
        for (int w = 0; w <= 2 * rad; w++) v |= bin[ty][tx + w];
        rowor[ty][tx] = v;
    }
    __syncthreads();
    for (int i = tid; i < (kTY + 2) * (kTX + 2); i += kTX * kTY) {
        const int ty = i / (kTX + 2), tx = i - ty * (kTX + 2);
        const int y = oy - 1 + ty, x = ox - 1 + tx;
        uint8_t v = 0;
        if (y >= 0 && y < m.rows && x >= 0 && x < m.cols)
            for (int u = 0; u <= 2 * rad; u++) v |= rowor[ty + u][tx];
        dil[ty][tx] = v;
    }
    __syncthreads();
    const int y = oy + threadIdx.y, x = ox + threadIdx.x;
    if (y >= m.rows || x >= m.cols) return;
    const int k[3] = {1, 2, 1};
    int acc = 0;
#pragma unroll
    for (int u = 0; u < 3; u++)
#pragma unroll
        for (int w = 0; w < 3; w++) acc += k[u] * k[w] * dil[threadIdx.y + u][threadIdx.x + w];
    m.out[(size_t)y * m.cols + x] = (uint8_t)((acc * 255 + 8) / 16);
}

cudaError_t launch_uvpost(const PostMap &a, const PostMap &b, int rad, cudaStream_t s) {
    const int n = tiles_of(a) + tiles_of(b);
    if (n == 0) return cudaSuccess;
    return launch_k(uvpost_kernel, dim3(n), dim3(kTX, kTY), 0, s, a, b, rad);
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
    const sgm::PostMap u{umap, h->D, h->W, p->u_threshold, p->u_roi[0], p->u_roi[1], p->u_roi[2], p->u_roi[3], uout};
    const sgm::PostMap v{vmap, h->H, h->D, p->v_threshold, p->v_roi[0], p->v_roi[1], p->v_roi[2], p->v_roi[3], vout};
    const cudaError_t e = sgm::launch_uvpost(u, v, p->dilate_r, s);
    if (prev != h->device) cudaSetDevice(prev);
    return e == cudaSuccess ? SGM_OK : SGM_ERR_CUDA;
}
