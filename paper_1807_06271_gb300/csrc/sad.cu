// SAD matching cost (Sec. 3.1.2: the pixel-wise sum of absolute differences,
// over the 5 x 5 support region of Sec. 4.1):
//     C(x,y,d) = sum over |u| <= rw, |v| <= rh of |I_l(x+u, y+v) - I_r(x-d+u, y+v)|
// with both images read at clamped (replicated) coordinates, and the maximum
// cmax = ww * wh * 255 where x - d < 0 and in the padding slots d >= D.
//
// One CTA per segment of kSeg pixels of kRows consecutive rows.  The left
// rows (kSeg + 2 rw columns) and right rows (kSeg + Dp - 1 + 2 rw columns)
// the segment reaches, kRows + wh - 1 of each, are staged once in shared
// memory, read through the rectification maps when they are set, directly
// as the packed 16-bit pairs the arithmetic uses: (l, l) for a left pixel
// and (R[c], R[c-4]) for right column c.  For each column j of the segment
// and its halo and each 8-disparity chunk the CTA keeps the vertical sums
//     V(j, d) = sum_v |I_l(j, v) - I_r(j - d, v)|
// as four words, word k = the pair (d+k, d+k+4): the first row sums wh rows
// of absolute differences, each later row adds the row entering the window
// and subtracts the one leaving it (halves never borrow: V holds the row
// that leaves).  |a - b| = max.u16x2 - min.u16x2 (full rate on GB300).
// Each row's costs then add ww neighbouring columns of V, four packed adds
// per chunk and column (halves never carry: a cost is at most
// ww * wh * 255 <= 32766), and go out as one 16-byte chunk per (pixel, lane)
// in the wide lane-chunk order; consecutive threads write consecutive chunks
// of the segment's contiguous pixel records.
#include "sgm_internal.cuh"

namespace sgm {
namespace {

// 64 pixels x 4 rows per CTA: rows per CTA against threads measured on GB300
// (640 x 360, D = 60, 5 x 5): 8 rows 29.0 us, 16 rows 38.3, 2 rows (128
// threads) 29.0, 4 rows 27.0 us; more CTAs hide the row staging better.
constexpr int kSeg = 64, kRows = 4, kThreads = 256;

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// |a - b| of the pair words of one staged row for chunk (j, i), added to or
// subtracted from the chunk's four vertical-sum words.
template <bool ADD>
__device__ __forceinline__ void absdiff_row(uint4 &v, uint32_t l, const uint32_t *r) {
    const uint32_t r0 = r[0], r1 = r[-1], r2 = r[-2], r3 = r[-3];
    const uint32_t a0 = vmax2(l, r0) - vmin2(l, r0), a1 = vmax2(l, r1) - vmin2(l, r1);
    const uint32_t a2 = vmax2(l, r2) - vmin2(l, r2), a3 = vmax2(l, r3) - vmin2(l, r3);
    if (ADD) {
        v.x += a0;
        v.y += a1;
        v.z += a2;
        v.w += a3;
    } else {
        v.x -= a0;
        v.y -= a1;
        v.z -= a2;
        v.w -= a3;
    }
}

template <bool RECT>
__global__ void __launch_bounds__(kThreads)
    sad_cost_kernel(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch,
                    int W, int H, int D, int Dp, int ww, int wh, RectMaps maps,
                    uint4 *__restrict__ cost, unsigned *__restrict__ job_state) {
    extern __shared__ __align__(16) unsigned char sad_smem[];
    wait_for_predecessor();
    if (job_state && blockIdx.x == 0 && blockIdx.y == 0)
        for (int i = threadIdx.x; i < (int)(kJobStateBytes / sizeof(unsigned)); i += kThreads) job_state[i] = 0u;
    const int rw = ww / 2, rh = wh / 2;
    const int ncol = kSeg + 2 * rw;          // V columns (segment + halo)
    const int lcols = ncol, rcols = kSeg + Dp - 1 + 2 * rw;
    const int chunks = Dp / 8;
    const int y0 = blockIdx.y * kRows, x0 = blockIdx.x * kSeg;
    const int nrows = min(kRows, H - y0);   // output rows of this CTA
    const int srows = nrows + wh - 1;       // staged rows: y0 - rh .. y0 + nrows - 1 + rh
    uint4 *V = reinterpret_cast<uint4 *>(sad_smem);                              // [ncol][chunks]
    uint32_t *Lp = reinterpret_cast<uint32_t *>(V + (size_t)ncol * chunks);      // [srows][lcols]: (l, l)
    uint8_t *Rb = reinterpret_cast<uint8_t *>(Lp + srows * lcols);               // [srows][rcols] bytes
    uint32_t *Rp = reinterpret_cast<uint32_t *>(Rb + ((srows * rcols + 3) & ~3));  // [srows][rcols]: (R[c], R[c-4])
    const int xl0 = x0 - rw;            // image column of left column 0
    const int xr0 = x0 - rw - (Dp - 1);  // image column of right column 0
    for (int i = threadIdx.x; i < srows * lcols; i += kThreads) {
        const int v = i / lcols, c = i - v * lcols;
        const int gy = min(max(y0 + v - rh, 0), H - 1), gx = min(max(xl0 + c, 0), W - 1);
        Lp[i] = rect_pixel<RECT>(left, pitch, W, H, gx, gy, maps.lx, maps.ly) * 0x00010001u;
    }
    for (int i = threadIdx.x; i < srows * rcols; i += kThreads) {
        const int v = i / rcols, c = i - v * rcols;
        const int gy = min(max(y0 + v - rh, 0), H - 1), gx = min(max(xr0 + c, 0), W - 1);
        Rb[i] = rect_pixel<RECT>(right, pitch, W, H, gx, gy, maps.rx, maps.ry);
    }
    __syncthreads();
    // right pairs; columns c < 4 have no c - 4 and are only read as the low half
    for (int i = threadIdx.x; i < srows * rcols; i += kThreads) {
        const int v = i / rcols, c = i - v * rcols;
        Rp[i] = Rb[i] | (c >= 4 ? (uint32_t)Rb[i - 4] << 16 : 0u);
    }
    __syncthreads();
    const uint32_t cmax = (uint32_t)(ww * wh * 255);
    const int npx = min(kSeg, W - x0);
    const bool ragged = D != Dp, border = x0 < Dp;
    for (int r = 0; r < nrows; r++) {
        // Vertical sums of output row y0 + r (staged rows r .. r + wh - 1).  Word k
        // of chunk (j, i) reads the right pair at c0 - k, c0 = j + Dp - 1 - 8i:
        // column j - d + Dp - 1 for d = 8i + k, high half 4 columns left (>= j >= 0).
        for (int it = threadIdx.x; it < ncol * chunks; it += kThreads) {
            const int j = it / chunks, i = it - j * chunks;
            const int c0 = j + Dp - 1 - 8 * i;
            uint4 v;
            if (r == 0) {
                v = make_uint4(0u, 0u, 0u, 0u);
                for (int q = 0; q < wh; q++) absdiff_row<true>(v, Lp[q * lcols + j], Rp + q * rcols + c0);
            } else {
                v = V[it];
                const int qin = r + wh - 1, qout = r - 1;
                absdiff_row<true>(v, Lp[qin * lcols + j], Rp + qin * rcols + c0);
                absdiff_row<false>(v, Lp[qout * lcols + j], Rp + qout * rcols + c0);
            }
            V[it] = v;
        }
        __syncthreads();
        // C(x, d) = sum over u < ww of V(x - x0 + u, d); cmax where x - d < 0 or d >= D.
        uint4 *out = cost + ((size_t)(y0 + r) * W + x0) * chunks;
        for (int it = threadIdx.x; it < npx * chunks; it += kThreads) {
            const int px = it / chunks, i = it - px * chunks;
            uint32_t s[4] = {0u, 0u, 0u, 0u};
            for (int u = 0; u < ww; u++) {
                const uint4 q = V[(px + u) * chunks + i];
                s[0] += q.x;
                s[1] += q.y;
                s[2] += q.z;
                s[3] += q.w;
            }
            if (ragged || border) {
                const int x = x0 + px;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int dlo = 8 * i + k, dhi = dlo + 4;
                    const bool mlo = dlo >= D || x - dlo < 0, mhi = dhi >= D || x - dhi < 0;
                    s[k] = (mlo ? cmax : (s[k] & 0xFFFFu)) | ((mhi ? cmax : (s[k] >> 16)) << 16);
                }
            }
            out[it] = make_uint4(s[0], s[1], s[2], s[3]);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_sad_cost(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                            int D, int ww, int wh, const RectMaps &maps, uint16_t *cost,
                            unsigned *job_state, cudaStream_t s) {
    if (disparities_per_lane(D) != 8 || ww < 1 || wh < 1 || ww > kMaxSadWindow || wh > kMaxSadWindow)
        return cudaErrorInvalidValue;
    const int Dp = padded_disparities(D);
    const int rw = ww / 2;
    const int ncol = kSeg + 2 * rw, rcols = kSeg + Dp - 1 + 2 * rw;
    const size_t srows = (size_t)kRows + wh - 1;
    const size_t smem = (size_t)ncol * (Dp / 8) * sizeof(uint4) + srows * ncol * 4 +
                        ((srows * rcols + 3) & ~(size_t)3) + srows * rcols * 4;
    const dim3 grid((W + kSeg - 1) / kSeg, (H + kRows - 1) / kRows);
    uint4 *out = reinterpret_cast<uint4 *>(cost);
    cudaError_t e;
    auto kernel = maps.lx ? sad_cost_kernel<true> : sad_cost_kernel<false>;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_k(kernel, grid, dim3(kThreads), smem, s, left, right, pitch, W, H, D, Dp, ww, wh, maps, out,
                    job_state);
}

}  // namespace sgm
