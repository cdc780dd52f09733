// Semi-global path aggregation (Sec. 3.1.3, Eq. 2) with the matching cost of
// Eq. 1 computed on the fly from census codes.
//
// Work decomposition: every path direction splits the image into independent
// scanlines (rows for the horizontal paths, columns for the vertical ones,
// W+H-1 diagonals for each diagonal direction).  One warp walks one scanline
// from the image border; the D disparities of the current pixel are spread
// over the 32 lanes, DPL consecutive disparities per lane.  Per step a lane
//   - computes its DPL costs C(p,d) = popc(code_l(p) ^ code_r(p_x - d)), or the
//     code width when p_x - d < 0,
//   - fetches the d-1 / d+1 neighbours across its lane boundary with one
//     shuffle each way,
//   - applies L(p,d) = C + min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m'+P2) - m',
//   - and the warp reduces m = min_d L(p,d) with one redux instruction.
// L values never exceed code bits + P2 <= 255, so each path writes its own
// uint8 plane [H][W][D]; the WTA kernel sums the planes.
#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr uint32_t kInf = 0x7FFF;  // above every reachable value, small enough not to overflow

__device__ __forceinline__ uint32_t popcnt(uint32_t v) { return __popc(v); }
__device__ __forceinline__ uint32_t popcnt(uint64_t v) { return __popcll(v); }

template <int DPL, typename CodeT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    aggregate_kernel(const CodeT *__restrict__ codes, int W, int H, int D, int nbits, int P1,
                     int P2, PathJobs jobs, uint8_t *__restrict__ planes, size_t plane_elems) {
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (g >= jobs.begin[jobs.n]) return;  // uniform per warp
    int k = 0;
    while (g >= jobs.begin[k + 1]) k++;
    const int s = g - jobs.begin[k];
    const int dx = jobs.dx[k], dy = jobs.dy[k];
    int x, y;
    if (dy == 0) {
        y = s;
        x = dx > 0 ? 0 : W - 1;
    } else if (dx == 0) {
        x = s;
        y = dy > 0 ? 0 : H - 1;
    } else if (s < W) {
        x = s;
        y = dy > 0 ? 0 : H - 1;
    } else {
        const int t = s - W + 1;
        x = dx > 0 ? 0 : W - 1;
        y = dy > 0 ? t : H - 1 - t;
    }
    const CodeT *__restrict__ cl = codes;
    const CodeT *__restrict__ cr = codes + (size_t)W * H;
    uint8_t *__restrict__ plane = planes + (size_t)jobs.plane[k] * plane_elems;
    const int d0 = lane * DPL;
    const bool packed_store = (DPL == 4) && ((D & 3) == 0);

    uint32_t L[DPL];
    uint32_t m = 0;
    bool first = true;
    while (x >= 0 && x < W && y >= 0 && y < H) {
        const size_t pix = (size_t)y * W + x;
        const CodeT code_l = cl[pix];
        const CodeT *__restrict__ crow = cr + (size_t)y * W;
        uint32_t c[DPL];
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            const int xr = x - (d0 + j);
            c[j] = xr >= 0 ? popcnt(code_l ^ crow[xr]) : (uint32_t)nbits;
        }
        uint32_t Ln[DPL];
        if (first) {
#pragma unroll
            for (int j = 0; j < DPL; j++) Ln[j] = c[j];
        } else {
            uint32_t lnb = __shfl_up_sync(0xffffffffu, L[DPL - 1], 1);
            uint32_t rnb = __shfl_down_sync(0xffffffffu, L[0], 1);
            if (lane == 0) lnb = kInf;
            if (lane == 31) rnb = kInf;
            const uint32_t mp2 = m + P2;
#pragma unroll
            for (int j = 0; j < DPL; j++) {
                const uint32_t lm = j == 0 ? lnb : L[j - 1];
                const uint32_t rm = j == DPL - 1 ? rnb : L[j + 1];
                uint32_t t = min(L[j], min(lm, rm) + P1);
                t = min(t, mp2);
                Ln[j] = c[j] + t - m;
            }
        }
        uint32_t lmin = kInf;
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            if (d0 + j >= D) Ln[j] = kInf;  // disparities past D never win and never act as d+1
            lmin = min(lmin, Ln[j]);
        }
        m = __reduce_min_sync(0xffffffffu, lmin);
        uint8_t *out = plane + pix * D;
        if (packed_store) {
            if (d0 < D)
                *reinterpret_cast<uint32_t *>(out + d0) =
                    Ln[0] | (Ln[1 % DPL] << 8) | (Ln[2 % DPL] << 16) | (Ln[3 % DPL] << 24);
        } else {
#pragma unroll
            for (int j = 0; j < DPL; j++)
                if (d0 + j < D) out[d0 + j] = (uint8_t)Ln[j];
        }
#pragma unroll
        for (int j = 0; j < DPL; j++) L[j] = Ln[j];
        first = false;
        x += dx;
        y += dy;
    }
}

template <typename CodeT>
cudaError_t launch_t(const CodeT *codes, int W, int H, int D, int nbits, int P1, int P2,
                     const PathJobs &jobs, uint8_t *planes, size_t plane_elems, cudaStream_t s) {
    const int warps = jobs.begin[jobs.n];
    const int blocks = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks == 0) return cudaSuccess;
    const int threads = kWarpsPerBlock * 32;
    if (D <= 32)
        aggregate_kernel<1, CodeT><<<blocks, threads, 0, s>>>(codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems);
    else if (D <= 64)
        aggregate_kernel<2, CodeT><<<blocks, threads, 0, s>>>(codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems);
    else if (D <= 128)
        aggregate_kernel<4, CodeT><<<blocks, threads, 0, s>>>(codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems);
    else
        aggregate_kernel<8, CodeT><<<blocks, threads, 0, s>>>(codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_aggregate(const void *codes, int code_bytes, int W, int H, int D, int nbits,
                             int P1, int P2, const PathJobs &jobs, uint8_t *planes,
                             size_t plane_elems, cudaStream_t s) {
    if (code_bytes == 4)
        return launch_t((const uint32_t *)codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems, s);
    return launch_t((const uint64_t *)codes, W, H, D, nbits, P1, P2, jobs, planes, plane_elems, s);
}

}  // namespace sgm
