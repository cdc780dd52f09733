// k x k median filter (Sec. 3.1.5) and the U-/V-disparity maps (Sec. 3.2).
#include "sgm_internal.cuh"

namespace sgm {
namespace {

// ---------------------------------------------------------------------------
// Median.  A 32 x 8 tile plus a (k-1)/2 halo with clamped (replicated)
// borders is staged in shared memory; each thread sorts its k*k window with
// Batcher's odd-even merge sort network (padded to a power of two with a
// value above every byte) and keeps element (k*k-1)/2.  Invalid pixels (0xFF)
// take part and sort above every valid disparity.
// ---------------------------------------------------------------------------

constexpr int kMX = 32, kMY = 8;

__device__ __forceinline__ void cmpswap(uint32_t &a, uint32_t &b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

template <int LO, int N, int R>
struct OddEvenMerge {
    static __device__ __forceinline__ void run(uint32_t *a) {
        constexpr int M = R * 2;
        if constexpr (M < N) {
            OddEvenMerge<LO, N, M>::run(a);
            OddEvenMerge<LO + R, N, M>::run(a);
#pragma unroll
            for (int i = LO + R; i + R < LO + N; i += M) cmpswap(a[i], a[i + R]);
        } else {
            cmpswap(a[LO], a[LO + R]);
        }
    }
};

template <int LO, int N>
struct OddEvenMergeSort {
    static __device__ __forceinline__ void run(uint32_t *a) {
        if constexpr (N > 1) {
            OddEvenMergeSort<LO, N / 2>::run(a);
            OddEvenMergeSort<LO + N / 2, N / 2>::run(a);
            OddEvenMerge<LO, N, 1>::run(a);
        }
    }
};

constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

template <int K>
__global__ void __launch_bounds__(kMX *kMY)
    median_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int W, int H) {
    wait_for_predecessor();
    constexpr int R = K / 2, TW = kMX + K - 1, TH = kMY + K - 1;
    constexpr int N = K * K, NP = pow2_at_least(N);
    __shared__ uint8_t tile[TH][TW];
    const int x0 = blockIdx.x * kMX - R, y0 = blockIdx.y * kMY - R;
    for (int i = threadIdx.y * kMX + threadIdx.x; i < TW * TH; i += kMX * kMY) {
        const int ty = i / TW, tx = i - ty * TW;
        const int gx = min(max(x0 + tx, 0), W - 1), gy = min(max(y0 + ty, 0), H - 1);
        const long long gi = (long long)gy * W + gx;
        tile[ty][tx] = in_range(gi, (long long)W * H) ? in[gi] : 0xFF;
    }
    __syncthreads();
    const int x = blockIdx.x * kMX + threadIdx.x, y = blockIdx.y * kMY + threadIdx.y;
    if (x >= W || y >= H) return;
    uint32_t v[NP];
#pragma unroll
    for (int i = 0; i < NP; i++)
        v[i] = i < N ? (uint32_t)tile[threadIdx.y + i / K][threadIdx.x + i % K] : 0x100u;
    OddEvenMergeSort<0, NP>::run(v);
    if (in_range((long long)y * W + x, (long long)W * H)) out[(size_t)y * W + x] = (uint8_t)v[(N - 1) / 2];
}

// ---------------------------------------------------------------------------
// U- and V-maps in one launch of 1024-thread CTAs.  The first ceil(W/32)
// CTAs build the U-map of a 32-column strip: 32 row phases x 32 columns walk
// the strip and bump a shared [D][32] histogram; each column's counts are
// then written once.  The remaining CTAs build the V-map of 8 rows each with
// shared [8][D] histograms.  Every output element is written exactly once,
// so no clearing is needed.
// ---------------------------------------------------------------------------

constexpr int kUVThreads = 1024, kVRows = 8;

__global__ void __launch_bounds__(kUVThreads)
    uvmap_kernel(const uint8_t *__restrict__ disp, int W, int H, int D, int ustrips,
                 uint16_t *__restrict__ umap, uint16_t *__restrict__ vmap) {
    extern __shared__ uint32_t hist[];
    wait_for_predecessor();
    if ((int)blockIdx.x < ustrips) {
        const int x0 = blockIdx.x * 32;
        const int col = threadIdx.x & 31, phase = threadIdx.x >> 5, nphase = kUVThreads / 32;
        for (int i = threadIdx.x; i < D * 32; i += kUVThreads) hist[i] = 0;
        __syncthreads();
        const int x = x0 + col;
        if (x < W) {
            for (int y = phase; y < H; y += nphase) {
                const int d = in_range((long long)y * W + x, (long long)W * H) ? disp[(size_t)y * W + x] : 0xFF;
                if (d < D && in_range(d * 32 + col, D * 32)) atomicAdd(&hist[d * 32 + col], 1u);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < D * 32; i += kUVThreads) {
            const int d = i >> 5, c = i & 31;
            if (x0 + c < W && in_range((long long)d * W + x0 + c, (long long)D * W)) umap[(size_t)d * W + x0 + c] = (uint16_t)hist[i];
        }
    } else {
        const int y0 = ((int)blockIdx.x - ustrips) * kVRows;
        for (int i = threadIdx.x; i < kVRows * D; i += kUVThreads) hist[i] = 0;
        __syncthreads();
        const int rows = min(kVRows, H - y0);
        for (int i = threadIdx.x; i < rows * W; i += kUVThreads) {
            const int r = i / W, x = i - r * W;
            const int d = in_range((long long)(y0 + r) * W + x, (long long)W * H) ? disp[(size_t)(y0 + r) * W + x] : 0xFF;
            if (d < D && in_range(r * D + d, kVRows * D)) atomicAdd(&hist[r * D + d], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < rows * D; i += kUVThreads)
            if (in_range((long long)y0 * D + i, (long long)H * D)) vmap[(size_t)y0 * D + i] = (uint16_t)hist[i];
    }
}

}  // namespace

SGM_GUARD_COUNTER(guard_hits_post)

cudaError_t launch_median(const uint8_t *in, uint8_t *out, int W, int H, int k, cudaStream_t s) {
    dim3 block(kMX, kMY), grid((W + kMX - 1) / kMX, (H + kMY - 1) / kMY);
    switch (k) {
        case 3: return launch_k(median_kernel<3>, grid, block, 0, s, in, out, W, H);
        case 5: return launch_k(median_kernel<5>, grid, block, 0, s, in, out, W, H);
        case 7: return launch_k(median_kernel<7>, grid, block, 0, s, in, out, W, H);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_uvmap(const uint8_t *disp, int W, int H, int D, uint16_t *umap, uint16_t *vmap,
                         cudaStream_t s) {
    const int ustrips = (W + 31) / 32, vblocks = (H + kVRows - 1) / kVRows;
    const size_t smem = (size_t)(D * 32 > kVRows * D ? D * 32 : kVRows * D) * sizeof(uint32_t);
    return launch_k(uvmap_kernel, dim3(ustrips + vblocks), dim3(kUVThreads), smem, s, disp, W, H, D, ustrips,
                    umap, vmap);
}

}  // namespace sgm
