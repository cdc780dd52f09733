// Winner-takes-all on S = sum of the path planes (Sec. 3.1.3), the right
// disparity taken from the same S (Sec. 3.1.4) and the left-right check.
//
// One CTA per image row.  The planes share the aggregation kernel's layout
// (all planes of a pixel back to back): LPS lanes hold a pixel's
// disparities, DPL per lane, so a warp covers G = 32 / LPS neighbouring
// pixels.  A lane loads its chunk of every plane (8 bytes of 8-bit path
// costs, or 16 bytes of 16-bit ones) at fixed offsets from one pointer, one
// or two pixel groups ahead of its use (register buffers), turns each into
// DPL/2 packed 16-bit pairs (d+k, d+k+DPL/2) (masks and byte-permutes for
// 8-bit planes; 16-bit planes are stored that way) and adds them.  No half
// carries: S <= 8 * 255 for 8-bit planes, and the host bounds the 16-bit
// path costs so that their sum fits 16 bits.  For each disparity it forms the
// key (S << 8) | d; the left winner is the minimum key over the pixel's lanes
// (ties go to the smallest d, which sits in the low bits), and every key is
// folded into slot x - d of a shared-memory array with atomicMin, which leaves
// D_right(x') = argmin_d S(x' + d, d) with the same tie rule.  After a CTA
// barrier the row's LR check runs from shared memory.  HBM traffic: the
// planes once (npaths * Dp path costs per pixel) plus 1 byte written per pixel.
#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kLo = 0x00FF00FFu;

// Minimum of v over the LPS lanes of this lane's pixel: one full-warp
// redux.sync per pixel group, fed 0xFFFFFFFF by the other groups' lanes.
template <int LPS>
__device__ __forceinline__ uint32_t group_min(uint32_t v, int lane) {
    constexpr int G = 32 / LPS;
    if constexpr (LPS == 1) {
        return v;
    } else if constexpr (G == 1) {
        return __reduce_min_sync(0xffffffffu, v);
    } else {
        const int grp = lane / LPS;
        uint32_t m = 0;
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t r = __reduce_min_sync(0xffffffffu, grp == g ? v : 0xFFFFFFFFu);
            if (grp == g) m = r;
        }
        return m;
    }
}

// The planes are read exactly once: keep them out of L1 and evict them first from L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// One lane's chunk of one plane: DPL bytes (8-bit path costs) or 2*DPL bytes
// (16-bit, "wide"), loaded as 32-bit words w[0..kWords).
template <int DPL, bool WIDE>
struct PlaneChunk {
    static constexpr int kWords = WIDE ? DPL / 2 : DPL / 4;
    static_assert(kWords == 2 || kWords == 4, "a lane chunk is 8 or 16 bytes");
    uint32_t w[kWords];
};
template <int DPL, bool WIDE>
__device__ __forceinline__ PlaneChunk<DPL, WIDE> ld_plane(const uint8_t *p, uint64_t pol) {
    PlaneChunk<DPL, WIDE> v;
    if constexpr (PlaneChunk<DPL, WIDE>::kWords == 2) {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                     : "=r"(v.w[0]), "=r"(v.w[1])
                     : "l"(p), "l"(pol));
    } else {
        asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
                     : "l"(p), "l"(pol));
    }
    return v;
}

// XOR mask on the lane's visiting order of its disparities: with it the
// shared-memory atomics that a warp issues together fall into distinct banks
// (checked exhaustively for every (DPL, LPS) in use).
template <int DPL, int LPS>
__device__ __forceinline__ int visit_mask(int li) {
    static_assert(DPL == 8, "masks are tabulated for 8 disparities per lane");
    if constexpr (LPS == 8) return 4 * ((li >> 2) & 1);
    else if constexpr (LPS == 16) return 2 * ((li >> 2) & 3);
    else if constexpr (LPS == 32) return ((li >> 2) & 3) + 4 * ((li >> 4) & 1);
    else return 0;
}

// Sums the path planes of one pixel into DPL/2 packed pairs S[k] = (S(d0+k), S(d0+k+h)),
// h = DPL/2, folds its keys into the right-disparity slots and returns its smallest key.
// NP > 0: NP planes (compile time); NP == 0: nplanes at run time.
template <int LPS, int DPL, bool WIDE, int NP, bool RAGGED, bool DEBUG>
__device__ __forceinline__ uint32_t pixel_keys(const PlaneChunk<DPL, WIDE> (&v)[kMaxPaths], int nplanes,
                                               bool active, int x, int y, int W, int D, int li,
                                               uint32_t *key_right, uint16_t *dbg_sum) {
    constexpr int NR = DPL / 2;
    uint32_t S[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) S[k] = 0u;
#pragma unroll
    for (int q = 0; q < (NP > 0 ? NP : kMaxPaths); q++)
        if (NP > 0 || q < nplanes) {
            if constexpr (WIDE) {
#pragma unroll
                for (int k = 0; k < NR; k++) S[k] += v[q].w[k];  // stored as (d+k, d+k+h)
            } else {
#pragma unroll
                for (int w = 0; w < DPL / 4; w++) {
                    S[2 * w] += v[q].w[w] & kLo;
                    S[2 * w + 1] += __byte_perm(v[q].w[w], 0u, 0x4341);
                }
            }
        }
    const int d0 = DPL * li;
    const int m = visit_mask<DPL, LPS>(li);
    // T[k] = S[k ^ (m mod NR)], halves swapped when m has the bit NR
#pragma unroll
    for (int b = 1; b < NR; b <<= 1) {
        if (m & b) {
#pragma unroll
            for (int k = 0; k < NR; k++)
                if (!(k & b)) {
                    const uint32_t t = S[k];
                    S[k] = S[k | b];
                    S[k | b] = t;
                }
        }
    }
    if (m & NR) {
#pragma unroll
        for (int k = 0; k < NR; k++) S[k] = __byte_perm(S[k], S[k], 0x1032);
    }
    uint32_t best = 0xFFFFFFFFu;
    // every slot x - d of this lane lies in the row when x >= d0 + DPL - 1
    const bool inside = active && x >= d0 + DPL - 1;
#pragma unroll
    for (int j = 0; j < DPL; j++) {
        const int d = d0 + (j ^ m);
        const uint32_t sv = (j < NR) ? (S[j % NR] & 0xFFFFu) : (S[j % NR] >> 16);
        uint32_t key = sv * 256u + (uint32_t)d;
        if (RAGGED && d >= D) key = 0xFFFFFFFFu;
        best = min(best, key);
        if (inside) {
            if ((!RAGGED || d < D) && in_range(x - d, W)) atomicMin(&key_right[x - d], key);
        } else if (active && x - d >= 0 && (!RAGGED || d < D) && in_range(x - d, W)) {
            atomicMin(&key_right[x - d], key);
        }
        if (DEBUG && active && (!RAGGED || d < D)) dbg_sum[((size_t)y * W + x) * D + d] = (uint16_t)sv;
    }
    return best;
}

// PF: pixel groups whose planes are loaded ahead of the one being reduced (1
// or 2).  The HBM read rate of this kernel rises with the bytes in flight:
// two groups ahead took the 1242 x 375, D = 128 WTA from 87.5 to 81.4 us, but
// the extra registers leave 3 instead of 4 CTAs per SM, so the launcher takes
// PF = 2 only when that needs no more waves of rows.
template <int LPS, int DPL, bool WIDE, int NP, bool RAGGED, bool DEBUG, int PF>
__global__ void __launch_bounds__(kThreads, PF == 2 ? 2 : 1)
    wta_kernel(const uint8_t *__restrict__ planes, int nplanes, int W, int H,
               int D, int tol, uint8_t *__restrict__ disp_lr, uint8_t *__restrict__ dbg_left,
               uint8_t *__restrict__ dbg_right, uint16_t *__restrict__ dbg_sum) {
    wait_for_predecessor();
    constexpr int G = 32 / LPS;
    constexpr int Dp = DPL * LPS;
    constexpr int EB = WIDE ? 2 : 1;  // bytes per path cost
    constexpr int NQ = NP > 0 ? NP : kMaxPaths;
    extern __shared__ uint32_t smem[];
    uint32_t *key_right = smem;                                // W keys
    uint8_t *dl_row = reinterpret_cast<uint8_t *>(smem + W);  // W bytes
    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kThreads / 32;
    const int grp = lane / LPS, li = lane % LPS;
    for (int i = threadIdx.x; i < W; i += kThreads) key_right[i] = 0xFFFFFFFFu;
    __syncthreads();
    // pixel records hold all planes of a pixel back to back: nplanes * Dp * EB bytes
    const int np = NP > 0 ? NP : nplanes;
    const size_t rec = (size_t)np * Dp * EB;
    const uint8_t *row = planes + (size_t)y * W * rec + DPL * EB * li;
    const uint64_t pol = policy_evict_first();
    const int stride = nwarps * G;
    // byte offset of a lane's chunk from `planes`, and the last one that fits
    const long long row_off = (long long)y * W * (long long)rec + DPL * EB * li;
    const long long chunk_limit = (long long)W * H * (long long)rec - DPL * EB + 1;
    // software pipeline: the planes of the next PF pixel groups are loaded
    // while the current one is reduced (buf[0] is the current group)
    static_assert(PF == 1 || PF == 2, "one or two pixel groups ahead");
    PlaneChunk<DPL, WIDE> buf[PF + 1][kMaxPaths];
    int x = warp * G + grp;
#pragma unroll
    for (int b = 0; b <= PF; b++)
#pragma unroll
        for (int q = 0; q < kMaxPaths; q++)
#pragma unroll
            for (int w = 0; w < PlaneChunk<DPL, WIDE>::kWords; w++) buf[b][q].w[w] = 0u;
#pragma unroll
    for (int b = 0; b < PF; b++)
#pragma unroll
        for (int q = 0; q < NQ; q++)
            if ((NP > 0 || q < np) && x + b * stride < W &&
                in_range(row_off + (long long)(x + b * stride) * (long long)rec + q * Dp * EB, chunk_limit))
                buf[b][q] = ld_plane<DPL, WIDE>(row + (size_t)(x + b * stride) * rec + q * Dp * EB, pol);
    for (int xb = warp * G; xb < W; xb += stride) {
        const int xn = x + stride, xf = x + PF * stride;
#pragma unroll
        for (int q = 0; q < NQ; q++)
            if ((NP > 0 || q < np) && xf < W && in_range(row_off + (long long)xf * (long long)rec + q * Dp * EB, chunk_limit))
                buf[PF][q] = ld_plane<DPL, WIDE>(row + (size_t)xf * rec + q * Dp * EB, pol);
        const bool active = x < W;
        uint32_t best = pixel_keys<LPS, DPL, WIDE, NP, RAGGED, DEBUG>(buf[0], np, active, x, y, W, D, li, key_right, dbg_sum);
        best = group_min<LPS>(best, lane);
        if (li == 0 && active && in_range(x, W)) dl_row[x] = (uint8_t)(best & 0xFFu);
#pragma unroll
        for (int b = 0; b < PF; b++)
#pragma unroll
            for (int q = 0; q < NQ; q++) buf[b][q] = buf[b + 1][q];
        x = xn;
    }
    __syncthreads();
    for (int xx = threadIdx.x; xx < W; xx += kThreads) {
        const int dl = dl_row[xx];
        uint8_t v = (uint8_t)dl;
        if (tol >= 0) {
            const int xr = xx - dl;
            if (xr < 0 || !in_range(xr, W)) {
                v = SGM_INVALID;
            } else {
                const int dr = (int)(key_right[xr] & 0xFFu);
                const int diff = dl > dr ? dl - dr : dr - dl;
                if (diff > tol) v = SGM_INVALID;
            }
        }
        const size_t pix = (size_t)y * W + xx;
        if (!in_range((long long)pix, (long long)W * H)) continue;
        disp_lr[pix] = v;
        if (dbg_left) dbg_left[pix] = (uint8_t)dl;
        if (dbg_right) dbg_right[pix] = (uint8_t)(key_right[xx] & 0xFFu);
    }
}

// Launches one CTA per row of the PF = 2 variant when it needs no more waves
// of rows than PF = 1 (resident CTAs per SM from the occupancy calculator).
template <typename K1, typename K2>
cudaError_t launch_rows(K1 k1, K2 k2, int H, size_t smem, cudaStream_t s, const uint8_t *planes, int nplanes, int W,
                        int D, int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right, uint16_t *dbg_sum) {
    int dev = 0, sms = 0, n1 = 0, n2 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k1, kThreads, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, k2, kThreads, smem);
    if (e != cudaSuccess) return e;
    const long long c1 = (long long)n1 * sms, c2 = (long long)n2 * sms;
    const bool deep = c2 > 0 && c1 > 0 && (H + c2 - 1) / c2 <= (H + c1 - 1) / c1;
    if (deep)
        return launch_k(k2, dim3(H), dim3(kThreads), smem, s, planes, nplanes, W, H, D, tol, disp_lr, dbg_left,
                        dbg_right, dbg_sum);
    return launch_k(k1, dim3(H), dim3(kThreads), smem, s, planes, nplanes, W, H, D, tol, disp_lr, dbg_left, dbg_right,
                    dbg_sum);
}

template <bool WIDE>
cudaError_t launch_wta_t(const uint8_t *planes, int nplanes, int W, int H, int D, int tol, uint8_t *disp_lr,
                         uint8_t *dbg_left, uint8_t *dbg_right, uint16_t *dbg_sum, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
#define SGM_WTA4(L, N, R, G)                                                                                          \
    e = (G) ? launch_k(wta_kernel<L, 8, WIDE, N, R, G, 1>, dim3(H), dim3(kThreads), smem, s, planes, nplanes, W, H, D, \
                       tol, disp_lr, dbg_left, dbg_right, dbg_sum)                                                      \
            : launch_rows(wta_kernel<L, 8, WIDE, N, R, G, 1>, wta_kernel<L, 8, WIDE, N, R, G, 2>, H, smem, s, planes, \
                          nplanes, W, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum)
#define SGM_WTA(L)                                       \
    do {                                                 \
        const bool rag = D != 8 * (L);                   \
        if (dbg_sum) {                                   \
            if (rag) SGM_WTA4(L, 0, true, true);         \
            else SGM_WTA4(L, 0, false, true);            \
        } else if (nplanes == 8) {                       \
            if (rag) SGM_WTA4(L, 8, true, false);        \
            else SGM_WTA4(L, 8, false, false);           \
        } else if (nplanes == 4) {                       \
            if (rag) SGM_WTA4(L, 4, true, false);        \
            else SGM_WTA4(L, 4, false, false);           \
        } else {                                         \
            if (rag) SGM_WTA4(L, 0, true, false);        \
            else SGM_WTA4(L, 0, false, false);           \
        }                                                \
    } while (0)
    switch (lanes_per_scanline(D)) {
        case 1: SGM_WTA(1); break;
        case 2: SGM_WTA(2); break;
        case 4: SGM_WTA(4); break;
        case 8: SGM_WTA(8); break;
        case 16: SGM_WTA(16); break;
        default: SGM_WTA(32); break;
    }
#undef SGM_WTA4
#undef SGM_WTA
    return e;
}

}  // namespace

SGM_GUARD_COUNTER(guard_hits_wta)

cudaError_t launch_wta(const uint8_t *planes, int nplanes, int W, int H, int D, bool wide,
                       int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                       uint16_t *dbg_sum, cudaStream_t s) {
    if (disparities_per_lane(D) != 8) return cudaErrorInvalidValue;
    const size_t smem = (size_t)W * sizeof(uint32_t) + (size_t)((W + 3) & ~3);
    if (wide) return launch_wta_t<true>(planes, nplanes, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum, smem, s);
    return launch_wta_t<false>(planes, nplanes, W, H, D, tol, disp_lr, dbg_left, dbg_right, dbg_sum, smem, s);
}

}  // namespace sgm
