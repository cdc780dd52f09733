// Semi-global path aggregation (Sec. 3.1.3, Eq. 2) over a precomputed cost
// volume (Eq. 1).
//
// Decomposition.  Every enabled direction cuts the image into independent
// scanlines: rows for the horizontal directions, columns for the vertical
// ones and W+H-1 diagonals for each diagonal direction.  The D disparities of
// one pixel are held by LPS lanes, 8 disparities per lane, so one warp walks
// G = 32 / LPS neighbouring scanlines in lock-step (D = 128: two scanlines).
// The kernel is persistent: warps pull jobs (one direction, G scanlines)
// from a global counter, the longest scanlines first, until the list is
// exhausted; blocks_per_sm blocks of 4 warps run on every SM.  Two blocks
// (two warps per scheduler) measured fastest: the horizontal scanlines, the
// longest, set the kernel's duration, and each extra co-resident warp takes
// issue slots from them.
//
// Arithmetic.  A lane keeps its 8 path costs as four packed 16-bit pairs
// R_k = (L[k], L[k+4]), k = 0..3.  With this interleaving the d-1 / d+1
// neighbours of R1 and R2 are the registers R0/R2 and R1/R3 themselves, and
// those of R0 and R3 cost one byte-permute each with the value fetched from
// the neighbouring lane (one shuffle each way).  One update is
//     t = min(min(L(d-1), L(d+1)) + P1, L(d), m + P2);   L' = t + C - m
// evaluated two disparities at a time with the full-rate min.u16x2 and plain
// 32-bit adds (no half ever carries: values stay below 0x7FFF + 255, and
// t >= m makes t + C - m non-negative in each half).  m = min_d L is reduced
// within the lane (3 min.u16x2), then across the scanline's lanes with
// one full-warp redux.sync per scanline of the warp.
// Starting from L = 0, m = 0 makes the first step produce L = C without a
// special case.  Disparities d >= D (padding) are parked at 0x7FFF so they
// never win a minimum or act as a neighbour.
//
// Memory.  The cost of step t + PF is loaded while step t computes (a ring of
// PF = 16 8-byte registers), with an L2 evict_last hint: all directions
// re-read the volume; the line of step t + 32 is prefetched into L2 at step t.  Each step stores the lane's 8 path costs (8 bytes) to the
// direction's plane, in the cost volume's byte order, with evict_first: the
// planes are read back only once, by the WTA kernel.
#include "sgm_internal.cuh"

namespace sgm {

PathJobs make_path_jobs(int W, int H, int D, int mask) {
    PathJobs j = {};
    const int G = 32 / lanes_per_scanline(D);
    // long axis first, then the short axis, then the diagonals
    const bool wide = W >= H;
    const int order[kMaxPaths] = {wide ? 0 : 2, wide ? 1 : 3, wide ? 2 : 0, wide ? 3 : 1, 4, 5, 6, 7};
    for (int i = 0; i < kMaxPaths; i++) {
        const int r = order[i];
        if (!((mask >> r) & 1)) continue;
        const int k = j.n++;
        j.dx[k] = dir_dx(r);
        j.dy[k] = dir_dy(r);
        j.plane[k] = __builtin_popcount((unsigned)mask & ((1u << r) - 1u));
        j.nlines[k] = (int)scanlines_of(r, W, H);
        j.jbegin[k + 1] = j.jbegin[k] + (j.nlines[k] + G - 1) / G;
    }
    return j;
}

namespace {

constexpr int kWarps = 4;
constexpr int kL2Ahead = 32;  // steps between the L2 prefetch of a cost line and its use
constexpr uint32_t kInf2 = 0x7FFF7FFFu;
constexpr uint32_t kLo = 0x00FF00FFu;

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

// L2 policies: the cost volume is re-read by every direction and should stay
// in L2 (evict_last); the planes are written once and read back only by the
// WTA kernel, so they go first (evict_first).
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint2 ld_cost(const uint2 *p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void prefetch_l2(const uint2 *p) {
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p));
}
__device__ __forceinline__ void st_plane(uint2 *p, uint2 v, uint64_t pol) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x),
                 "r"(v.y), "l"(pol)
                 : "memory");
}

// (m, m) with m the minimum over the LPS lanes of this lane's scanline of
// both halves of x.  One full-warp redux.sync per scanline of the warp, each
// fed 0xFFFF by the lanes of the other scanlines (redux.sync with per-group
// masks measured 2.4x slower on GB300).
template <int LPS>
__device__ __forceinline__ uint32_t line_min2(uint32_t x, int grp) {
    constexpr int G = 32 / LPS;
    const uint32_t m32 = min(x & 0xFFFFu, x >> 16);
    uint32_t m;
    if constexpr (LPS == 1) {
        m = m32;
    } else if constexpr (G == 1) {
        m = __reduce_min_sync(0xffffffffu, m32);
    } else {
        m = 0;
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t r = __reduce_min_sync(0xffffffffu, grp == g ? m32 : 0xFFFFu);
            if (grp == g) m = r;
        }
    }
    return m * 0x00010001u;
}

// Path state of one lane: R_k = (L[k], L[k+4]) packed, m2 = (m, m), mP2 = m2 + (P2, P2).
struct PathState {
    uint32_t R0, R1, R2, R3, m2, mP2;
};

// One step of Eq. 2 for the lane's 8 disparities with cost chunk c.
template <int LPS, bool RAGGED>
__device__ __forceinline__ void path_step(PathState &st, uint2 c, uint32_t P1x2, uint32_t P2x2,
                                          int grp, uint32_t lo_edge, uint32_t hi_edge,
                                          const uint32_t (&inv)[4]) {
    // bytes (1, 3) of a word, zero-extended to 16-bit halves, in one byte-permute
    const uint32_t c0 = c.x & kLo, c1 = __byte_perm(c.x, 0u, 0x4341);
    const uint32_t c2 = c.y & kLo, c3 = __byte_perm(c.y, 0u, 0x4341);
    const uint32_t prev = __shfl_up_sync(0xffffffffu, st.R3, 1);
    const uint32_t next = __shfl_down_sync(0xffffffffu, st.R0, 1);
    // (L[-1], L[3]) and (L[4], L[8]); the first/last lane of a scanline ORs in
    // 0x7FFF for the missing neighbour (lo_edge / hi_edge are 0 elsewhere)
    const uint32_t dm0 = __byte_perm(prev, st.R3, 0x5432) | lo_edge;
    const uint32_t dp3 = __byte_perm(st.R0, next, 0x5432) | hi_edge;
    uint32_t n0 = vmin2(vmin2(vmin2(dm0, st.R1) + P1x2, st.R0), st.mP2) + c0 - st.m2;
    uint32_t n1 = vmin2(vmin2(vmin2(st.R0, st.R2) + P1x2, st.R1), st.mP2) + c1 - st.m2;
    uint32_t n2 = vmin2(vmin2(vmin2(st.R1, st.R3) + P1x2, st.R2), st.mP2) + c2 - st.m2;
    uint32_t n3 = vmin2(vmin2(vmin2(st.R2, dp3) + P1x2, st.R3), st.mP2) + c3 - st.m2;
    if (RAGGED) {
        n0 = vmax2(n0, inv[0]);
        n1 = vmax2(n1, inv[1]);
        n2 = vmax2(n2, inv[2]);
        n3 = vmax2(n3, inv[3]);
    }
    st.R0 = n0;
    st.R1 = n1;
    st.R2 = n2;
    st.R3 = n3;
    st.m2 = line_min2<LPS>(vmin2(vmin2(n0, n1), vmin2(n2, n3)), grp);
    st.mP2 = st.m2 + P2x2;
}

// The lane's 8 path costs as the plane's 8 bytes (cost-volume byte order).
template <bool RAGGED>
__device__ __forceinline__ uint2 pack_plane(const PathState &st) {
    uint32_t o0 = st.R0, o1 = st.R1, o2 = st.R2, o3 = st.R3;
    if (RAGGED) {
        o0 &= kLo;
        o1 &= kLo;
        o2 &= kLo;
        o3 &= kLo;
    }
    return make_uint2(o1 * 256u + o0, o3 * 256u + o2);
}

template <int LPS, bool RAGGED, int PF>
__global__ void __launch_bounds__(kWarps * 32)
    aggregate_kernel(const uint2 *__restrict__ cost, int W, int H, int D, uint32_t P1x2,
                     uint32_t P2x2, PathJobs jobs, uint2 *__restrict__ planes, int nplanes,
                     unsigned *__restrict__ job_counter) {
    constexpr int G = 32 / LPS;
    const int lane = threadIdx.x & 31;
    const int grp = lane / LPS, li = lane % LPS;
    const uint32_t lo_edge = li == 0 ? 0x7FFFu : 0u;              // no d = -1
    const uint32_t hi_edge = li == LPS - 1 ? 0x7FFF0000u : 0u;    // no d = Dp
    const int total = jobs.jbegin[jobs.n];
    const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();
    uint32_t inv[4] = {0u, 0u, 0u, 0u};
    if (RAGGED) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            inv[k] = (8 * li + k >= D ? 0x7FFFu : 0u) | (8 * li + k + 4 >= D ? 0x7FFF0000u : 0u);
    }
    for (;;) {
        unsigned job = 0;
        if (lane == 0) job = atomicAdd(job_counter, 1u);
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= (unsigned)total) return;
        int k = 0;
        while ((int)job >= jobs.jbegin[k + 1]) k++;
        const int s = ((int)job - jobs.jbegin[k]) * G + grp;
        const int dx = jobs.dx[k], dy = jobs.dy[k];
        int x = 0, y = 0, len = 0;
        if (s < jobs.nlines[k]) {
            if (dy == 0) {
                y = s;
                x = dx > 0 ? 0 : W - 1;
                len = W;
            } else if (dx == 0) {
                x = s;
                y = dy > 0 ? 0 : H - 1;
                len = H;
            } else if (s < W) {
                x = s;
                y = dy > 0 ? 0 : H - 1;
                len = min(dx > 0 ? W - s : s + 1, H);
            } else {
                const int tt = s - W + 1;
                x = dx > 0 ? 0 : W - 1;
                y = dy > 0 ? tt : H - 1 - tt;
                len = min(H - tt, W);
            }
        }
        const int steps = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
        // 8-byte-unit indices: cost chunk (x, y, li) is cost[(y*W + x)*LPS + li], plane
        // chunk is planes[((y*W + x)*nplanes + plane)*LPS + li] (all planes of a pixel
        // are adjacent).  Indices stay below 2^31 (checked when the handle is made).
        const int pix = y * W + x;
        const int cstep = (dy * W + dx) * LPS;
        const int ostep = cstep * nplanes;
        int ci_ld = pix * LPS + li;  // next cost chunk to load into the ring
        // one lane per 128-byte line of a pixel's cost record prefetches into L2
        const bool pf_lane = ((8 * li) & 127) == 0;
        int ci_pf = ci_ld;
        if (pf_lane)
            for (int i = 0; i < kL2Ahead && i < len; i++) prefetch_l2(cost + ci_pf + i * cstep);
        ci_pf += kL2Ahead * cstep;
        int oi = (pix * nplanes + jobs.plane[k]) * LPS + li;
        uint2 ring[PF];
#pragma unroll
        for (int i = 0; i < PF; i++) {
            ring[i] = i < len ? ld_cost(cost + ci_ld, pol_keep) : make_uint2(0u, 0u);
            ci_ld += cstep;
        }
        PathState st = {inv[0], inv[1], inv[2], inv[3], 0u, P2x2};
        int rem = len;  // steps of this lane's scanline not yet taken
        int t0 = 0;
        for (; t0 + PF <= steps; t0 += PF) {
#pragma unroll
            for (int i = 0; i < PF; i++) {
                const uint2 c = ring[i];
                if (rem > PF) ring[i] = ld_cost(cost + ci_ld, pol_keep);
                ci_ld += cstep;
                if (pf_lane && rem > kL2Ahead) prefetch_l2(cost + ci_pf);
                ci_pf += cstep;
                path_step<LPS, RAGGED>(st, c, P1x2, P2x2, grp, lo_edge, hi_edge, inv);
                if (rem > 0) st_plane(planes + oi, pack_plane<RAGGED>(st), pol_stream);
                oi += ostep;
                rem--;
            }
        }
#pragma unroll
        for (int i = 0; i < PF; i++) {  // the last steps < PF
            if (t0 + i < steps) {
                path_step<LPS, RAGGED>(st, ring[i], P1x2, P2x2, grp, lo_edge, hi_edge, inv);
                if (rem > 0) st_plane(planes + oi, pack_plane<RAGGED>(st), pol_stream);
                oi += ostep;
                rem--;
            }
        }
    }
}

template <int LPS>
cudaError_t launch_lps(const uint8_t *cost, int W, int H, int D, uint32_t P1x2, uint32_t P2x2,
                       const PathJobs &jobs, uint8_t *planes, int nplanes, unsigned *job_counter,
                       int blocks, cudaStream_t s) {
    constexpr int PF = 16;  // cost loads issued 16 steps ahead
    const uint2 *c = reinterpret_cast<const uint2 *>(cost);
    uint2 *p = reinterpret_cast<uint2 *>(planes);
    if (D == 8 * LPS)
        aggregate_kernel<LPS, false, PF><<<blocks, kWarps * 32, 0, s>>>(c, W, H, D, P1x2, P2x2, jobs, p, nplanes, job_counter);
    else
        aggregate_kernel<LPS, true, PF><<<blocks, kWarps * 32, 0, s>>>(c, W, H, D, P1x2, P2x2, jobs, p, nplanes, job_counter);
    return cudaGetLastError();
}

// Plane 0 ([H][W][Dp], lane-chunk byte order) -> L ([H][W][D], natural order).
__global__ void unpermute_kernel(const uint8_t *__restrict__ plane, int npx, int D, int Dp,
                                 uint8_t *__restrict__ L) {
    const size_t n = (size_t)npx * D;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / D;
        const int d = (int)(i - p * D);
        L[i] = plane[p * Dp + 8 * (d >> 3) + chunk_byte_of(d & 7)];
    }
}

}  // namespace

cudaError_t launch_aggregate(const uint8_t *cost, int W, int H, int D, int P1, int P2,
                             const PathJobs &jobs, uint8_t *planes, int nplanes,
                             unsigned *job_counter, int blocks_per_sm, cudaStream_t s) {
    if (jobs.jbegin[jobs.n] == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(job_counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (blocks_per_sm > 0 ? blocks_per_sm : 2);
    const uint32_t P1x2 = (uint32_t)P1 * 0x00010001u, P2x2 = (uint32_t)P2 * 0x00010001u;
    switch (lanes_per_scanline(D)) {
        case 1: return launch_lps<1>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
        case 2: return launch_lps<2>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
        case 4: return launch_lps<4>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
        case 8: return launch_lps<8>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
        case 16: return launch_lps<16>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
        default: return launch_lps<32>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
    }
}

cudaError_t launch_unpermute(const uint8_t *plane, int W, int H, int D, uint8_t *L, cudaStream_t s) {
    const int npx = W * H;
    const size_t n = (size_t)npx * D;
    const size_t want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    unpermute_kernel<<<blocks, 256, 0, s>>>(plane, npx, D, padded_disparities(D), L);
    return cudaGetLastError();
}

}  // namespace sgm
