// Semi-global path aggregation (Sec. 3.1.3, Eq. 2) over a precomputed cost
// volume (Eq. 1).
//
// Decomposition.  Every enabled direction cuts the image into independent
// scanlines: rows for the horizontal directions, columns for the vertical
// ones and W+H-1 diagonals for each diagonal direction.  The D disparities of
// one pixel are held by LPS lanes, DPL = 8 disparities per lane, so one warp
// walks G = 32 / LPS neighbouring scanlines in lock-step (D = 128: two
// scanlines of 16 lanes).  The kernel is persistent: blocks_per_sm blocks of
// 4 warps run on every SM and pull jobs (one direction, G scanlines) from a
// work queue until it is empty.  The long-axis scanlines (rows when W >= H)
// set the kernel's duration, and they run about 1.5x slower when two of them
// share a warp scheduler, so each scheduler takes at most one of them first
// (see next_job); the other warps fill the issue slots left with the
// remaining directions.  Three blocks per SM measured fastest on the
// 1242 x 375, D = 128 workload; sgm_autotune picks the count per shape.
//
// Arithmetic.  A lane keeps its DPL path costs as DPL/2 packed 16-bit pairs
// R_k = (L[k], L[k+h]), h = DPL/2.  With this interleaving the d-1 / d+1
// neighbours of the inner registers are the registers R_{k-1} / R_{k+1}
// themselves, and those of the first and last cost one byte-permute each
// with the value fetched from the neighbouring lane (one shuffle each way).
// One update is
//     t = min(min(L(d-1), L(d+1), m + P2 - P1) + P1, L(d));   L' = t + C - m
// (the same minimum as min(L(d±1) + P1, L(d), m + P2)), evaluated two
// disparities at a time with a three-way packed minimum, a packed
// add-then-minimum and a plain 32-bit three-input add (no half ever carries:
// values stay below 0x7FFF + 255, and t >= m makes t + C - m non-negative in
// each half).  m = min_d L is reduced
// within the lane (min.u16x2), then across the scanline's lanes: xor-shuffles
// for scanlines of up to 4 lanes, one full-warp redux.sync per scanline of
// the warp for wider ones (an xor-shuffle tree over 16 lanes measured 1.5x
// slower).  Starting from L = 0, m = 0 makes the first step produce L = C
// without a special case.  Disparities d >= D (padding) are parked at 0x7FFF
// so they never win a minimum or act as a neighbour.
//
// Pipes.  On GB300 the packed minima, the byte-permutes and the logic
// operations issue on the ALU pipe at 16 lanes per cycle, and that pipe
// bounds the kernel (29.6 of the 42.5 warp instructions of a step on the
// 1242 x 375, D = 128 workload, 8.1 on the FMA pipe).  The adds that need no
// three inputs are therefore written as multiply-adds by a 1 the compiler
// cannot see (the job table's unit field), which run on the FMA pipe: the
// edge markers, m + P2 - P1, the biased inputs of the cross-lane minimum, the
// even cost bytes (v - odd * 256) and the plane bytes (hi * 256 + lo).  That
// moved 6 instructions a step (23.6 ALU, 14.0 FMA) and measured 4-6 % faster;
// moving the three-input adds as well (two multiply-adds each) balanced the
// pipes (20.1 / 21.4) but ran slower.  Without any memory access the kernel
// still takes 135 of its 157 us: the step-to-step chain (lane minimum,
// cross-lane minimum, next update) bounds it, not HBM, and capping registers
// for more resident warps (5, 6 or 8 blocks per SM) made that chain slower.
//
// Measured and rejected on GB300: 16 disparities per lane (15 % fewer
// instructions, but the fatter long-axis warps lengthen the critical path);
// taking the next minimum from the previous step's costs, which moves the
// reduction off the step-to-step chain (15 % more instructions, slower); a
// 24-step cost ring; an L2 prefetch of the cost line 32 steps ahead and an
// evict_last hint on the cost loads (together 9 % slower: the cost volume
// is re-read from DRAM either way, and the extra requests compete with it);
// cost loads that bypass L1 (L1::no_allocate: 12 % slower, .cg: 6 %).
//
// Memory.  The cost of step t + PF is loaded while step t computes (a ring of
// PF lane chunks: 16 of 8 bytes for 8-bit costs, 8 of 16 bytes for the
// 16-bit costs of SAD).  While every scanline of the warp has at least 2 * PF
// steps left the loop runs without bounds checks.  Each step stores the
// lane's DPL path costs to the direction's plane, in the cost volume's order
// and width, with evict_first: the planes are read back only once, by the
// WTA kernel.  16-bit path costs run through the same packed arithmetic: the
// host keeps cmax + P2 below the 0x7FFF padding marker.

#include "sgm_internal.cuh"

namespace sgm {

PathJobs make_path_jobs_mixed(int W, int H, int D, int mask, int cpl_long, int cpl_other) {
    PathJobs j = {};
    j.unit = 1u;
    // long axis first, then the short axis, then the diagonals
    const bool wide = W >= H;
    const int order[kMaxPaths] = {wide ? 0 : 2, wide ? 1 : 3, wide ? 2 : 0, wide ? 3 : 1, 4, 5, 6, 7};
    for (int i = 0; i < kMaxPaths; i++) {
        const int r = order[i];
        if (!((mask >> r) & 1)) continue;
        const int k = j.n++;
        j.cpl[k] = i < 2 ? cpl_long : cpl_other;
        const int G = 32 / (lanes_per_scanline(D) / j.cpl[k]);
        j.dx[k] = dir_dx(r);
        j.dy[k] = dir_dy(r);
        j.plane[k] = __builtin_popcount((unsigned)mask & ((1u << r) - 1u));
        j.nlines[k] = (int)scanlines_of(r, W, H);
        j.jbegin[k + 1] = j.jbegin[k] + (j.nlines[k] + G - 1) / G;
        if (i < 2) j.nlong = j.jbegin[k + 1];
    }
    return j;
}

PathJobs make_path_jobs(int W, int H, int D, int mask, int cpl) { return make_path_jobs_mixed(W, H, D, mask, cpl, cpl); }

namespace {

constexpr int kWarps = 4;
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
// a * b + c on the FMA pipe.  With b = `one`, a 1 the compiler cannot see
// (PathJobs::unit), it is an add that stays off the ALU pipe.
__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// The planes are written once and read back only by the WTA kernel, so they
// leave L2 first (evict_first).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Job scheduling.  The long-axis scanlines (rows when W >= H) set the
// kernel's duration: one of them takes about 145 cycles per step on a warp
// scheduler of its own and much longer when two share a scheduler.  So the
// first warp on each (SM, scheduler) slot that claims the slot takes a
// long-axis job, the other warps start on the remaining directions, and after
// its first job every warp drains the long-axis jobs first.  The slot comes
// from %smid and %warpid (warp slot modulo the 4 schedulers): the placement
// only affects speed, never results.
__device__ __forceinline__ unsigned sched_slot() {
    unsigned w, sm;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(w));
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    return sm * 4u + (w & 3u);
}

__device__ __forceinline__ unsigned next_job(unsigned *state, unsigned nlong, unsigned total, bool first) {
    bool want_long = true;
    if (first) {
        const unsigned slot = sched_slot();
        want_long = slot < (unsigned)kJobClaimSlots && atomicExch(state + kJobClaimBase + slot, 1u) == 0u;
    }
    if (want_long) {
        const unsigned j = atomicAdd(state, 1u);
        if (j < nlong) return j;
        return nlong + atomicAdd(state + 1, 1u);
    }
    const unsigned j = nlong + atomicAdd(state + 1, 1u);
    if (j < total) return j;
    const unsigned jl = atomicAdd(state, 1u);
    return jl < nlong ? jl : total;
}

// (m, m) with m the minimum over the LPS lanes of this lane's scanline of
// both halves of x.  The halves are folded first ((m, m) = m * 0x10001 is
// monotonic in m, so it can be reduced as one 32-bit value).  Scanlines of up
// to 4 lanes reduce with xor-shuffles; wider ones use one full-warp
// redux.sync per scanline of the warp, fed x + 0x80008000 by the other
// scanlines' lanes, more than any (m, m) with m <= 0x7FFF (redux.sync with
// per-scanline masks measured 2.4x slower on GB300).
template <int LPS>
__device__ __forceinline__ uint32_t line_min2(uint32_t x, int grp, uint32_t one) {
    constexpr int G = 32 / LPS;
    x = vmin2(x, __byte_perm(x, 0u, 0x1032));
    if constexpr (LPS <= 4) {
#pragma unroll
        for (int o = 1; o < LPS; o <<= 1) x = vmin2(x, __shfl_xor_sync(0xffffffffu, x, o));
        return x;
    } else if constexpr (G == 1) {
        return __reduce_min_sync(0xffffffffu, x);
    } else if constexpr (G == 2) {
        const uint32_t r0 = __reduce_min_sync(0xffffffffu, mad(x, one, grp == 0 ? 0u : 0x80008000u));
        const uint32_t r1 = __reduce_min_sync(0xffffffffu, mad(x, one, grp == 1 ? 0u : 0x80008000u));
        return grp ? r1 : r0;
    } else {
        uint32_t m = 0;
#pragma unroll
        for (int g = 0; g < G; g++) {
            const uint32_t r = __reduce_min_sync(0xffffffffu, mad(x, one, grp == g ? 0u : 0x80008000u));
            if (grp == g) m = r;
        }
        return m;
    }
}

// The CPL consecutive 8-disparity chunks one lane holds, as they sit in the
// cost volume and the planes: 8 bytes per chunk for 8-bit costs, 16 for the
// 16-bit costs of SAD.
template <int CPL, bool WIDE>
struct Blk {
    static constexpr int kWords = CPL * (WIDE ? 4 : 2);
    static_assert(kWords == 2 || kWords % 4 == 0, "a lane block is 8 bytes or whole 16-byte vectors");
    uint32_t w[kWords];
};

template <int CPL, bool WIDE>
__device__ __forceinline__ Blk<CPL, WIDE> ld_blk(const Blk<CPL, WIDE> *p) {
    Blk<CPL, WIDE> v;
    if constexpr (Blk<CPL, WIDE>::kWords == 2) {
        asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.w[0]), "=r"(v.w[1]) : "l"(p));
    } else {
#pragma unroll
        for (int q = 0; q < Blk<CPL, WIDE>::kWords; q += 4)
            asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.w[q]), "=r"(v.w[q + 1]), "=r"(v.w[q + 2]), "=r"(v.w[q + 3])
                         : "l"(reinterpret_cast<const uint32_t *>(p) + q));
    }
    return v;
}
template <int CPL, bool WIDE>
__device__ __forceinline__ void st_blk(Blk<CPL, WIDE> *p, const Blk<CPL, WIDE> &v, uint64_t pol) {
    if constexpr (Blk<CPL, WIDE>::kWords == 2) {
        asm volatile("st.global.L1::no_allocate.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.w[0]),
                     "r"(v.w[1]), "l"(pol)
                     : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < Blk<CPL, WIDE>::kWords; q += 4)
            asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(
                             reinterpret_cast<uint32_t *>(p) + q),
                         "r"(v.w[q]), "r"(v.w[q + 1]), "r"(v.w[q + 2]), "r"(v.w[q + 3]), "l"(pol)
                         : "memory");
    }
}

// Cost blocks loaded PF steps ahead: 16 for 8-byte blocks, 8 for 16- and 32-byte ones.
template <int CPL, bool WIDE>
constexpr int prefetch_depth() {
    return Blk<CPL, WIDE>::kWords == 2 ? 16 : 8;
}

// Path state of one lane: chunk c holds R[c][k] = (L[d_c+k], L[d_c+k+4]) packed
// (d_c its first disparity), m2 = (m, m), mQ = m2 + (P2 - P1, P2 - P1).
template <int CPL>
struct PathState {
    uint32_t R[CPL][4];
    uint32_t m2, mQ;
};

// One step of Eq. 2 for the lane's CPL chunks with cost block b.  Inside a
// chunk the d-1 / d+1 neighbours of the inner words are the neighbouring
// words; the first and last words take their outer neighbour from the
// previous / next chunk, which is in the same lane except at the lane's ends
// (one shuffle each way per step, whatever CPL is).
template <int LPS, int CPL, bool WIDE, bool RAGGED>
__device__ __forceinline__ void path_step(PathState<CPL> &st, const Blk<CPL, WIDE> &b, uint32_t P1x2,
                                          uint32_t QPx2, int grp, uint32_t lo_edge, uint32_t hi_edge,
                                          const uint32_t (&inv)[CPL][4], uint32_t one, uint32_t neg256) {
    uint32_t cc[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        if constexpr (WIDE) {
#pragma unroll
            for (int k = 0; k < 4; k++) cc[c][k] = b.w[4 * c + k];  // (C[k], C[k+4]) as stored
        } else {
#pragma unroll
            for (int w = 0; w < 2; w++) {
                const uint32_t v = b.w[2 * c + w];
                cc[c][2 * w + 1] = __byte_perm(v, 0u, 0x4341);     // bytes 1, 3
                cc[c][2 * w] = mad(cc[c][2 * w + 1], neg256, v);  // bytes 0, 2: v - (bytes 1, 3) * 256
            }
        }
    }
    const uint32_t prev = __shfl_up_sync(0xffffffffu, st.R[CPL - 1][3], 1);
    const uint32_t next = __shfl_down_sync(0xffffffffu, st.R[0][0], 1);
    uint32_t n[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        // (L[d_c-1], L[d_c+3]) and (L[d_c+4], L[d_c+8]); the first/last lane of a
        // scanline adds 0x7FFF to the missing neighbour (lo_edge / hi_edge are 0
        // elsewhere), which lifts it to >= 0x7FFF without a carry out of its
        // half.  That needs every lane's values <= 0x7FFF, the neighbour lane's
        // too when its scanline does not exist or has ended: such lanes run on
        // zeroed or real cost blocks (run_job), never on uninitialised memory.
        uint32_t dm0 = __byte_perm(c == 0 ? prev : st.R[c - 1][3], st.R[c][3], 0x5432);
        if (c == 0) dm0 = mad(lo_edge, one, dm0);
        uint32_t dpN = __byte_perm(st.R[c][0], c == CPL - 1 ? next : st.R[c + 1][0], 0x5432);
        if (c == CPL - 1) dpN = mad(hi_edge, one, dpN);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t lm = k == 0 ? dm0 : st.R[c][k - 1];
            const uint32_t rm = k == 3 ? dpN : st.R[c][k + 1];
            // min(L(d-1) + P1, L(d+1) + P1, m + P2, L(d)) as min(min(L(d-1), L(d+1),
            // m + P2 - P1) + P1, L(d)): a three-way packed minimum and a packed
            // add-then-minimum (the dynamic-programming instructions of sm_90+);
            // no half wraps, as every value stays below 0x7FFF + P1
            n[c][k] = __viaddmin_u16x2(__vimin3_u16x2(lm, rm, st.mQ), P1x2, st.R[c][k]) + cc[c][k] - st.m2;
            if (RAGGED) n[c][k] = vmax2(n[c][k], inv[c][k]);
        }
    }
    // lane minimum: three-way minima over the lane's words
    uint32_t mc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; c++) mc[c] = vmin2(__vimin3_u16x2(n[c][0], n[c][1], n[c][2]), n[c][3]);
    uint32_t mn = mc[0];
#pragma unroll
    for (int c = 1; c < CPL; c += 2) mn = c + 1 < CPL ? __vimin3_u16x2(mn, mc[c], mc[c + 1]) : vmin2(mn, mc[c]);
#pragma unroll
    for (int c = 0; c < CPL; c++)
#pragma unroll
        for (int k = 0; k < 4; k++) st.R[c][k] = n[c][k];
    st.m2 = line_min2<LPS>(mn, grp, one);
    st.mQ = mad(st.m2, one, QPx2);
}

// The lane's path costs in the cost volume's order.  Padding slots (0x7FFF)
// are stored as their low byte (8-bit) or as 0 (16-bit), so that sums over
// the planes never carry out of a 16-bit half; no WTA key uses them.
template <int CPL, bool WIDE, bool RAGGED>
__device__ __forceinline__ Blk<CPL, WIDE> pack_plane(const PathState<CPL> &st, const uint32_t (&inv)[CPL][4],
                                                     uint32_t c256) {
    Blk<CPL, WIDE> b;
#pragma unroll
    for (int c = 0; c < CPL; c++) {
        if constexpr (WIDE) {
#pragma unroll
            for (int k = 0; k < 4; k++) b.w[4 * c + k] = RAGGED ? st.R[c][k] & ~inv[c][k] : st.R[c][k];
        } else {
#pragma unroll
            for (int i = 0; i < 2; i++) {
                uint32_t lo = st.R[c][2 * i], hi = st.R[c][2 * i + 1];
                if (RAGGED) {
                    lo &= kLo;
                    hi &= kLo;
                }
                b.w[2 * c + i] = mad(hi, c256, lo);
            }
        }
    }
    return b;
}

// One job: the G neighbouring scanlines s0 .. s0+G-1 of one direction
// (dx, dy), scanline s0 + grp for this lane's group, written to plane
// `plane` of `nplanes`.  A scanline's pixel holds LPS lane blocks of CPL
// chunks each.
template <int LPS, int CPL, bool WIDE, bool RAGGED, int PF>
__device__ __forceinline__ void run_job(const Blk<CPL, WIDE> *__restrict__ cost, Blk<CPL, WIDE> *__restrict__ planes,
                                        int W, int H, int D, int nplanes, int dx, int dy, int plane, int nlines,
                                        int s0, uint32_t P1x2, uint32_t P2x2, uint64_t pol_stream, uint32_t one) {
    using BT = Blk<CPL, WIDE>;
    const int lane = threadIdx.x & 31;
    const uint32_t neg256 = one * 0xFFFFFF00u, c256 = one * 256u;
    const int grp = lane / LPS, li = lane % LPS;
    const uint32_t lo_edge = li == 0 ? 0x7FFFu : 0u;            // no d = -1
    const uint32_t hi_edge = li == LPS - 1 ? 0x7FFF0000u : 0u;  // no d = Dp
    uint32_t inv[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; c++)
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int d = (li * CPL + c) * 8 + k;
            inv[c][k] = RAGGED ? ((d >= D ? 0x7FFFu : 0u) | (d + 4 >= D ? 0x7FFF0000u : 0u)) : 0u;
        }
    const int s = s0 + grp;
    int x = 0, y = 0, len = 0;
    if (s < nlines) {
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
    // block indices: cost block (x, y, li) is cost[(y*W + x)*LPS + li], plane
    // block is planes[((y*W + x)*nplanes + plane)*LPS + li] (all planes of a
    // pixel are adjacent).  Indices stay below 2^31 (checked at handle creation).
    const int pix = y * W + x;
    const int cstep = (dy * W + dx) * LPS;
    const int ostep = cstep * nplanes;
    int ci_ld = pix * LPS + li;  // next cost block to load into the ring
    int oi = (pix * nplanes + plane) * LPS + li;
    // extents in blocks (guarded builds check every index against them)
    const long long cost_blocks = (long long)W * H * LPS, plane_blocks = cost_blocks * nplanes;
    BT ring[PF];
#pragma unroll
    for (int i = 0; i < PF; i++) {
        if (i < len && in_range(ci_ld, cost_blocks)) {
            ring[i] = ld_blk(cost + ci_ld);
        } else {  // zeros, so that lanes without a scanline keep bounded values
#pragma unroll
            for (int q = 0; q < BT::kWords; q++) ring[i].w[q] = 0u;
        }
        ci_ld += cstep;
    }
    PathState<CPL> st;
#pragma unroll
    for (int c = 0; c < CPL; c++)
#pragma unroll
        for (int k = 0; k < 4; k++) st.R[c][k] = inv[c][k];
    st.m2 = 0u;
    st.mQ = P2x2 - P1x2;
    const uint32_t QPx2 = P2x2 - P1x2;
    int rem = len;  // steps of this lane's scanline not yet taken
    int t0 = 0;
    // While every scanline of the warp has at least 2 * PF steps left, the
    // loads and stores need no checks.
    const int minlen = (int)__reduce_min_sync(0xffffffffu, (unsigned)len);
    for (; t0 + 2 * PF <= minlen; t0 += PF) {
#pragma unroll
        for (int i = 0; i < PF; i++) {
            const BT c = ring[i];
            if (in_range(ci_ld, cost_blocks)) ring[i] = ld_blk(cost + ci_ld);
            ci_ld += cstep;
            path_step<LPS, CPL, WIDE, RAGGED>(st, c, P1x2, QPx2, grp, lo_edge, hi_edge, inv, one, neg256);
            if (in_range(oi, plane_blocks)) st_blk(planes + oi, pack_plane<CPL, WIDE, RAGGED>(st, inv, c256), pol_stream);
            oi += ostep;
        }
        rem -= PF;
    }
    for (; t0 + PF <= steps; t0 += PF) {
#pragma unroll
        for (int i = 0; i < PF; i++) {
            const BT c = ring[i];
            if (rem > PF && in_range(ci_ld, cost_blocks)) ring[i] = ld_blk(cost + ci_ld);
            ci_ld += cstep;
            path_step<LPS, CPL, WIDE, RAGGED>(st, c, P1x2, QPx2, grp, lo_edge, hi_edge, inv, one, neg256);
            if (rem > 0 && in_range(oi, plane_blocks))
                st_blk(planes + oi, pack_plane<CPL, WIDE, RAGGED>(st, inv, c256), pol_stream);
            oi += ostep;
            rem--;
        }
    }
#pragma unroll
    for (int i = 0; i < PF; i++) {  // the last steps < PF
        if (t0 + i < steps) {
            path_step<LPS, CPL, WIDE, RAGGED>(st, ring[i], P1x2, QPx2, grp, lo_edge, hi_edge, inv, one, neg256);
            if (rem > 0 && in_range(oi, plane_blocks))
                st_blk(planes + oi, pack_plane<CPL, WIDE, RAGGED>(st, inv, c256), pol_stream);
            oi += ostep;
            rem--;
        }
    }
}

// CPL: chunks per lane of the jobs; with CPL2 > CPL, the entries whose
// jobs.cpl is CPL2 run with CPL2 chunks per lane (LPS * CPL / CPL2 lanes per
// scanline) and the others with CPL (same cost and plane layout either way).
template <int LPS, int CPL, bool WIDE, bool RAGGED, int PF, int CPL2 = CPL>
__global__ void __launch_bounds__(kWarps * 32)
    aggregate_kernel(const Blk<CPL, WIDE> *__restrict__ cost, int W, int H, int D, uint32_t P1x2, uint32_t P2x2,
                     PathJobs jobs, Blk<CPL, WIDE> *__restrict__ planes, int nplanes,
                     unsigned *__restrict__ job_counter) {
    wait_for_predecessor();
    const int lane = threadIdx.x & 31;
    const int total = jobs.jbegin[jobs.n];
    const uint64_t pol_stream = policy_evict_first();
    bool first = true;
    for (;;) {
        unsigned job = 0;
        if (lane == 0) job = next_job(job_counter, (unsigned)jobs.nlong, (unsigned)total, first);
        first = false;
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= (unsigned)total) return;
        int k = 0;
        while ((int)job >= jobs.jbegin[k + 1]) k++;
        if (CPL2 != CPL && jobs.cpl[k] == CPL2) {
            constexpr int L2 = LPS * CPL / CPL2 > 0 ? LPS * CPL / CPL2 : 1;
            using B2 = Blk<CPL2, WIDE>;
            run_job<L2, CPL2, WIDE, RAGGED, prefetch_depth<CPL2, WIDE>()>(
                reinterpret_cast<const B2 *>(cost), reinterpret_cast<B2 *>(planes), W, H, D, nplanes, jobs.dx[k],
                jobs.dy[k], jobs.plane[k], jobs.nlines[k], ((int)job - jobs.jbegin[k]) * (32 / L2), P1x2, P2x2,
                pol_stream, jobs.unit);
        } else {
            run_job<LPS, CPL, WIDE, RAGGED, PF>(cost, planes, W, H, D, nplanes, jobs.dx[k], jobs.dy[k], jobs.plane[k],
                                                jobs.nlines[k], ((int)job - jobs.jbegin[k]) * (32 / LPS), P1x2,
                                                P2x2, pol_stream, jobs.unit);
        }
    }
}

// Many pairs in one persistent launch.  The work list of pair p is its
// PathJobs; the two queues number all pairs' long-axis jobs (queue 0) and
// all their other jobs (queue 1) in pair order, pair p's starting at
// pfx[0][p] and pfx[1][p].  Each job runs with its pair's lanes per scanline.
template <int CPL, bool WIDE, int PF>
__global__ void __launch_bounds__(kWarps * 32)
    aggregate_batch_kernel(const BatchAggPair *__restrict__ pairs, int npairs, const int *__restrict__ prefix,
                           uint32_t P1x2, uint32_t P2x2, unsigned *__restrict__ job_counter) {
    wait_for_predecessor();
    extern __shared__ int spfx[];  // [2][npairs + 1]
    for (int i = threadIdx.x; i < 2 * (npairs + 1); i += blockDim.x) spfx[i] = prefix[i];
    __syncthreads();
    using BT = Blk<CPL, WIDE>;
    const int lane = threadIdx.x & 31;
    const int nlong = spfx[npairs], nother = spfx[npairs + 1 + npairs];
    const int total = nlong + nother;
    const uint64_t pol_stream = policy_evict_first();
    bool first = true;
    for (;;) {
        unsigned job = 0;
        if (lane == 0) job = next_job(job_counter, (unsigned)nlong, (unsigned)total, first);
        first = false;
        job = __shfl_sync(0xffffffffu, job, 0);
        if (job >= (unsigned)total) return;
        // the pair: binary search in the queue's prefix
        const bool lq = (int)job < nlong;
        const int *q = lq ? spfx : spfx + npairs + 1;
        const int jq = lq ? (int)job : (int)job - nlong;
        int lo = 0, hi = npairs;  // q[lo] <= jq < q[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (q[mid] <= jq) lo = mid;
            else hi = mid;
        }
        const BatchAggPair &p = pairs[lo];
        const int local = lq ? jq - q[lo] : p.jobs.nlong + (jq - q[lo]);
        int k = 0;
        while (local >= p.jobs.jbegin[k + 1]) k++;
        const int G = 32 / p.lps;
        const int s0 = (local - p.jobs.jbegin[k]) * G;
        const BT *cost = reinterpret_cast<const BT *>(p.cost);
        BT *planes = reinterpret_cast<BT *>(p.planes);
#define SGM_JOB(L, RG)                                                                                      \
    run_job<L, CPL, WIDE, RG, PF>(cost, planes, p.W, p.H, p.D, p.nplanes, p.jobs.dx[k], p.jobs.dy[k],       \
                                  p.jobs.plane[k], p.jobs.nlines[k], s0, P1x2, P2x2, pol_stream, p.jobs.unit)
#define SGM_JOB_L(L)              \
    if (p.ragged) SGM_JOB(L, true); \
    else SGM_JOB(L, false)
        switch (p.lps) {
            case 1: SGM_JOB_L(1); break;
            case 2: SGM_JOB_L(2); break;
            case 4: SGM_JOB_L(4); break;
            case 8: SGM_JOB_L(8); break;
            case 16: if (CPL <= 2) SGM_JOB_L(16); break;
            default: if (CPL == 1) SGM_JOB_L(32); break;
        }
#undef SGM_JOB_L
#undef SGM_JOB
    }
}

template <int LPS, int CPL, bool WIDE>
cudaError_t launch_lps(const uint8_t *cost, int W, int H, int D, uint32_t P1x2, uint32_t P2x2,
                       const PathJobs &jobs, uint8_t *planes, int nplanes, unsigned *job_counter,
                       int blocks, cudaStream_t s) {
    using BT = Blk<CPL, WIDE>;
    constexpr int PF = prefetch_depth<CPL, WIDE>();
    const BT *c = reinterpret_cast<const BT *>(cost);
    BT *p = reinterpret_cast<BT *>(planes);
    auto kernel = D == 8 * CPL * LPS ? aggregate_kernel<LPS, CPL, WIDE, false, PF>
                                     : aggregate_kernel<LPS, CPL, WIDE, true, PF>;
    return launch_k(kernel, dim3(blocks), dim3(kWarps * 32), 0, s, c, W, H, D, P1x2, P2x2, jobs, p, nplanes,
                    job_counter);
}

template <int CPL, bool WIDE>
cudaError_t launch_cpl(const uint8_t *cost, int W, int H, int D, uint32_t P1x2, uint32_t P2x2,
                       const PathJobs &jobs, uint8_t *planes, int nplanes, unsigned *job_counter,
                       int blocks, cudaStream_t s) {
#define SGM_AGG(L) launch_lps<L, CPL, WIDE>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s)
    switch (lanes_per_scanline(D) / CPL) {
        case 1: return SGM_AGG(1);
        case 2: return SGM_AGG(2);
        case 4: return SGM_AGG(4);
        case 8: return SGM_AGG(8);
        case 16: if constexpr (CPL <= 2) return SGM_AGG(16); else return cudaErrorInvalidValue;
        default: if constexpr (CPL == 1) return SGM_AGG(32); else return cudaErrorInvalidValue;
    }
#undef SGM_AGG
}

// Plane 0 ([H][W][Dp], lane-chunk order) -> L ([H][W][D] uint16, natural order).
__global__ void unpermute_kernel(const uint8_t *__restrict__ plane, int npx, int D, int Dp, int dpl,
                                 bool wide, uint16_t *__restrict__ L) {
    wait_for_predecessor();
    const size_t n = (size_t)npx * D;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / D;
        const int d = (int)(i - p * D), j = d % dpl;
        if (wide) {
            // word k of a chunk holds the pair (k, k + dpl/2) as two uint16
            const uint16_t *w = reinterpret_cast<const uint16_t *>(plane);
            L[i] = w[p * Dp + dpl * (d / dpl) + 2 * (j % (dpl / 2)) + j / (dpl / 2)];
        } else {
            L[i] = plane[p * Dp + dpl * (d / dpl) + chunk_byte(dpl, j)];
        }
    }
}

}  // namespace

// Rows (long-axis scanlines) at one chunk per lane, the other directions at two.
cudaError_t launch_mixed(const uint8_t *cost, int W, int H, int D, uint32_t P1x2, uint32_t P2x2, const PathJobs &jobs,
                         uint8_t *planes, int nplanes, unsigned *job_counter, int blocks, cudaStream_t s) {
    using BT = Blk<1, false>;
    const BT *c = reinterpret_cast<const BT *>(cost);
    BT *p = reinterpret_cast<BT *>(planes);
    const int L = lanes_per_scanline(D);
    const bool rag = D != 8 * L;
#define SGM_MIX(LL)                                                                                              \
    return launch_k(rag ? aggregate_kernel<LL, 1, false, true, 16, 2> : aggregate_kernel<LL, 1, false, false, 16, 2>, \
                    dim3(blocks), dim3(kWarps * 32), 0, s, c, W, H, D, P1x2, P2x2, jobs, p, nplanes, job_counter)
    switch (L) {
        case 2: SGM_MIX(2);
        case 4: SGM_MIX(4);
        case 8: SGM_MIX(8);
        case 16: SGM_MIX(16);
        case 32: SGM_MIX(32);
        default: return cudaErrorInvalidValue;
    }
#undef SGM_MIX
}

int chunks_per_lane_max(int D, bool wide) {
    const int chunks = lanes_per_scanline(D);  // 8-disparity chunks per pixel
    return wide ? 1 : (chunks >= 4 ? 4 : chunks);
}

cudaError_t launch_aggregate(const uint8_t *cost, int W, int H, int D, int P1, int P2, bool wide,
                             const PathJobs &jobs, uint8_t *planes, int nplanes,
                             unsigned *job_counter, int blocks_per_sm, int cpl, cudaStream_t s) {
    if (jobs.jbegin[jobs.n] == 0) return cudaSuccess;
    if (disparities_per_lane(D) != 8) return cudaErrorInvalidValue;
    if (cpl != 1 && cpl != 2 && cpl != 4 && cpl != kMixedCpl) return cudaErrorInvalidValue;
    if ((cpl == kMixedCpl ? 2 : cpl) > chunks_per_lane_max(D, wide)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (blocks_per_sm > 0 ? blocks_per_sm : 2);
    const uint32_t P1x2 = (uint32_t)P1 * 0x00010001u, P2x2 = (uint32_t)P2 * 0x00010001u;
    if (wide) return launch_cpl<1, true>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
    if (cpl == kMixedCpl) return launch_mixed(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
    if (cpl == 4) return launch_cpl<4, false>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
    if (cpl == 2) return launch_cpl<2, false>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
    return launch_cpl<1, false>(cost, W, H, D, P1x2, P2x2, jobs, planes, nplanes, job_counter, blocks, s);
}

cudaError_t launch_aggregate_batch(const BatchAggPair *pairs, int npairs, const int *prefix, int P1, int P2,
                                   bool wide, int cpl, unsigned *job_counter, int blocks_per_sm, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (blocks_per_sm > 0 ? blocks_per_sm : 2);
    const uint32_t P1x2 = (uint32_t)P1 * 0x00010001u, P2x2 = (uint32_t)P2 * 0x00010001u;
    const size_t smem = sizeof(int) * 2 * (size_t)(npairs + 1);
    if (wide)
        return launch_k(aggregate_batch_kernel<1, true, prefetch_depth<1, true>()>, dim3(blocks), dim3(kWarps * 32),
                        smem, s, pairs, npairs, prefix, P1x2, P2x2, job_counter);
    if (cpl == 4)
        return launch_k(aggregate_batch_kernel<4, false, prefetch_depth<4, false>()>, dim3(blocks), dim3(kWarps * 32),
                        smem, s, pairs, npairs, prefix, P1x2, P2x2, job_counter);
    return launch_k(aggregate_batch_kernel<1, false, prefetch_depth<1, false>()>, dim3(blocks), dim3(kWarps * 32),
                    smem, s, pairs, npairs, prefix, P1x2, P2x2, job_counter);
}

SGM_GUARD_COUNTER(guard_hits_aggregate)

cudaError_t launch_unpermute(const uint8_t *plane, int W, int H, int D, bool wide, uint16_t *L,
                             cudaStream_t s) {
    const int npx = W * H;
    const size_t n = (size_t)npx * D;
    const size_t want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    unpermute_kernel<<<blocks, 256, 0, s>>>(plane, npx, D, padded_disparities(D), disparities_per_lane(D),
                                            wide, L);
    return cudaGetLastError();
}

}  // namespace sgm
