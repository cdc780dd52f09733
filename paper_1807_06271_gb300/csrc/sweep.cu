// The paper's streaming aggregation (Sec. 3.1.3, Fig. 2): the 0, 45, 90 and
// 135 degree paths are all causal in one top-down pass over the image, so
// the matching cost (Eq. 1), the four path recurrences (Eq. 2), the sum S,
// the left winner, the right winner taken from the same S (Sec. 3.1.4) and
// the left-right check run in a single sweep.  Neither the cost volume, nor a
// path plane, nor S is ever written to memory: the kernel reads the two
// census code images and writes the checked disparity map (and, on request,
// the raw left and right maps).
//
// Decomposition.  One warp walks one image row from left to right, one pixel
// per step, with the D disparities of the pixel over its 32 lanes (DPL = 2 or
// 4 per lane, packed as 16-bit pairs; D <= 128).  In sweep terms the paths
// of pixel (x, y) continue from
//   H  (x-1, y)   the row itself (0 degrees, L->R), kept in registers;
//   V  (x, y-1)   90 degrees (T->B),
//   DL (x-1, y-1) 45 degrees (TL->BR),
//   DR (x+1, y-1) 135 degrees (TR->BL),
// so the warp of row y+1 runs behind the warp of row y and reads the three
// path vectors (and their minima) that row y leaves for it in a ring buffer:
// at least 2 pixels behind when DR is enabled, 1 when V is, 0 for DL alone.
// Consecutive rows of one CTA hand over through shared memory; the first row
// of a CTA reads the last row of the previous CTA from a ring in global
// memory, fetched kLandAhead pixels ahead with cp.async into a shared landing
// ring.  Every wait is bounded: after about a second it records a timeout in
// the handle's status word, raises the launch's abort word (which ends every
// other wait at once) and the warp returns; the launch is cooperative, so all
// CTAs are resident at once.
//
// Arithmetic per step and lane (DPL disparities d0 .. d0+DPL-1, d0 = DPL*lane):
//   C(d)  = popc(codeL(x) ^ codeR(x - d)), the code bits where x - d < 0; the
//           right codes slide through the lanes (one shuffle per step);
//   L'(d) = C(d) + min(L(d), min(L(d-1), L(d+1)) + P1, m + P2) - m  per path,
//           min.u16x2 and plain adds as in the aggregation kernel;
//   S     = sum of the enabled paths' L'; key(d) = (S << 8) | d;
//   left winner  = min key over the row's lanes (redux.sync), ties to small d;
//   right winner of x' = min over d of key(x' + d, d): a conveyor
//           T_d(x) = min(T_{d-1}(x-1), key(x, d)) moves one disparity per
//           step, and T_{D-1}(x) is final for x' = x - (D-1).
// After the row the warp applies the LR check (Sec. 3.1.4) to its row.
#include <atomic>

#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSlots = 8;       // slots of a ring between two rows of one CTA
constexpr int kLandSlots = 16;  // slots of the landing ring of a CTA's first row
constexpr int kLandAhead = 8;   // pixels fetched ahead from the global ring
constexpr int kGSlots = 64;     // slots of a global ring between two CTAs
constexpr int kPub = 4;         // a global ring's counters move every kPub pixels
constexpr unsigned long long kWaitNs = 1000000000ull;  // bounded waits: one second
constexpr unsigned long long kStallTestNs = 2000000ull;  // the stalled-wait test gives up after 2 ms

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
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(uint32_t *p, uint32_t v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// 16-byte copy global -> shared that bypasses L1 (.cg): the global rings are
// rewritten every kGSlots pixels, so a copy must never see a stale L1 line.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One hand-over ring between row y (producer) and row y+1 (consumer).  Slot
// s (pixel s mod SLOTS) holds, per lane, the N words of the V path of pixel
// s, of the DL path of pixel s-1 and of the DR path of pixel s+1 (the
// producer writes them one step apart so that the consumer of pixel s finds
// all three in slot s), and the three paths' packed minima (m, m).  A lane's
// words sit in 16-byte chunks, chunk-major so that lanes are 16 bytes apart:
// N = 1: chunk 0 = (V, DL, DR, -); N = 2: chunk 0 = (V, V, DL, DL), chunk 1 =
// (DR, DR, -, -).
template <int N, int SLOTS>
struct Ring {
    static constexpr int kChunks = N == 1 ? 1 : 2;
    uint32_t w[SLOTS][kChunks][32][4];
    uint32_t m[SLOTS][4];
};
// Word 0 of path p (0 = V, 1 = DL, 2 = DR) of `lane` in slot `slot`.
template <int N, typename RingT>
__device__ __forceinline__ uint32_t *ring_words(RingT *r, int slot, int p, int lane) {
    if constexpr (N == 1) return &r->w[slot][0][lane][p];
    else return p < 2 ? &r->w[slot][0][lane][2 * p] : &r->w[slot][1][lane][0];
}
template <int N, typename RingT>
__device__ __forceinline__ const uint32_t *ring_words(const RingT *r, int slot, int p, int lane) {
    return ring_words<N>(const_cast<RingT *>(r), slot, p, lane);
}
// Copies slot gs of global ring g into slot ls of the landing ring (every lane its chunks, lane 0 the minima).
template <int N, typename LandT, typename GT>
__device__ __forceinline__ void fetch_slot(LandT *land, int ls, const GT *g, int gs, int lane) {
#pragma unroll
    for (int c = 0; c < LandT::kChunks; c++) cp_async16(&land->w[ls][c][lane][0], &g->w[gs][c][lane][0]);
    if (lane == 0) cp_async16(&land->m[ls][0], &g->m[gs][0]);
}

struct SweepArgs {
    const void *codes;      // [2][H][W] census codes, left then right
    int W, H, D;
    uint32_t nbits;         // code bits: the cost where x - d < 0
    uint32_t P1x2, P2x2;    // penalties as packed pairs
    int flags;              // kSweep* bits of the enabled paths
    int tol;                // LR tolerance, < 0: off
    int rows_per_cta;
    uint8_t *disp_lr;       // [H][W] out: the checked map (holds the left map during the row)
    uint8_t *dr_map;        // [H][W] scratch/out: the right map
    uint8_t *dbg_left;      // [H][W] optional copy of the left map
    void *grings;           // one global ring per CTA boundary (index = consumer CTA)
    uint32_t *gprog;        // [2 * (nctas + 1)]: producer progress, consumer progress per boundary,
                            // then the grid's abort word (all zeroed before the launch)
    uint32_t *status;       // device status word (SGM_ERR_TIMEOUT record), may be null
    unsigned long long wait_ns;  // how long a wait may take before it gives up
    int stall_row;          // test of the bounded waits: this row waits for a pixel
                            // the row above never publishes (-1: none)
};

constexpr int kSweepH = 1, kSweepV = 2, kSweepDL = 4, kSweepDR = 8;
constexpr uint32_t kSweepTimeout = 2u;  // bit set in the status word when a wait gave up

// min(L(d-1), L(d+1)) of the lane's words; the first and last lanes see
// 0x7FFF for the missing neighbour (lo_edge / hi_edge).
template <int N>
__device__ __forceinline__ void nbr_min(const uint32_t (&w)[N], uint32_t (&nm)[N], uint32_t lo_edge, uint32_t hi_edge) {
    if constexpr (N == 1) {
        // w = (L[2l], L[2l+1])
        const uint32_t prev = __shfl_up_sync(kFull, w[0], 1);
        const uint32_t next = __shfl_down_sync(kFull, w[0], 1);
        const uint32_t left = __byte_perm(prev, w[0], 0x5432) | lo_edge;   // (L[2l-1], L[2l])
        const uint32_t right = __byte_perm(w[0], next, 0x5432) | hi_edge;  // (L[2l+1], L[2l+2])
        nm[0] = vmin2(left, right);
    } else {
        // A = w[0] = (L[4l], L[4l+2]), B = w[1] = (L[4l+1], L[4l+3])
        const uint32_t prevB = __shfl_up_sync(kFull, w[1], 1);
        const uint32_t nextA = __shfl_down_sync(kFull, w[0], 1);
        const uint32_t a_left = __byte_perm(prevB, w[1], 0x5432) | lo_edge;  // (L[4l-1], L[4l+1])
        const uint32_t b_right = __byte_perm(w[0], nextA, 0x5432) | hi_edge; // (L[4l+2], L[4l+4])
        nm[0] = vmin2(a_left, w[1]);
        nm[1] = vmin2(w[0], b_right);
    }
}

// One step of Eq. 2 for the lane's disparities: out = C + min(in, nbr + P1, m + P2) - m.
template <int N, bool RAGGED>
__device__ __forceinline__ void path_update(const uint32_t (&in)[N], uint32_t m2, uint32_t mP2, const uint32_t (&c)[N],
                                            uint32_t P1x2, uint32_t lo_edge, uint32_t hi_edge,
                                            const uint32_t (&inv)[N], uint32_t (&out)[N]) {
    uint32_t nm[N];
    nbr_min<N>(in, nm, lo_edge, hi_edge);
#pragma unroll
    for (int k = 0; k < N; k++) {
        const uint32_t t = vmin2(vmin2(nm[k] + P1x2, in[k]), mP2);
        out[k] = t + c[k] - m2;
        if (RAGGED) out[k] = vmax2(out[k], inv[k]);
    }
}

// (m, m): the minimum over the row's disparities of the packed words w.
template <int N>
__device__ __forceinline__ uint32_t row_min2(const uint32_t (&w)[N]) {
    uint32_t x = w[0];
    if constexpr (N == 2) x = vmin2(x, w[1]);
    x = vmin2(x, __byte_perm(x, 0u, 0x1032));
    return __reduce_min_sync(kFull, x);
}

template <typename CodeT>
__device__ __forceinline__ uint32_t hamming(CodeT a, CodeT b) {
    if constexpr (sizeof(CodeT) == 8) return (uint32_t)__popcll(a ^ b);
    else return (uint32_t)__popc(a ^ b);
}

template <typename CodeT>
__device__ __forceinline__ CodeT shfl_code(CodeT v, int src) {
    if constexpr (sizeof(CodeT) == 8) {
        const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src);
        const uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
        return ((CodeT)hi << 32) | lo;
    } else {
        return __shfl_sync(kFull, v, src);
    }
}

template <typename CodeT>
__device__ __forceinline__ CodeT shfl_up_code(CodeT v) {
    if constexpr (sizeof(CodeT) == 8) {
        const uint32_t lo = __shfl_up_sync(kFull, (uint32_t)v, 1);
        const uint32_t hi = __shfl_up_sync(kFull, (uint32_t)(v >> 32), 1);
        return ((CodeT)hi << 32) | lo;
    } else {
        return __shfl_up_sync(kFull, v, 1);
    }
}

// Abort state of one launch: a bounded wait that gives up raises the grid's
// abort word (and records the timeout in the status word), and every other
// wait then returns at once.
struct Abort {
    uint32_t *word;    // zeroed before the launch
    uint32_t *status;  // the handle's status word, may be null
    unsigned long long limit_ns;
    __device__ __forceinline__ bool raised() const { return *(volatile const uint32_t *)word != 0u; }
    __device__ __forceinline__ void raise() const {
        atomicExch(word, 1u);
        if (status) atomicOr(status, kSweepTimeout);
    }
};

// Waits (every lane) until *p >= need; false when the wait gave up.  The
// result is the same in every lane.
__device__ __forceinline__ bool wait_cta(const uint32_t *p, uint32_t need, const Abort &ab) {
    bool ok = ld_acquire_cta(p) >= need;
    if (!__all_sync(kFull, ok)) {
        const unsigned long long t0 = now_ns();
        for (;;) {
            ok = ld_acquire_cta(p) >= need;
            if (__all_sync(kFull, ok)) break;
            if (ab.raised() || now_ns() - t0 > ab.limit_ns) {
                ok = false;
                break;
            }
        }
    }
    ok = __all_sync(kFull, ok);
    if (!ok && (threadIdx.x & 31) == 0) ab.raise();
    return ok;
}
// Global counter; `seen` caches the last value read (the same in every lane).
__device__ __forceinline__ bool wait_gpu(const uint32_t *p, uint32_t need, const Abort &ab, uint32_t &seen) {
    if (seen >= need) return true;
    seen = __shfl_sync(kFull, ld_acquire_gpu(p), 0);
    bool ok = seen >= need;
    if (!ok) {
        const unsigned long long t0 = now_ns();
        for (;;) {
            __nanosleep(64);
            seen = __shfl_sync(kFull, ld_acquire_gpu(p), 0);
            if (seen >= need) {
                ok = true;
                break;
            }
            if (ab.raised() || now_ns() - t0 > ab.limit_ns) break;
        }
    }
    ok = __all_sync(kFull, ok);
    if (!ok && (threadIdx.x & 31) == 0) ab.raise();
    // every lane reads what the producer wrote before the counter moved
    __syncwarp();
    return ok;
}

// FLAGS: the enabled paths fixed at compile time (kSweep* bits), or 0 to take
// them from a.flags; with them fixed the four paths' updates form one
// straight block the compiler can interleave.
template <int DPL, typename CodeT, bool RAGGED, int FLAGS>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs a) {
    constexpr int N = DPL / 2;
    using LRing = Ring<N, kSlots>;
    using LandRing = Ring<N, kLandSlots>;
    using GRing = Ring<N, kGSlots>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = a.rows_per_cta;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * R + warp;
    LRing *rings = reinterpret_cast<LRing *>(smem);                     // ring k: row k -> row k+1 of this CTA
    LandRing *land = reinterpret_cast<LandRing *>(rings + (R - 1));     // first row's landing ring
    uint32_t *prog = reinterpret_cast<uint32_t *>(land + 1);            // [R] pixels published per row
    for (int i = threadIdx.x; i < R; i += blockDim.x) prog[i] = 0u;
    __syncthreads();
    if (y >= a.H) return;

    const int W = a.W, D = a.D;
    const int d0 = DPL * lane;
    const int flags = FLAGS ? FLAGS : a.flags;
    const bool fH = flags & kSweepH, fV = flags & kSweepV, fDL = flags & kSweepDL, fDR = flags & kSweepDR;
    const bool vert = fV || fDL || fDR;
    // consumer: pixel x needs the producer row's pixels up to x + lag - 1
    const int lag = fDR ? 2 : (fV ? 1 : 0);
    const bool has_prod = vert && y > 0;
    const bool has_cons = vert && y + 1 < a.H;
    const bool prod_global = has_prod && warp == 0;        // producer is the previous CTA's last row
    const bool cons_global = has_cons && warp == R - 1;    // consumer is the next CTA's first row
    const int nb = gridDim.x + 1;  // boundaries, indexed by the consuming CTA
    GRing *gin = reinterpret_cast<GRing *>(a.grings) + blockIdx.x;        // boundary (blockIdx-1 -> blockIdx)
    GRing *gout = reinterpret_cast<GRing *>(a.grings) + blockIdx.x + 1;   // boundary (blockIdx -> blockIdx+1)
    uint32_t *gprod_in = a.gprog + blockIdx.x, *gcons_in = a.gprog + nb + blockIdx.x;
    uint32_t *gprod_out = a.gprog + blockIdx.x + 1, *gcons_out = a.gprog + nb + blockIdx.x + 1;
    const Abort ab{a.gprog + 2 * nb, a.status, a.wait_ns};
    LRing *rin = warp > 0 ? rings + (warp - 1) : nullptr;
    LRing *rout = (has_cons && !cons_global) ? rings + warp : nullptr;
    uint32_t *my_prog = prog + warp;
    const uint32_t *in_prog = warp > 0 ? prog + (warp - 1) : nullptr;
    const uint32_t *out_prog = warp + 1 < R ? prog + (warp + 1) : nullptr;

    const uint32_t lo_edge = lane == 0 ? 0x7FFFu : 0u;
    const uint32_t hi_edge = lane == 31 ? 0x7FFF0000u : 0u;
    // padding disparities d >= D are parked at 0x7FFF in the path words and
    // get no key (packed words: N == 1 (d0, d0+1); N == 2 (d0, d0+2), (d0+1, d0+3))
    uint32_t inv[N];
    uint32_t kinv[DPL];  // 0xFFFFFFFF for a padding disparity's key
#pragma unroll
    for (int k = 0; k < N; k++) {
        const int dlo = N == 1 ? d0 : d0 + k, dhi = N == 1 ? d0 + 1 : d0 + k + 2;
        inv[k] = RAGGED ? ((dlo >= D ? 0x7FFFu : 0u) | (dhi >= D ? 0x7FFF0000u : 0u)) : 0u;
    }
#pragma unroll
    for (int j = 0; j < DPL; j++) kinv[j] = (RAGGED && d0 + j >= D) ? 0xFFFFFFFFu : 0u;

    const CodeT *cl_row = reinterpret_cast<const CodeT *>(a.codes) + (size_t)y * W;
    const CodeT *cr_row = reinterpret_cast<const CodeT *>(a.codes) + (size_t)a.H * W + (size_t)y * W;
    uint8_t *dl_row = a.disp_lr + (size_t)y * W;
    uint8_t *dr_row = a.dr_map + (size_t)y * W;

    // path states: H in registers; m2 = (m, m), mP2 = m2 + (P2, P2)
    uint32_t Lh[N], mh2 = 0u, mhP2 = a.P2x2;
#pragma unroll
    for (int k = 0; k < N; k++) Lh[k] = inv[k];
    // right codes of this lane's disparities: rc[j] = codeR(x - d0 - j), kept
    // in rotation order (see the step below); T[j] the right-winner conveyor
    CodeT rc[DPL];
    uint32_t T[DPL];
#pragma unroll
    for (int j = 0; j < DPL; j++) {
        rc[j] = 0;
        T[j] = 0xFFFFFFFFu;
    }
    // the lane holding disparity D-1 emits the right winner of x - (D-1)
    const int lane_last = (D - 1) / DPL, j_last = (D - 1) % DPL;

    uint32_t seen_prod = 0, seen_cons = 0;  // last values read of the global counters
    bool ok = true;
    if (prod_global) {
        // request the first kLandAhead slots of the global ring into the
        // landing ring, one commit group per slot (empty past the row's end),
        // so that after the group of step x, wait_group(kLandAhead) leaves
        // slot x landed
        for (int s = 0; s < kLandAhead; s++) {
            if (s < W && ok) {
                ok = wait_gpu(gprod_in, (uint32_t)min(s + lag, W), ab, seen_prod);
                if (ok) fetch_slot<N>(land, s % kLandSlots, gin, s % kGSlots, lane);
            }
            cp_async_commit();
        }
    }
    // census codes in 32-pixel chunks, lane i holding pixel x0 + i: the chunk
    // in use (cur) and the next one (nxt); a chunk is loaded when the one two
    // ahead of it is taken into use, 32 to 64 steps before it is needed, and
    // each step broadcasts its pixel's codes with a shuffle
    CodeT cur_l = lane < W ? cl_row[lane] : 0, cur_r = lane < W ? cr_row[lane] : 0;
    CodeT nxt_l = 32 + lane < W ? cl_row[32 + lane] : 0, nxt_r = 32 + lane < W ? cr_row[32 + lane] : 0;

    for (int x = 0; x < W && ok; x++) {
        // ---- inputs of the vertical paths --------------------------------
        uint32_t Lv[N], Ldl[N], Ldr[N], mv = 0u, mdl = 0u, mdr = 0u;
#pragma unroll
        for (int k = 0; k < N; k++) Lv[k] = Ldl[k] = Ldr[k] = inv[k];
        if (has_prod) {
            const uint32_t *wv, *wdl, *wdr, *ms;  // this lane's words of slot x, and its minima
            if (prod_global) {
                // slot x was requested kLandAhead pixels ago; request slot x + kLandAhead
                const int s = x + kLandAhead;
                if (s < W) {
                    ok = wait_gpu(gprod_in, (uint32_t)min(s + lag, W), ab, seen_prod);
                    if (!ok) break;
                    fetch_slot<N>(land, s % kLandSlots, gin, s % kGSlots, lane);
                }
                cp_async_commit();
                cp_async_wait<kLandAhead>();
                __syncwarp();
                const int ls = x % kLandSlots;
                wv = ring_words<N>(land, ls, 0, lane);
                wdl = ring_words<N>(land, ls, 1, lane);
                wdr = ring_words<N>(land, ls, 2, lane);
                ms = land->m[ls];
                // consumption, for the producer's back-pressure
                if (lane == 0 && ((x + 1) % kPub == 0 || x + 1 == W)) st_release_gpu(gcons_in, (uint32_t)(x + 1));
            } else {
                // (the stalled-wait test asks for a pixel past the row's end)
                ok = wait_cta(in_prog, y == a.stall_row ? (uint32_t)W + 1u : (uint32_t)min(x + lag, W), ab);
                if (!ok) break;
                const int ls = x % kSlots;
                wv = ring_words<N>(rin, ls, 0, lane);
                wdl = ring_words<N>(rin, ls, 1, lane);
                wdr = ring_words<N>(rin, ls, 2, lane);
                ms = rin->m[ls];
            }
            if (fV) {
#pragma unroll
                for (int k = 0; k < N; k++) Lv[k] = wv[k];
                mv = ms[0];
            }
            if (fDL && x > 0) {
#pragma unroll
                for (int k = 0; k < N; k++) Ldl[k] = wdl[k];
                mdl = ms[1];
            }
            if (fDR && x + 1 < W) {
#pragma unroll
                for (int k = 0; k < N; k++) Ldr[k] = wdr[k];
                mdr = ms[2];
            }
        }

        // ---- matching cost (Eq. 1) ------------------------------------------
        const int xi = x & 31;
        const CodeT cl = shfl_code<CodeT>(cur_l, xi);
        {
            // shift the right codes up one disparity: lane 0 takes codeR(x)
            const CodeT crx = shfl_code<CodeT>(cur_r, xi);
            const CodeT from_prev = shfl_up_code<CodeT>(rc[DPL - 1]);
#pragma unroll
            for (int j = DPL - 1; j > 0; j--) rc[j] = rc[j - 1];
            rc[0] = lane == 0 ? crx : from_prev;
        }
        if (xi == 31) {
            cur_l = nxt_l;
            cur_r = nxt_r;
            const int xn = x + 33 + lane;  // pixel of this lane in the chunk after next
            nxt_l = xn < W ? cl_row[xn] : 0;
            nxt_r = xn < W ? cr_row[xn] : 0;
        }
        uint32_t cj[DPL];
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            cj[j] = hamming<CodeT>(cl, rc[j]);
            if (x < d0 + j) cj[j] = a.nbits;  // x - d < 0
        }
        uint32_t C[N];
        if constexpr (N == 1) {
            C[0] = cj[0] | (cj[1] << 16);
        } else {
            C[0] = cj[0] | (cj[2] << 16);
            C[1] = cj[1] | (cj[3] << 16);
        }

        // ---- path updates (Eq. 2) -------------------------------------------
        uint32_t S[N];
#pragma unroll
        for (int k = 0; k < N; k++) S[k] = 0u;
        if (fH) {
            uint32_t o[N];
            path_update<N, RAGGED>(Lh, mh2, mhP2, C, a.P1x2, lo_edge, hi_edge, inv, o);
#pragma unroll
            for (int k = 0; k < N; k++) {
                Lh[k] = o[k];
                S[k] += o[k];
            }
            mh2 = row_min2<N>(o);
            mhP2 = mh2 + a.P2x2;
        }
        uint32_t Ov[N], Odl[N], Odr[N], nv = 0u, ndl = 0u, ndr = 0u;
        if (fV) {
            path_update<N, RAGGED>(Lv, mv, mv + a.P2x2, C, a.P1x2, lo_edge, hi_edge, inv, Ov);
            if (has_cons) nv = row_min2<N>(Ov);
#pragma unroll
            for (int k = 0; k < N; k++) S[k] += Ov[k];
        }
        if (fDL) {
            path_update<N, RAGGED>(Ldl, mdl, mdl + a.P2x2, C, a.P1x2, lo_edge, hi_edge, inv, Odl);
            if (has_cons) ndl = row_min2<N>(Odl);
#pragma unroll
            for (int k = 0; k < N; k++) S[k] += Odl[k];
        }
        if (fDR) {
            path_update<N, RAGGED>(Ldr, mdr, mdr + a.P2x2, C, a.P1x2, lo_edge, hi_edge, inv, Odr);
            if (has_cons) ndr = row_min2<N>(Odr);
#pragma unroll
            for (int k = 0; k < N; k++) S[k] += Odr[k];
        }

        // ---- hand the vertical paths to the next row -----------------------
        if (has_cons) {
            const int nslots = cons_global ? kGSlots : kSlots;
            if (cons_global) {
                // back-pressure: writing slot x+1 overwrites slot x+1-kGSlots
                ok = wait_gpu(gcons_out, (uint32_t)max(0, x + 2 - kGSlots), ab, seen_cons);
            } else {
                ok = wait_cta(out_prog, (uint32_t)max(0, x + 2 - kSlots), ab);
            }
            if (!ok) break;
            const int sv = x % nslots, sdl = (x + 1) % nslots, sdr = (x + nslots - 1) % nslots;
            uint32_t *pv, *pdl, *pdr, *mv_, *mdl_, *mdr_;
            if (cons_global) {
                pv = ring_words<N>(gout, sv, 0, lane);
                pdl = ring_words<N>(gout, sdl, 1, lane);
                pdr = ring_words<N>(gout, sdr, 2, lane);
                mv_ = &gout->m[sv][0];
                mdl_ = &gout->m[sdl][1];
                mdr_ = &gout->m[sdr][2];
            } else {
                pv = ring_words<N>(rout, sv, 0, lane);
                pdl = ring_words<N>(rout, sdl, 1, lane);
                pdr = ring_words<N>(rout, sdr, 2, lane);
                mv_ = &rout->m[sv][0];
                mdl_ = &rout->m[sdl][1];
                mdr_ = &rout->m[sdr][2];
            }
            if (fV) {
#pragma unroll
                for (int k = 0; k < N; k++) pv[k] = Ov[k];
                if (lane == 0) *mv_ = nv;
            }
            if (fDL) {
#pragma unroll
                for (int k = 0; k < N; k++) pdl[k] = Odl[k];
                if (lane == 0) *mdl_ = ndl;
            }
            if (fDR && x > 0) {
#pragma unroll
                for (int k = 0; k < N; k++) pdr[k] = Odr[k];
                if (lane == 0) *mdr_ = ndr;
            }
            if (cons_global && ((x + 1) % kPub == 0 || x + 1 == W)) {
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release_gpu(gprod_out, (uint32_t)(x + 1));
            }
        }
        // this row's pixel x is done: its inputs are consumed and its outputs written
        __syncwarp();
        if (lane == 0) st_release_cta(my_prog, (uint32_t)(x + 1));

        // ---- winners ---------------------------------------------------------
        // keys (S << 8) | d; S <= 4 * 255 fits 16 bits, and a padding half
        // (0x7FFF per path) can only carry out of the top of its word
        uint32_t key[DPL];
        if constexpr (N == 1) {
            key[0] = ((S[0] & 0xFFFFu) << 8) | (uint32_t)d0;
            key[1] = ((S[0] >> 16) << 8) | (uint32_t)(d0 + 1);
        } else {
            key[0] = ((S[0] & 0xFFFFu) << 8) | (uint32_t)d0;
            key[2] = ((S[0] >> 16) << 8) | (uint32_t)(d0 + 2);
            key[1] = ((S[1] & 0xFFFFu) << 8) | (uint32_t)(d0 + 1);
            key[3] = ((S[1] >> 16) << 8) | (uint32_t)(d0 + 3);
        }
        uint32_t best = 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            key[j] |= kinv[j];
            best = min(best, key[j]);
        }
        best = __reduce_min_sync(kFull, best);
        if (lane == 0) dl_row[x] = (uint8_t)(best & 0xFFu);
        // right-winner conveyor: T_d(x) = min(T_{d-1}(x-1), key(x, d))
        {
            uint32_t in0 = __shfl_up_sync(kFull, T[DPL - 1], 1);
            if (lane == 0) in0 = 0xFFFFFFFFu;
#pragma unroll
            for (int j = DPL - 1; j > 0; j--) T[j] = min(T[j - 1], key[j]);
            T[0] = min(in0, key[0]);
        }
        if (lane == lane_last && x >= D - 1) {
            uint32_t t = T[0];
#pragma unroll
            for (int j = 1; j < DPL; j++)
                if (j == j_last) t = T[j];
            dr_row[x - (D - 1)] = (uint8_t)(t & 0xFFu);
        }
    }
    if (prod_global) cp_async_wait<0>();
    if (!ok) return;
    // targets W-1-d for d < D-1 never saw disparity D-1: T_d(W-1) is their winner
#pragma unroll
    for (int j = 0; j < DPL; j++) {
        const int d = d0 + j;
        if (d < D - 1 && W - 1 - d >= 0) dr_row[W - 1 - d] = (uint8_t)(T[j] & 0xFFu);
    }
    __syncwarp();
    // LR check of the row (Sec. 3.1.4)
    for (int xx = lane; xx < W; xx += 32) {
        const int dl = dl_row[xx];
        uint8_t v = (uint8_t)dl;
        if (a.dbg_left) a.dbg_left[(size_t)y * W + xx] = (uint8_t)dl;
        if (a.tol >= 0) {
            const int xr = xx - dl;
            if (xr < 0) {
                v = SGM_INVALID;
            } else {
                const int dr = dr_row[xr];
                const int diff = dl > dr ? dl - dr : dr - dl;
                if (diff > a.tol) v = SGM_INVALID;
            }
        }
        dl_row[xx] = v;
    }
}

template <int DPL>
size_t sweep_smem(int R) {
    constexpr int N = DPL / 2;
    return sizeof(Ring<N, kSlots>) * (R - 1) + sizeof(Ring<N, kLandSlots>) + sizeof(uint32_t) * R;
}

// Raises the kernel's dynamic shared-memory limit to the largest any rows-per-
// CTA setting needs (once per device and instantiation).
template <int DPL, typename CodeT, bool RAGGED, int FLAGS>
cudaError_t prepare(int dev) {
    static std::atomic<unsigned long long> done{0};
    if (dev >= 0 && dev < 64 && (done.load() >> dev) & 1ull) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(sweep_kernel<DPL, CodeT, RAGGED, FLAGS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sweep_smem<DPL>(8));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done.fetch_or(1ull << dev);
    return e;
}

template <int DPL, typename CodeT, bool RAGGED, int FLAGS>
cudaError_t launch_t(const SweepArgs &a, int R, cudaStream_t s) {
    auto k = sweep_kernel<DPL, CodeT, RAGGED, FLAGS>;
    const size_t smem = sweep_smem<DPL>(R);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = prepare<DPL, CodeT, RAGGED, FLAGS>(dev);
    if (e != cudaSuccess) return e;
    const int nctas = (a.H + R - 1) / R;
    // residency of the whole grid was checked by sweep_fits when the schedule
    // was chosen; the cooperative launch fails rather than run it otherwise
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nctas);
    cfg.blockDim = dim3(R * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace

bool sweep_supported(int D, int mask, int code_bytes) {
    return code_bytes > 0 && D >= 1 && D <= 128 && mask != 0 && (mask & ~0x55) == 0;
}

// Scratch of one launch: a global ring per CTA boundary, the boundaries'
// counters and the abort word (16-byte padded), and the right map.
static size_t ring_bytes(int D) { return D <= 64 ? sizeof(Ring<1, kGSlots>) : sizeof(Ring<2, kGSlots>); }
static size_t counter_bytes(int nctas) { return (sizeof(uint32_t) * (2 * (size_t)(nctas + 1) + 1) + 15) / 16 * 16; }

size_t sweep_scratch_bytes(int W, int H, int D, int rows_per_cta) {
    const int nctas = (H + rows_per_cta - 1) / rows_per_cta;
    return (size_t)(nctas + 1) * ring_bytes(D) + counter_bytes(nctas) + (size_t)W * H;
}

cudaError_t launch_sweep(const void *codes, int code_bytes, int W, int H, int D, int nbits, int P1, int P2,
                         int mask, int tol, uint8_t *disp_lr, uint8_t *dbg_left, uint8_t *dbg_right,
                         void *scratch, unsigned *status, int rows_per_cta, cudaStream_t s, int stall_test) {
    if (!sweep_supported(D, mask, code_bytes) || rows_per_cta < 1 || rows_per_cta > 8) return cudaErrorInvalidValue;
    // the stalled row must have a producer inside its block (row 1, same block as row 0)
    if (stall_test && (H < 2 || rows_per_cta < 2 || !(mask & 0x54))) return cudaErrorInvalidValue;
    const int R = rows_per_cta;
    const int nctas = (H + R - 1) / R;
    const int DPL = D <= 64 ? 2 : 4;
    const size_t ring = ring_bytes(D);
    unsigned char *p = reinterpret_cast<unsigned char *>(scratch);
    SweepArgs a;
    a.codes = codes;
    a.W = W;
    a.H = H;
    a.D = D;
    a.nbits = (uint32_t)nbits;
    a.P1x2 = (uint32_t)P1 * 0x00010001u;
    a.P2x2 = (uint32_t)P2 * 0x00010001u;
    a.flags = ((mask & 0x01) ? kSweepH : 0) | ((mask & 0x04) ? kSweepV : 0) | ((mask & 0x10) ? kSweepDL : 0) |
              ((mask & 0x40) ? kSweepDR : 0);
    a.tol = tol;
    a.rows_per_cta = R;
    a.disp_lr = disp_lr;
    a.grings = p;
    a.gprog = reinterpret_cast<uint32_t *>(p + (size_t)(nctas + 1) * ring);
    a.dr_map = dbg_right ? dbg_right : reinterpret_cast<uint8_t *>(a.gprog) + counter_bytes(nctas);
    a.dbg_left = dbg_left;
    a.status = status;
    a.wait_ns = stall_test ? kStallTestNs : kWaitNs;
    a.stall_row = stall_test ? 1 : -1;
    cudaError_t e = cudaMemsetAsync(a.gprog, 0, counter_bytes(nctas), s);
    if (e != cudaSuccess) return e;
    const bool rag = D != 32 * DPL;
    // the paper's four streaming paths get their own instantiation
    const bool all4 = a.flags == (kSweepH | kSweepV | kSweepDL | kSweepDR);
#define SGM_SWEEP_FL(P, C, G) (all4 ? launch_t<P, C, G, 15>(a, R, s) : launch_t<P, C, G, 0>(a, R, s))
    if (DPL == 2) {
        if (code_bytes == 8) return rag ? SGM_SWEEP_FL(2, uint64_t, true) : SGM_SWEEP_FL(2, uint64_t, false);
        return rag ? SGM_SWEEP_FL(2, uint32_t, true) : SGM_SWEEP_FL(2, uint32_t, false);
    }
    if (code_bytes == 8) return rag ? SGM_SWEEP_FL(4, uint64_t, true) : SGM_SWEEP_FL(4, uint64_t, false);
    return rag ? SGM_SWEEP_FL(4, uint32_t, true) : SGM_SWEEP_FL(4, uint32_t, false);
#undef SGM_SWEEP_FL
}

}  // namespace sgm

namespace sgm {

// True when the sweep's grid for this shape is resident at once on the current device.
bool sweep_fits(int H, int D, int code_bytes, int rows_per_cta) {
    if (rows_per_cta < 1 || rows_per_cta > 8) return false;
    const int R = rows_per_cta, nctas = (H + R - 1) / R;
    const bool rag = D != 32 * (D <= 64 ? 2 : 4);
    int dev = 0, sms = 0, per_sm = 0, per_sm2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaError_t e;
    // both instantiations (fixed and run-time path flags) must fit
#define SGM_FIT(P, C, G)                                                                                                    \
    do {                                                                                                                    \
        e = prepare<P, C, G, 0>(dev);                                                                                       \
        if (e == cudaSuccess) e = prepare<P, C, G, 15>(dev);                                                                \
        if (e == cudaSuccess)                                                                                               \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<P, C, G, 0>, R * 32, sweep_smem<P>(R));  \
        if (e == cudaSuccess)                                                                                               \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, sweep_kernel<P, C, G, 15>, R * 32, sweep_smem<P>(R)); \
    } while (0)
    if (D <= 64) {
        if (code_bytes == 8) { if (rag) SGM_FIT(2, uint64_t, true); else SGM_FIT(2, uint64_t, false); }
        else { if (rag) SGM_FIT(2, uint32_t, true); else SGM_FIT(2, uint32_t, false); }
    } else {
        if (code_bytes == 8) { if (rag) SGM_FIT(4, uint64_t, true); else SGM_FIT(4, uint64_t, false); }
        else { if (rag) SGM_FIT(4, uint32_t, true); else SGM_FIT(4, uint32_t, false); }
    }
#undef SGM_FIT
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)min(per_sm, per_sm2) * sms >= nctas;
}

}  // namespace sgm
