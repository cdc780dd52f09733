// Hamming matching cost (Eq. 1) on the tensor cores (tcgen05).
//
// Write a census code c of nbits bits as the vector c^ with entry +1 where a
// bit is clear and -1 where it is set.  For two codes the inner product counts
// equal bits minus differing bits, <a^, b^> = nbits - 2 H(a, b), so
//     C(x, y, d) = H(c_l(x, y), c_r(x - d, y)) = (nbits - <c_l^(x), c_r^(x - d)>) / 2.
// The KB - nbits entries past the code (KB = 32 or 64 entries per pixel) are
// +1 in both vectors, which adds KB - nbits to every product: H = (KB - <,>) / 2.
//
// Segments.  For the 128 pixels x0 .. x0+127 of one row, every (x, d) with
// 0 <= d < Dp reads a right pixel x - d in [x0 - Dp, x0 + 127], so the
// segment's costs lie in a band of the 128 x (Dp + 128) product A B^T: row i
// of A is the left vector of pixel x0 + i; B is the last Dp right vectors of
// the previous segment (R(k-1)) followed by the 128 of this one (R(k)), and
// column j of the product holds right pixel x0 - Dp + j.  Two tcgen05.mma
// groups (kind::f8f6f4: +-1 is exact in e4m3, the f32 sums are exact
// integers) write it to tensor memory, row i in lane i: A x R(k-1)^T into
// columns 0 .. Dp-1 and A x R(k)^T into Dp .. Dp+127, 32 code bits per MMA.
//
// Persistent pipeline.  One CTA per SM walks a contiguous run of segments
// (row-major), so each R(k) is expanded once and serves two segments.  Shared
// memory holds two A stages and three R slots; tensor memory two accumulator
// buffers of 256 columns.  Sixteen cost warps stage operands and turn sums
// into costs; a seventeenth warp only issues the MMAs (an issuing thread
// stalls while the tensor pipe takes them, so it must not hold up the cost
// warps).  The cost warps hand over segment k+1's operands with a named
// barrier arrival and wait for segment k's MMAs on an mbarrier; while they
// convert segment k, the MMAs of k+1 run and every thread holds its share of
// the codes of k+2.
//
// Standing.  On GB300 this kernel takes 41 us for the 1242 x 375, D = 128
// cost volume against 37.7 us for the CUDA-core kernel, which stays the
// default (SGM_COST_KERNEL_AUTO).  The matrix products are a small part of
// the time: a 128-pixel segment costs about 2800 cycles, most of them moving
// bytes through shared memory (operand expansion, the cost tile, the record
// staging, plus the tensor core's and the bulk copy's reads).
//   Operands: canonical K-major layout without swizzling (core matrices of
//   8 rows x 16 bytes; each 16-byte row holds 16 code bits of one pixel as
//   e4m3 entries 0x38 = +1 / 0xB8 = -1); a thread expands one 32-bit half of
//   a code (or 16 bits of a 32-bit code).
//   Sums to costs: warp w reads TMEM lanes 32(w%4) .. +31 (its lane quarter),
//   a quarter of the LC = Dp + 32 columns 32(w%4) + s the quarter needs
//   (pixel i = 32(w%4) + t uses s = t+1 .. t+Dp for d = Dp-1 .. 0).  An FMA
//   with a power-of-two scale leaves a cost in the low mantissa bits of
//   2^23 + scale * H, three such patterns XOR into three bytes and a byte
//   permute adds the fourth; the bytes go to the pixel's row of a tile T.
//   Records: each thread then takes a quarter of one pixel's 8-disparity
//   groups: it reads its window of T (word loads and one funnel shift, since
//   the start differs per pixel), puts each group in the lane-chunk byte
//   order (two byte permutes) and writes it into the segment's records in a
//   staging buffer; one cp.async.bulk copies the segment's contiguous records
//   to the cost volume.  Slots with x - d < 0 or d >= D get nbits, as in the
//   CUDA-core kernel.
//
// Waits.  The waits are on the mbarriers that MMA completion arrives on; each
// gives up after about one second.  The CTA then records the timeout in
// *status, waits once more for its MMAs and copies in flight, frees its
// tensor memory and stops (segments it had not finished keep old costs).  A
// test mode (stall_test) points the first wait at a third mbarrier that
// nothing arrives at, with a 2 ms limit, so the whole timeout path runs
// without any fault: the MMAs still complete, and the handle stays usable.
#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kM = 128;        // pixels per segment = MMA M = TMEM lanes
constexpr int kWarps = 16;     // cost warps: four per TMEM lane quarter
constexpr int kThreads = 32 * kWarps + 32;  // plus one warp that issues the MMAs
// Named barriers (0 is __syncthreads): the operands of segment k are handed to
// the MMA warp on barrier kBarOperands + 2 (k % 2), so consecutive handoffs use
// different barriers (a second arrival on one of them needs the MMA that the
// MMA warp issues only after the first has been taken); the cost warps sync
// among themselves on kBarCost.
constexpr int kBarOperands = 1, kBarCost = 2;
__device__ __forceinline__ int operand_bar(int k) { return kBarOperands + 2 * (k & 1); }
constexpr uint32_t kTmemCols = 512;  // two accumulator buffers of 256 columns
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
constexpr unsigned long long kStallTestLimitNs = 2000000ull;  // the stalled-wait test gives up after 2 ms
constexpr int kOneCtaPerSm = 116 * 1024;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Matrix descriptor of a K-major operand in shared memory without swizzling:
// start address, LBO = byte distance of K-adjacent core matrices, SBO = byte
// distance of 8-row groups (all >> 4), descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: f32 accumulators (bits 4-5 = 1), A
// and B e4m3 (0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Four code bits -> four e4m3 entries: 0x38 (+1) for a clear bit, 0xB8 (-1)
// for a set bit.  The multiply places bit m of nib at bit 8m (the four shifted
// copies do not overlap), the shift moves it to the sign bit of byte m.
__device__ __forceinline__ uint32_t pm_one4(uint32_t nib) {
    return 0x38383838u | ((nib * 0x00204081u) << 7 & 0x80808080u);
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// Costs of four sums as one word of bytes.  With b_s = KB * s / 2 + 2^23,
// fma(v, -s/2, b_s) = 2^23 + s * H exactly (|v| <= KB, s * H < 2^23), so the
// bit patterns hold H, 256 H and 65536 H above a common exponent field; the
// XOR of three leaves H0, H1, H2 in bytes 0..2 and the byte permute puts H3
// in byte 3.
__device__ __forceinline__ uint32_t costs4(const uint32_t *v, float b1, float b256, float b65536) {
    const uint32_t f0 = __float_as_uint(fmaf(__uint_as_float(v[0]), -0.5f, b1));
    const uint32_t f1 = __float_as_uint(fmaf(__uint_as_float(v[1]), -128.0f, b256));
    const uint32_t f2 = __float_as_uint(fmaf(__uint_as_float(v[2]), -32768.0f, b65536));
    const uint32_t f3 = __float_as_uint(fmaf(__uint_as_float(v[3]), -0.5f, b1));
    return __byte_perm(f0 ^ f1 ^ f2, f3, 0x4210);
}

// Named barriers: `count` threads (whole warps) take part; arrive does not wait.
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_or(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Waits for the phase of parity `parity` of the mbarrier at bar, giving up after limit_ns.
__device__ __forceinline__ bool wait_mbar(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kWaitLimitNs) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Shared-memory layout of one CTA (byte offsets).
template <int DP, int KB>
struct Smem {
    static constexpr int LC = DP + 32;            // columns a lane quarter reads
    static constexpr int kOp = kM * KB;           // one operand slot: 128 rows of KB bytes
    static constexpr int kA = 0;                  // A stages [2]
    static constexpr int kR = 2 * kOp;            // R slots [3]
    static constexpr int kT = 5 * kOp;            // cost bytes, [128] rows
    static constexpr int kTPitch = LC + 8;        // odd number of 8-byte units: conflict-free row stores
    static constexpr int kO = kT + kM * kTPitch;  // staged records [2][128][DP]
    static constexpr int kBar = kO + 2 * kM * DP; // two mbarriers, then one nothing arrives at
    static constexpr int kSlot = kBar + 32;      // TMEM address, then the abort flag
    static constexpr int kBytes = kSlot + 16;
    static_assert(kT % 16 == 0 && kO % 16 == 0 && kBar % 16 == 0, "16-byte aligned regions");
};

template <int DP, int KB, bool RAGGED>
__global__ void __launch_bounds__(kThreads, 1)
    hamming_mma_kernel(const uint32_t *__restrict__ codes, int W, int H, int D, int nbits,
                       uint8_t *__restrict__ cost, unsigned *__restrict__ job_state,
                       unsigned *__restrict__ status, int stall_test) {
    using L = Smem<DP, KB>;
    constexpr int LC = L::LC, NCH = DP / 8, CPP = NCH / 4;  // chunks per thread in the record step
    constexpr int CW = KB / 32;                             // 32-bit words per code
    static_assert(DP == 32 || DP == 64 || DP == 128, "tensor-core cost kernel: Dp of 32, 64 or 128");
    extern __shared__ __align__(1024) unsigned char mma_smem[];
    wait_for_predecessor();
    if (job_state && blockIdx.x == 0)
        for (int i = threadIdx.x; i < (int)(kJobStateBytes / sizeof(unsigned)); i += kThreads) job_state[i] = 0u;
    const int tid = threadIdx.x, warp = tid >> 5, t = tid & 31;
    const int segs_row = (W + kM - 1) / kM;
    const long long nseg = (long long)segs_row * H;
    const int s_begin = (int)(nseg * blockIdx.x / gridDim.x), s_end = (int)(nseg * (blockIdx.x + 1) / gridDim.x);
    unsigned char *T = mma_smem + L::kT;
    const uint32_t bar0 = smem_addr(mma_smem + L::kBar);
    uint32_t *slot = reinterpret_cast<uint32_t *>(mma_smem + L::kSlot);
    const size_t npix = (size_t)W * H;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 16) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // Operand expansion.  Thread tid owns operand row r of a segment (r < 128:
    // A row r, left pixel x0 + r; else R row r - 128, right pixel x0 + r - 128)
    // and the 32 entries 32h .. 32h+31 of it, that is code word h (KB = 64) or
    // half h of the code (KB = 32); r = tid % 8 + 8 (tid / 16), h = (tid / 8) % 2,
    // so the eight threads of a quarter warp store to eight different core-matrix rows.
    const int orow = (tid & 7) | ((tid >> 4) << 3), oh = (tid >> 3) & 1;
    const int wbit = KB == 64 ? 32 * oh : 0;  // first code bit of the thread's code word
    const uint32_t keep = nbits - wbit >= 32 ? 0xFFFFFFFFu : nbits - wbit <= 0 ? 0u : (1u << (nbits - wbit)) - 1u;
    // (the mask is applied when a word is expanded, so a load is waited for only then)
    auto code_word = [&](size_t p) { return codes[p * CW + (KB == 64 ? oh : 0)]; };
    auto load_code = [&](int s, int row) -> uint32_t {  // the thread's code word of operand row `row`
        const int y = s / segs_row, x0 = (s - y * segs_row) * kM;
        const int x = x0 + (row & (kM - 1));
        if (x >= W) return 0u;
        return code_word((row < kM ? 0 : npix) + (size_t)y * W + x);
    };
    auto expand = [&](unsigned char *op, int r, uint32_t w) {  // row r of a 128-row operand slot
        unsigned char *row = op + (r >> 3) * (8 * KB) + (r & 7) * 16;
        w &= keep;
        if constexpr (KB == 64) {
#pragma unroll
            for (int u = 0; u < 2; u++) {  // core-matrix columns 2h, 2h+1: bits 16u .. 16u+15 of word h
                const uint32_t b = w >> (16 * u);
                *reinterpret_cast<uint4 *>(row + (2 * oh + u) * 128) = make_uint4(
                    pm_one4(b & 15u), pm_one4((b >> 4) & 15u), pm_one4((b >> 8) & 15u), pm_one4((b >> 12) & 15u));
            }
        } else {  // core-matrix column h: bits 16h .. 16h+15 of the code
            const uint32_t b = w >> (16 * oh);
            *reinterpret_cast<uint4 *>(row + oh * 128) = make_uint4(
                pm_one4(b & 15u), pm_one4((b >> 4) & 15u), pm_one4((b >> 8) & 15u), pm_one4((b >> 12) & 15u));
        }
    };
    auto a_slot = [&](int k) { return mma_smem + L::kA + (k & 1) * L::kOp; };
    auto r_slot = [&](int k) { return mma_smem + L::kR + ((k % 3 + 3) % 3) * L::kOp; };
    auto put_segment = [&](int k, uint32_t w) {  // operand rows of iteration k's segment
        if (orow < kM) expand(a_slot(k), orow, w);
        else expand(r_slot(k), orow - kM, w);
    };
    auto issue_mma = [&](int k, uint32_t tmem_base) {
        const uint32_t tb = tmem_base + 256u * (uint32_t)(k & 1);
        const uint32_t a0 = smem_addr(a_slot(k));
        const uint32_t p0 = smem_addr(r_slot(k - 1)) + (uint32_t)((kM - DP) / 8 * (8 * KB));  // rows 128-DP .. 127
        const uint32_t c0 = smem_addr(r_slot(k));
#pragma unroll
        for (int q = 0; q < KB / 32; q++) {  // 32 code bits (two 16-byte core matrices) per MMA
            const uint64_t ad = smem_desc(a0 + 256 * q, 128, 8 * KB);
            mma_f8(tb, ad, smem_desc(p0 + 256 * q, 128, 8 * KB), mma_idesc(kM, DP), q);
            mma_f8(tb + DP, ad, smem_desc(c0 + 256 * q, 128, 8 * KB), mma_idesc(kM, kM), q);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar0 + 8u * (uint32_t)(k & 1))
                     : "memory");
    };

    // prologue: operands of the first segment (and the R(k-1) it reads), codes of the second
    const bool mma_warp = warp == kWarps;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(slot + 1);
    uint32_t cw = 0u;
    if (!mma_warp) {
        put_segment(0, load_code(s_begin, orow));
        if ((s_begin % segs_row) != 0 && orow < kM) {  // right codes of the previous segment of the row
            const int y = s_begin / segs_row, x = (s_begin - y * segs_row) * kM - kM + orow;
            expand(r_slot(-1), orow, code_word(npix + (size_t)y * W + x));
        }
        if (s_begin + 1 < s_end) cw = load_code(s_begin + 1, orow);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    } else if (t == 0) {
        *abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;

    if (mma_warp) {
        // MMA k waits until the cost warps have staged its operands and finished reading
        // TMEM buffer k & 1 (iteration k-2), which they signal in iteration k-1
        const int n = s_end - s_begin;
        for (int kk = 0; kk < n; kk++) {
            if (kk > 0) {
                bar_sync(operand_bar(kk), kThreads);
                if (*abort_flag) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            if (t == 0) issue_mma(kk, tmem);
            __syncwarp();
        }
    } else {

    const float b1 = 0.5f * KB + 8388608.0f, b256 = 128.0f * KB + 8388608.0f, b65536 = 32768.0f * KB + 8388608.0f;
    const int quarter = warp & 3, part = warp >> 2;
    constexpr int kCostThreads = 32 * kWarps;
    int k = 0;
    for (int s = s_begin; s < s_end; s++, k++) {
        const bool has_next = s + 1 < s_end;
        if (has_next) {
            put_segment(k + 1, cw);  // stage and slot last read by the MMAs of iteration k-1 (complete)
            if (s + 2 < s_end) cw = load_code(s + 2, orow);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            bar_arrive(operand_bar(k + 1), kThreads);  // operands of k+1 staged, TMEM buffer (k+1) & 1 free
        }
        // stall_test: the first wait is on the barrier nothing arrives at, so it runs out (tests the timeout path)
        const bool ok = stall_test && k == 0 ? wait_mbar(bar0 + 16u, 0u, kStallTestLimitNs)
                                             : wait_mbar(bar0 + 8u * (uint32_t)(k & 1), (uint32_t)(k >> 1) & 1u);
        if (bar_or(kBarCost, kCostThreads, !ok)) {
            if (tid == 0) {
                if (status) atomicOr(status, 1u);
                *abort_flag = 1;
                wait_mbar(bar0 + 8u * (uint32_t)(k & 1), (uint32_t)(k >> 1) & 1u);  // let the MMAs drain
                if (has_next) wait_mbar(bar0 + 8u * (uint32_t)((k + 1) & 1), (uint32_t)((k + 1) >> 1) & 1u);
            }
            bar_sync(kBarCost, kCostThreads);  // abort flag written
            // the MMA warp waits for the operands of k+2 when there are any: release it
            if (s + 2 < s_end) bar_arrive(operand_bar(k + 2), kThreads);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        {
            // sums -> cost bytes of columns 32 * quarter + part * LC/4 + 0 .. LC/4 - 1 of TMEM lane 32 * quarter + t
            constexpr int NLD = LC / 32;  // loads of 8 columns per part
            uint32_t v[NLD][8];
            const uint32_t taddr = tmem + 256u * (uint32_t)(k & 1) + ((uint32_t)(32 * quarter) << 16) +
                                   (uint32_t)(32 * quarter + part * (LC / 4));
#pragma unroll
            for (int c8 = 0; c8 < NLD; c8++) tmem_ld8(taddr + 8u * c8, v[c8]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            unsigned char *trow = T + (32 * quarter + t) * L::kTPitch + part * (LC / 4);
#pragma unroll
            for (int c8 = 0; c8 < NLD; c8++)
                *reinterpret_cast<uint2 *>(trow + 8 * c8) =
                    make_uint2(costs4(v[c8], b1, b256, b65536), costs4(v[c8] + 4, b1, b256, b65536));
        }
        // the bulk copy that read staging buffer k & 1 (iteration k-2) has finished reading it
        if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        bar_sync(kBarCost, kCostThreads);  // every row of T written
        const int y = s / segs_row, x0 = (s - y * segs_row) * kM;
        unsigned char *O = mma_smem + L::kO + (k & 1) * (kM * DP);
        {
            // records: pixel i = 8 * warp + t / 4, chunks CPP * p .. CPP * p + CPP - 1, p = t % 4.
            // Pixel i (lane t_i = i % 32 of its quarter) reads bytes u = 0 .. DP-1 of its T row from
            // t_i + 1 on, u <-> d = DP - 1 - u.  With word U[m] = bytes 4m .. 4m+3 of the part that
            // starts at u = DP - 8 CPP (p + 1), chunk q = CPP p + m (d = 8q .. 8q+7) is
            // U[2 CPP - 2 - 2m] (d = 8q+7 .. 8q+4) and the next word (d = 8q+3 .. 8q).
            const int i = 8 * warp + (t >> 2), p = t & 3, x = x0 + i;
            const int ti = (i & 31) + 1;
            const uint32_t *tw = reinterpret_cast<const uint32_t *>(T + i * L::kTPitch) + (ti >> 2) +
                                 (DP / 4 - 2 * CPP * (p + 1));
            const uint32_t sh = 8u * (uint32_t)(ti & 3);
            uint32_t U[2 * CPP];
            uint32_t prev = tw[0];
#pragma unroll
            for (int m = 0; m < 2 * CPP; m++) {
                const uint32_t nx = tw[m + 1];
                U[m] = __funnelshift_r(prev, nx, sh);
                prev = nx;
            }
            const bool edge = RAGGED || x < DP - 1;
            uint32_t c[2 * CPP];
#pragma unroll
            for (int m = 0; m < CPP; m++) {
                const int q = CPP * p + m;
                const uint32_t hi = U[2 * CPP - 2 - 2 * m], lo = U[2 * CPP - 1 - 2 * m];
                uint32_t c0 = __byte_perm(hi, lo, 0x2367), c1 = __byte_perm(hi, lo, 0x0145);
                if (edge) {
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const int d = 8 * q + e;
                        if ((RAGGED && d >= D) || x - d < 0) {
                            const int pos = chunk_byte(8, e);
                            const uint32_t mk = 0xFFu << (8 * (pos & 3));
                            if (pos < 4) c0 = (c0 & ~mk) | ((uint32_t)nbits << (8 * (pos & 3)));
                            else c1 = (c1 & ~mk) | ((uint32_t)nbits << (8 * (pos & 3)));
                        }
                    }
                }
                c[2 * m] = c0;
                c[2 * m + 1] = c1;
            }
            unsigned char *rec = O + i * DP + p * (8 * CPP);
            if constexpr (CPP == 1) {
                *reinterpret_cast<uint2 *>(rec) = make_uint2(c[0], c[1]);
            } else if constexpr (CPP == 2) {
                *reinterpret_cast<uint4 *>(rec) = make_uint4(c[0], c[1], c[2], c[3]);
            } else {
                // two 16-byte halves; the odd pixel of a pair stores them in the other order (distinct banks)
                const bool sw = i & 1;
                const uint4 lo4 = make_uint4(c[0], c[1], c[2], c[3]), hi4 = make_uint4(c[4], c[5], c[6], c[7]);
                *reinterpret_cast<uint4 *>(rec + (sw ? 16 : 0)) = sw ? hi4 : lo4;
                *reinterpret_cast<uint4 *>(rec + (sw ? 0 : 16)) = sw ? lo4 : hi4;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_sync(kBarCost, kCostThreads);  // records staged
        if (tid == 0) {
            const int npx = min(kM, W - x0);
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                             cost + ((size_t)y * W + x0) * DP),
                         "r"(smem_addr(O)), "r"(npx * DP)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int DP, int KB, bool RAGGED>
cudaError_t launch_dp(const void *codes, int W, int H, int D, int nbits, uint8_t *cost, unsigned *job_state,
                      unsigned *status, int stall_test, cudaStream_t s) {
    auto kernel = hamming_mma_kernel<DP, KB, RAGGED>;
    // More than half an SM's shared memory: two CTAs never share an SM (the
    // second would wait in tcgen05.alloc until the first had finished).
    const int smem = Smem<DP, KB>::kBytes > kOneCtaPerSm ? Smem<DP, KB>::kBytes : kOneCtaPerSm;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long nseg = (long long)((W + kM - 1) / kM) * H;
    const int grid = nseg < sms ? (int)nseg : sms;
    return launch_k(kernel, dim3(grid), dim3(kThreads), (size_t)smem, s, (const uint32_t *)codes, W, H, D, nbits,
                    cost, job_state, status, stall_test);
}

template <int KB>
cudaError_t launch_kb(const void *codes, int W, int H, int D, int nbits, uint8_t *cost, unsigned *job_state,
                      unsigned *status, int stall_test, cudaStream_t s) {
    const int Dp = padded_disparities(D);
    const bool rag = D != Dp;
#define SGM_MMA(P)                                                                                 \
    return rag ? launch_dp<P, KB, true>(codes, W, H, D, nbits, cost, job_state, status, stall_test, s) \
               : launch_dp<P, KB, false>(codes, W, H, D, nbits, cost, job_state, status, stall_test, s)
    switch (Dp) {
        case 32: SGM_MMA(32);
        case 64: SGM_MMA(64);
        case 128: SGM_MMA(128);
        default: return cudaErrorInvalidValue;
    }
#undef SGM_MMA
}

}  // namespace

bool cost_mma_supported(int D) {
    const int Dp = padded_disparities(D);
    return disparities_per_lane(D) == 8 && (Dp == 32 || Dp == 64 || Dp == 128);
}

cudaError_t launch_cost_mma(const void *codes, int code_bytes, int W, int H, int D, int nbits, uint8_t *cost,
                            unsigned *job_state, unsigned *status, cudaStream_t s, int stall_test) {
    if (!cost_mma_supported(D) || nbits < 0 || nbits > 8 * code_bytes) return cudaErrorInvalidValue;
    if (W <= 0 || H <= 0) return cudaSuccess;
    if (code_bytes == 4) return launch_kb<32>(codes, W, H, D, nbits, cost, job_state, status, stall_test, s);
    if (code_bytes == 8) return launch_kb<64>(codes, W, H, D, nbits, cost, job_state, status, stall_test, s);
    return cudaErrorInvalidValue;
}

}  // namespace sgm
