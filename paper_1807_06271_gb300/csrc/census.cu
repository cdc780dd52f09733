// Census transform of both images of a pair (Sec. 3.1.2).
//
// One CTA covers a 32 x 8 pixel tile of one image (blockIdx.z selects left or
// right).  The tile and its (cw-1)/2, (ch-1)/2 halo are staged once in shared
// memory as 16-bit values with 256 standing for "outside the image", which is
// never darker than a centre pixel and so yields the 0 bit the border rule
// asks for.  Each thread then builds its pixel's code from shared memory.
// Bit k of a code is set iff the k-th window neighbour (raster order, centre
// skipped) is darker than the centre.  Codes of up to 32 bits are stored as
// uint32, longer ones as uint64.  HBM traffic: 1 byte read + 4/8 bytes
// written per pixel and image.
#include <type_traits>

#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kBX = 32, kBY = 8;
constexpr int kRows = 4;  // rows per thread of the unrolled census kernel

// One CTA covers 32 x 32 pixels of one image; a thread computes the pixels
// of kRows consecutive rows of one column.  The tile plus halo is staged as
// bytes with 255 for "outside the image": 255 is never darker than a centre
// pixel, which gives the 0 bit the border rule asks for.  Each bit is the
// sign of I(q) - I(p), shifted into one of two 32-bit halves (two
// instructions per bit).  The thread's windows overlap: it walks the
// kRows + CH - 1 tile rows it touches from the bottom up, loads each row's CW
// bytes once, and appends them to every pixel whose window holds that row;
// every pixel thus receives its window backwards, so the first neighbour in
// raster order ends at bit 0.
template <typename CodeT, int CW, int CH, bool RECT>
__global__ void __launch_bounds__(kBX *kBY)
    census_kernel(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch,
                  int W, int H, CodeT *__restrict__ codes, RectMaps maps) {
    wait_for_predecessor();
    constexpr int TW = kBX + CW - 1, TH = kBY * kRows + CH - 1;
    constexpr int RX = CW / 2, RY = CH / 2;
    constexpr int NB = CW * CH - 1;  // bits per code
    __shared__ uint8_t tile[TH][TW];
    const uint8_t *img = blockIdx.z ? right : left;
    const uint16_t *mx = blockIdx.z ? maps.rx : maps.lx, *my = blockIdx.z ? maps.ry : maps.ly;
    const int x0 = blockIdx.x * kBX - RX, y0 = blockIdx.y * kBY * kRows - RY;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    // All of a thread's tile loads are issued before any is stored, so their
    // latencies overlap instead of adding up.
    constexpr int kLoads = (TW * TH + kBX * kBY - 1) / (kBX * kBY);
    uint8_t v[kLoads];
#pragma unroll
    for (int k = 0; k < kLoads; k++) {
        const int i = tid + k * kBX * kBY;
        const int ty = i / TW, tx = i - ty * TW;
        const int gx = x0 + tx, gy = y0 + ty;
        v[k] = (i < TW * TH && gx >= 0 && gx < W && gy >= 0 && gy < H)
                   ? rect_pixel<RECT>(img, pitch, W, H, gx, gy, mx, my)
                   : 255;
    }
#pragma unroll
    for (int k = 0; k < kLoads; k++) {
        const int i = tid + k * kBX * kBY;
        if (i < TW * TH) tile[i / TW][i % TW] = v[k];
    }
    __syncthreads();
    const int x = blockIdx.x * kBX + threadIdx.x;
    if (x >= W) return;
    const int ly0 = threadIdx.y * kRows;  // first tile row of the thread's windows
    int c[kRows];
    uint32_t lo[kRows], hi[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        c[r] = tile[ly0 + r + RY][threadIdx.x + RX];
        lo[r] = hi[r] = 0u;
    }
#pragma unroll
    for (int t = kRows + CH - 2; t >= 0; t--) {  // tile row ly0 + t, bottom up
        int q[CW];
#pragma unroll
        for (int wx = 0; wx < CW; wx++) q[wx] = tile[ly0 + t][threadIdx.x + wx];
#pragma unroll
        for (int r = 0; r < kRows; r++) {
            const int wy = t - r;  // window row of tile row t for pixel r
            if (wy < 0 || wy >= CH) continue;
#pragma unroll
            for (int wx = CW - 1; wx >= 0; wx--) {
                if (wy == RY && wx == RX) continue;
                // bit index of neighbour (wy, wx) in raster order, centre skipped
                const int bit = wy * CW + wx - (wy * CW + wx > RY * CW + RX ? 1 : 0);
                const uint32_t diff = (uint32_t)(q[wx] - c[r]);
                if (bit >= 32) hi[r] = __funnelshift_l(diff, hi[r], 1);
                else lo[r] = __funnelshift_l(diff, lo[r], 1);
            }
        }
    }
    static_assert(NB <= 64, "codes hold at most 64 bits");
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const int y = blockIdx.y * kBY * kRows + ly0 + r;
        if (y >= H) break;
        CodeT code;
        if constexpr (sizeof(CodeT) == 8) code = ((uint64_t)hi[r] << 32) | lo[r];
        else code = lo[r];
        const long long ci = (long long)blockIdx.z * W * H + (long long)y * W + x;
        if (in_range(ci, 2LL * W * H)) codes[ci] = code;
    }
}

// Generic window (any odd size up to 64 bits), loops not unrolled.
template <typename CodeT, bool RECT>
__global__ void __launch_bounds__(kBX *kBY)
    census_kernel_any(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch,
                      int W, int H, int cw, int ch, CodeT *__restrict__ codes, RectMaps maps) {
    wait_for_predecessor();
    extern __shared__ uint16_t tile_any[];
    const int TW = kBX + cw - 1, TH = kBY + ch - 1;
    const int rx = cw / 2, ry = ch / 2;
    const uint8_t *img = blockIdx.z ? right : left;
    const uint16_t *mx = blockIdx.z ? maps.rx : maps.lx, *my = blockIdx.z ? maps.ry : maps.ly;
    const int x0 = blockIdx.x * kBX - rx, y0 = blockIdx.y * kBY - ry;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (int i = tid; i < TW * TH; i += kBX * kBY) {
        int ty = i / TW, tx = i - ty * TW;
        int gx = x0 + tx, gy = y0 + ty;
        tile_any[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H)
                          ? (uint16_t)rect_pixel<RECT>(img, pitch, W, H, gx, gy, mx, my)
                          : (uint16_t)256;
    }
    __syncthreads();
    const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint16_t c = tile_any[(threadIdx.y + ry) * TW + threadIdx.x + rx];
    CodeT code = 0;
    int bit = 0;
    for (int wy = 0; wy < ch; wy++)
        for (int wx = 0; wx < cw; wx++) {
            if (wy == ry && wx == rx) continue;
            code |= (CodeT)(tile_any[(threadIdx.y + wy) * TW + threadIdx.x + wx] < c) << bit;
            bit++;
        }
    const long long ci = (long long)blockIdx.z * W * H + (long long)y * W + x;
    if (in_range(ci, 2LL * W * H)) codes[ci] = code;
}

// ---------------------------------------------------------------------------
// Matching cost volume (Eq. 1): C(x,y,d) = popc(code_l(x,y) ^ code_r(x-d,y)),
// or the code width when x-d < 0, for d < D; padding slots d >= D hold the
// code width too.  One CTA per segment of kSeg pixels of one row: the
// segment's left codes and the right codes it reaches (kSeg + Dp + 2 of them)
// are staged in shared memory.  A thread computes one DPL-disparity chunk of
// two neighbouring pixels from DPL + 1 consecutive right codes read as
// aligned vectors, with consecutive threads on consecutive pixel pairs
// (conflict-free reads); the segment is transposed through a padded shared
// tile and written out with coalesced DPL-byte stores (the segment's Dp-byte
// pixel records are contiguous in global memory).  popc runs on the XU pipe
// (16 per SM per clock; two per estimate for 64-bit codes), which bounds
// this kernel.
// ---------------------------------------------------------------------------

// 2 warps per 32-pixel segment: each thread computes 4 chunks for D = 128
// (measured on GB300 against 64-pixel segments: 256 threads 37.8 us, 128
// threads 35.6 us, this 35.0 us on the 1242 x 375, D = 128 cost volume).
constexpr int kCostThreads = 64, kSeg = 32;

__device__ __forceinline__ uint32_t popcnt(uint32_t v) { return __popc(v); }
__device__ __forceinline__ uint32_t popcnt(uint64_t v) { return __popcll(v); }

// Bytes of one chunk word: word w of a lane holds disparities 2w, 2w+1, 2w+h, 2w+1+h
// (h = DPL/2) in its bytes 0..3, the order in which the aggregation unpacks them.
template <int DPL>
__device__ __forceinline__ void pack_chunk(const uint32_t (&c)[DPL], uint32_t (&w)[DPL / 4]) {
    constexpr int h = DPL / 2;
#pragma unroll
    for (int i = 0; i < DPL / 4; i++)
        w[i] = (c[2 * i + 1 + h] * 256u + c[2 * i + h]) * 65536u + (c[2 * i + 1] * 256u + c[2 * i]);
}

template <int DPL>
__device__ __forceinline__ void st_shared_chunk(uint8_t *p, const uint32_t (&w)[DPL / 4]) {
    if constexpr (DPL == 8) *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <typename CodeT, int DPL, bool RAGGED>
__global__ void __launch_bounds__(kCostThreads)
    cost_kernel(const CodeT *__restrict__ codes, int W, int H, int D, int Dp, int nbits,
                uint8_t *__restrict__ cost, unsigned *__restrict__ job_state) {
    wait_for_predecessor();
    if (job_state && blockIdx.x == 0 && blockIdx.y == 0)
        for (int i = threadIdx.x; i < (int)(kJobStateBytes / sizeof(unsigned)); i += kCostThreads) job_state[i] = 0u;
    using VecT = typename std::conditional<DPL == 8, uint2, uint4>::type;
    extern __shared__ __align__(16) unsigned char cost_smem[];
    const int stride = Dp + DPL;  // padded tile row (bytes)
    uint8_t *tile = cost_smem;                                          // [kSeg][stride]
    const int tile_bytes = (kSeg * stride + 15) & ~15;
    CodeT *cl = reinterpret_cast<CodeT *>(cost_smem + tile_bytes);     // [kSeg]
    CodeT *cr = cl + kSeg;                                              // [kSeg + Dp + 2]
    const int y = blockIdx.y, x0 = blockIdx.x * kSeg;
    const int xr0 = x0 - Dp - 1;  // right code cr[i] is column xr0 + i
    const CodeT *rowl = codes + (size_t)y * W;
    const CodeT *rowr = codes + (size_t)W * H + (size_t)y * W;
    for (int i = threadIdx.x; i < kSeg; i += kCostThreads)
        cl[i] = x0 + i < W && in_range((long long)y * W + x0 + i, (long long)W * H) ? rowl[x0 + i] : 0;
    for (int i = threadIdx.x; i < kSeg + Dp + 2; i += kCostThreads) {
        const int xr = xr0 + i;
        cr[i] = (xr >= 0 && xr < W && in_range((long long)W * H + (long long)y * W + xr, 2LL * W * H)) ? rowr[xr] : 0;
    }
    __syncthreads();
    const int chunks = Dp / DPL;
    const bool border = x0 < Dp;  // only the first segments see x - d < 0
    // A thread takes one DPL-disparity chunk i of the pixel pair (px, px+1), px even.
    // Column x - d of pixel px sits at cr[px - d + Dp + 1]: for the chunk's
    // disparities DPL*i + j the pair needs the DPL + 1 codes w[k] = cr[s + k],
    // s = px + Dp + 2 - DPL*(i + 1) (even, so the run is 16-byte aligned for
    // 8-byte codes; 2 <= s and s + DPL <= kSeg + Dp): pixel px uses
    // w[DPL - 1 - j], pixel px + 1 uses w[DPL - j].
    // A thread's pixel pair is the same for all its chunks (kCostThreads is a
    // multiple of kSeg / 2), so its two left codes are read once.
    static_assert(kCostThreads % (kSeg / 2) == 0, "one pixel pair per thread");
    const int px = 2 * (threadIdx.x % (kSeg / 2));
    CodeT a0, a1;
    if constexpr (sizeof(CodeT) == 8) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(cl + px);
        a0 = v.x;
        a1 = v.y;
    } else {
        const uint2 v = *reinterpret_cast<const uint2 *>(cl + px);
        a0 = v.x;
        a1 = v.y;
    }
    for (int it = threadIdx.x; it < (kSeg / 2) * chunks; it += kCostThreads) {
        const int i = it / (kSeg / 2);
        const int sidx = px + Dp + 2 - DPL * (i + 1);
        CodeT w[DPL + 1];
#pragma unroll
        for (int k = 0; k < DPL / 2; k++) {
            if constexpr (sizeof(CodeT) == 8) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(cr + sidx + 2 * k);
                w[2 * k] = v.x;
                w[2 * k + 1] = v.y;
            } else {
                const uint2 v = *reinterpret_cast<const uint2 *>(cr + sidx + 2 * k);
                w[2 * k] = v.x;
                w[2 * k + 1] = v.y;
            }
        }
        w[DPL] = cr[sidx + DPL];
        uint32_t c[DPL], e[DPL];
#pragma unroll
        for (int j = 0; j < DPL; j++) {
            c[j] = popcnt(a0 ^ w[DPL - 1 - j]);
            e[j] = popcnt(a1 ^ w[DPL - j]);
        }
        if (RAGGED || border) {
            const int x = x0 + px;
#pragma unroll
            for (int j = 0; j < DPL; j++) {
                const int d = DPL * i + j;
                if ((RAGGED && d >= D) || x - d < 0) c[j] = (uint32_t)nbits;
                if ((RAGGED && d >= D) || x + 1 - d < 0) e[j] = (uint32_t)nbits;
            }
        }
        uint32_t vc[DPL / 4], ve[DPL / 4];
        pack_chunk<DPL>(c, vc);
        pack_chunk<DPL>(e, ve);
        st_shared_chunk<DPL>(tile + px * stride + DPL * i, vc);
        st_shared_chunk<DPL>(tile + (px + 1) * stride + DPL * i, ve);
    }
    __syncthreads();
    const int npx = min(kSeg, W - x0);
    uint8_t *out = cost + ((size_t)y * W + x0) * Dp;
    for (int k = threadIdx.x; k < npx * chunks; k += kCostThreads) {
        const int px = k / chunks, q = k - px * chunks;
        // a record of DPL bytes starting at byte o of the W x H x Dp volume
        const long long o = ((long long)y * W + x0 + px) * Dp + DPL * q;
        if (in_range(o, (long long)W * H * Dp - DPL + 1))
            *reinterpret_cast<VecT *>(out + (size_t)px * Dp + DPL * q) =
                *reinterpret_cast<const VecT *>(tile + px * stride + DPL * q);
    }
}

}  // namespace

cudaError_t launch_census(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int cw, int ch, int code_bytes, void *codes, const RectMaps &maps,
                          cudaStream_t s) {
    dim3 block(kBX, kBY), grid((W + kBX - 1) / kBX, (H + kBY - 1) / kBY, 2);
    const dim3 grid4((W + kBX - 1) / kBX, (H + kBY * kRows - 1) / (kBY * kRows), 2);
    const bool rect = maps.lx != nullptr;
#define SGM_CENSUS(T, CWv, CHv)                                                                                     \
    (rect ? launch_k(census_kernel<T, CWv, CHv, true>, grid4, block, 0, s, left, right, pitch, W, H, (T *)codes, maps) \
          : launch_k(census_kernel<T, CWv, CHv, false>, grid4, block, 0, s, left, right, pitch, W, H, (T *)codes, maps))
    if (cw == 5 && ch == 5 && code_bytes == 4) return SGM_CENSUS(uint32_t, 5, 5);
    if (cw == 9 && ch == 7 && code_bytes == 8) return SGM_CENSUS(uint64_t, 9, 7);
#undef SGM_CENSUS
    const size_t smem = (size_t)(kBX + cw - 1) * (kBY + ch - 1) * sizeof(uint16_t);
    if (code_bytes == 4) {
        uint32_t *c = (uint32_t *)codes;
        return rect ? launch_k(census_kernel_any<uint32_t, true>, grid, block, smem, s, left, right, pitch, W, H, cw, ch, c, maps)
                    : launch_k(census_kernel_any<uint32_t, false>, grid, block, smem, s, left, right, pitch, W, H, cw, ch, c, maps);
    }
    uint64_t *c = (uint64_t *)codes;
    return rect ? launch_k(census_kernel_any<uint64_t, true>, grid, block, smem, s, left, right, pitch, W, H, cw, ch, c, maps)
                : launch_k(census_kernel_any<uint64_t, false>, grid, block, smem, s, left, right, pitch, W, H, cw, ch, c, maps);
}

SGM_GUARD_COUNTER(guard_hits_census)

}  // namespace sgm

namespace sgm {

// The CUDA-core kernel measured faster than the tensor-core one on GB300 for
// every D the latter supports (1242 x 375, D = 128: 37.7 against 41.0 us).
int cost_kernel_for(int) { return SGM_COST_KERNEL_CUDA_CORES; }

cudaError_t launch_cost(const void *codes, int code_bytes, int W, int H, int D, int nbits,
                        uint8_t *cost, unsigned *job_state, unsigned *status, int kernel, cudaStream_t s) {
    if (kernel == SGM_COST_KERNEL_AUTO) kernel = cost_kernel_for(D);
    if (kernel == SGM_COST_KERNEL_TENSOR_CORES)
        return launch_cost_mma(codes, code_bytes, W, H, D, nbits, cost, job_state, status, s);
    if (kernel != SGM_COST_KERNEL_CUDA_CORES) return cudaErrorInvalidValue;
    const int Dp = padded_disparities(D), dpl = disparities_per_lane(D);
    const size_t smem = (((size_t)kSeg * (Dp + dpl) + 15) & ~(size_t)15) + (size_t)(2 * kSeg + Dp + 2) * code_bytes;
    const dim3 grid((W + kSeg - 1) / kSeg, H);
    cudaError_t e;
    const bool rag = D != Dp;
#define SGM_COST(T, P, R)                                                                                        \
    do {                                                                                                         \
        e = cudaFuncSetAttribute(cost_kernel<T, P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                          \
        e = launch_k(cost_kernel<T, P, R>, grid, dim3(kCostThreads), smem, s, (const T *)codes, W, H, D, Dp,   \
                     nbits, cost, job_state);                                                                    \
        if (e != cudaSuccess) return e;                                                                          \
    } while (0)
#define SGM_COST2(T, P)                \
    do {                               \
        if (rag) SGM_COST(T, P, true); \
        else SGM_COST(T, P, false);    \
    } while (0)
    if (dpl != 8) return cudaErrorInvalidValue;
    if (code_bytes == 4) SGM_COST2(uint32_t, 8);
    else SGM_COST2(uint64_t, 8);
#undef SGM_COST2
#undef SGM_COST
    return cudaGetLastError();
}

}  // namespace sgm
