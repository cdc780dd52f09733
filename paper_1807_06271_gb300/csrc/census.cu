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
#include "sgm_internal.cuh"

namespace sgm {
namespace {

constexpr int kBX = 32, kBY = 8;

template <typename CodeT, int CW, int CH>
__global__ void __launch_bounds__(kBX *kBY)
    census_kernel(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch,
                  int W, int H, CodeT *__restrict__ codes) {
    constexpr int TW = kBX + CW - 1, TH = kBY + CH - 1;
    constexpr int RX = CW / 2, RY = CH / 2;
    __shared__ uint16_t tile[TH][TW];
    const uint8_t *img = blockIdx.z ? right : left;
    const int x0 = blockIdx.x * kBX - RX, y0 = blockIdx.y * kBY - RY;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (int i = tid; i < TW * TH; i += kBX * kBY) {
        int ty = i / TW, tx = i - ty * TW;
        int gx = x0 + tx, gy = y0 + ty;
        tile[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * pitch + gx] : 256;
    }
    __syncthreads();
    const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint16_t c = tile[threadIdx.y + RY][threadIdx.x + RX];
    CodeT code = 0;
    int bit = 0;
#pragma unroll
    for (int wy = 0; wy < CH; wy++) {
#pragma unroll
        for (int wx = 0; wx < CW; wx++) {
            if (wy == RY && wx == RX) continue;
            code |= (CodeT)(tile[threadIdx.y + wy][threadIdx.x + wx] < c) << bit;
            bit++;
        }
    }
    codes[(size_t)blockIdx.z * W * H + (size_t)y * W + x] = code;
}

// Generic window (any odd size up to 64 bits), loops not unrolled.
template <typename CodeT>
__global__ void __launch_bounds__(kBX *kBY)
    census_kernel_any(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch,
                      int W, int H, int cw, int ch, CodeT *__restrict__ codes) {
    extern __shared__ uint16_t tile_any[];
    const int TW = kBX + cw - 1, TH = kBY + ch - 1;
    const int rx = cw / 2, ry = ch / 2;
    const uint8_t *img = blockIdx.z ? right : left;
    const int x0 = blockIdx.x * kBX - rx, y0 = blockIdx.y * kBY - ry;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (int i = tid; i < TW * TH; i += kBX * kBY) {
        int ty = i / TW, tx = i - ty * TW;
        int gx = x0 + tx, gy = y0 + ty;
        tile_any[i] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * pitch + gx] : 256;
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
    codes[(size_t)blockIdx.z * W * H + (size_t)y * W + x] = code;
}

}  // namespace

cudaError_t launch_census(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int cw, int ch, int code_bytes, void *codes, cudaStream_t s) {
    dim3 block(kBX, kBY), grid((W + kBX - 1) / kBX, (H + kBY - 1) / kBY, 2);
    if (cw == 5 && ch == 5 && code_bytes == 4)
        census_kernel<uint32_t, 5, 5><<<grid, block, 0, s>>>(left, right, pitch, W, H, (uint32_t *)codes);
    else if (cw == 9 && ch == 7 && code_bytes == 8)
        census_kernel<uint64_t, 9, 7><<<grid, block, 0, s>>>(left, right, pitch, W, H, (uint64_t *)codes);
    else {
        size_t smem = (size_t)(kBX + cw - 1) * (kBY + ch - 1) * sizeof(uint16_t);
        if (code_bytes == 4)
            census_kernel_any<uint32_t><<<grid, block, smem, s>>>(left, right, pitch, W, H, cw, ch, (uint32_t *)codes);
        else
            census_kernel_any<uint64_t><<<grid, block, smem, s>>>(left, right, pitch, W, H, cw, ch, (uint64_t *)codes);
    }
    return cudaGetLastError();
}

}  // namespace sgm
