// Issue-rate probe for the integer operations the aggregation and cost
// kernels are built from, so that their roofline is a measured figure on the
// GPU at hand rather than a count of lanes times a nominal clock.
//
// Every thread runs 8 independent dependency chains; each chain alternates
// two operations of different kinds (an add with a minimum, or a packed
// 16-bit minimum with an add), so no two consecutive operations of a chain
// can be merged into one three-input instruction.  With 8 blocks of 256
// threads on every SM the schedulers always have independent work to issue.
#include "sgm_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

template <int KIND>
__device__ __forceinline__ void op_pair(uint32_t &x, uint32_t k, uint32_t m) {
    if constexpr (KIND == SGM_PROBE_INT32_ADD_MIN) {
        asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(k));
        asm volatile("min.u32 %0, %0, %1;" : "+r"(x) : "r"(m));
    } else if constexpr (KIND == SGM_PROBE_U16X2_MIN_ADD) {
        asm volatile("min.u16x2 %0, %0, %1;" : "+r"(x) : "r"(m));
        asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(k));
    } else {  // SGM_PROBE_POPC_XOR: the Hamming cost's two steps
        uint32_t t;
        asm volatile("xor.b32 %0, %1, %2;" : "=r"(t) : "r"(x), "r"(m));
        asm volatile("popc.b32 %0, %1;" : "=r"(x) : "r"(t));
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) probe_kernel(int iters, uint32_t k, uint32_t m, uint32_t *sink) {
    uint32_t x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = threadIdx.x * 977u + c * 131u + blockIdx.x;
    // iters is a multiple of 4 (the launcher rounds it), so the unrolled loop
    // spends about 1 % of its instructions on the loop itself
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) op_pair<KIND>(x[c], k, m);
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) r ^= x[c];
    if (r == 0x9E3779B9u) sink[0] = r;  // keeps the chains live; practically never stored
}

template <int KIND>
cudaError_t time_kind(int blocks, int iters, uint32_t *sink, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        probe_kernel<KIND><<<blocks, kThreads>>>(iters / 8, 0x00030003u, 0x7F007F00u, sink);  // warm-up
        e = cudaEventRecord(a);
    }
    if (e == cudaSuccess) {
        probe_kernel<KIND><<<blocks, kThreads>>>(iters, 0x00030003u, 0x7F007F00u, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

}  // namespace

extern "C" int sgm_probe_int_rate(int kind, int iters, double *lane_ops_per_s, float *ms) {
    if (!lane_ops_per_s || iters < 8 || kind < SGM_PROBE_INT32_ADD_MIN || kind > SGM_PROBE_POPC_XOR)
        return SGM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    const int blocks = sms * kBlocksPerSm;
    iters &= ~3;
    uint32_t *sink = nullptr;  // never written in practice; a small buffer keeps the store legal
    if (cudaMalloc(&sink, 256) != cudaSuccess) {
        cudaGetLastError();
        return SGM_ERR_OOM;
    }
    float t = 0.f;
    cudaError_t e;
    if (kind == SGM_PROBE_INT32_ADD_MIN) e = time_kind<SGM_PROBE_INT32_ADD_MIN>(blocks, iters, sink, &t);
    else if (kind == SGM_PROBE_U16X2_MIN_ADD) e = time_kind<SGM_PROBE_U16X2_MIN_ADD>(blocks, iters, sink, &t);
    else e = time_kind<SGM_PROBE_POPC_XOR>(blocks, iters, sink, &t);
    cudaFree(sink);
    if (e != cudaSuccess || t <= 0.f) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    // two operations per chain step, one lane each
    const double ops = (double)blocks * kThreads * kChains * 2.0 * iters;
    *lane_ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
    return SGM_OK;
}
