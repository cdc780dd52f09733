// sgm_compute_static: the disparity path for one small pair without any
// device allocation.
//
// Some callers cannot call cudaMalloc.  Examples: a camera loop with a hard
// per-frame deadline, where an allocation can block or fail in mid-flight; a
// host framework that owns all device memory through its own allocator and
// forbids direct cudaMalloc/cudaFree; code that must not add the implicit
// device synchronisation cudaFree brings.  For them the census codes, cost
// volume, path planes and LR map live in one file-scope device array of fixed size,
// reserved when the library's module is loaded on a device and held until
// the process exits.  The kernels are the same ones sgm_compute runs.
#include <mutex>

#include "sgm_internal.cuh"

namespace {

// Scratch shared by every call of sgm_compute_static on a device.
static __device__ __align__(256) unsigned char g_static_scratch[SGM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices];  // device address of g_static_scratch, per device

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol's host-side stand-in).
int scratch_for_current_device(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SGM_ERR_CUDA;
        }
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return SGM_OK;
}

}  // namespace

extern "C" int sgm_compute_static(int W, int H, int D, const sgm_params *params,
                                  const uint8_t *left, const uint8_t *right, uint8_t *disp,
                                  void *stream) {
    if (!left || !right || !disp) return SGM_ERR_INVALID_ARG;
    int rc = sgm::validate_params(W, H, D, params);
    if (rc != SGM_OK) return rc;
    const bool wide = params->cost == SGM_COST_SAD;
    const int nbits = params->census_w * params->census_h - 1;
    const int code_bytes = wide ? 0 : (nbits <= 32 ? 4 : 8);
    const size_t eb = wide ? 2 : 1;  // bytes per cost / path cost
    const int npaths = __builtin_popcount((unsigned)params->path_mask);
    const int Dp = sgm::padded_disparities(D);

    // Scratch layout: codes | cost volume | path planes | job counter | LR map,
    // each 256-byte aligned.
    const size_t npx = (size_t)W * H;
    const size_t codes_off = 0;
    const size_t cost_off = round_up(codes_off + 2 * npx * code_bytes, 256);
    const size_t planes_off = round_up(cost_off + npx * Dp * eb, 256);
    const size_t counter_off = round_up(planes_off + (size_t)npaths * npx * Dp * eb, 256);
    const size_t lr_off = round_up(counter_off + sgm::kJobStateBytes, 256);
    const size_t need = lr_off + npx;
    if (need > (size_t)SGM_STATIC_SCRATCH_BYTES) return SGM_ERR_UNSUPPORTED;

    unsigned char *base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc != SGM_OK) return rc;
    void *codes = base + codes_off;
    uint8_t *cost = base + cost_off;
    uint8_t *planes = base + planes_off;
    unsigned *counter = reinterpret_cast<unsigned *>(base + counter_off);
    uint8_t *disp_lr = base + lr_off;
    const sgm::PathJobs jobs = sgm::make_path_jobs(W, H, D, params->path_mask);

    // Every kernel below overwrites the scratch it later reads, and the cost
    // kernel clears the aggregation's work-queue state, so nothing left by an
    // earlier call needs clearing.
    cudaStream_t s = (cudaStream_t)stream;
    const int pitch = params->row_pitch ? params->row_pitch : W;
    const sgm::RectMaps no_maps{nullptr, nullptr, nullptr, nullptr};
    cudaError_t e;
    if (wide) {
        e = sgm::launch_sad_cost(left, right, pitch, W, H, D, params->census_w, params->census_h, no_maps,
                                 reinterpret_cast<uint16_t *>(cost), counter, s);
    } else {
        e = sgm::launch_census(left, right, pitch, W, H, params->census_w, params->census_h, code_bytes,
                               codes, no_maps, s);
        if (e == cudaSuccess) e = sgm::launch_cost(codes, code_bytes, W, H, D, nbits, cost, counter, nullptr, SGM_COST_KERNEL_AUTO, s);
    }
    if (e == cudaSuccess)
        e = sgm::launch_aggregate(cost, W, H, D, params->P1, params->P2, wide, jobs, planes, npaths,
                                  counter, 2, s);
    if (e == cudaSuccess)
        e = sgm::launch_wta(planes, npaths, W, H, D, wide, params->lr_tolerance, disp_lr, nullptr, nullptr,
                            nullptr, s);
    if (e == cudaSuccess) {
        if (params->median_k <= 1)
            e = cudaMemcpyAsync(disp, disp_lr, npx, cudaMemcpyDeviceToDevice, s);
        else
            e = sgm::launch_median(disp_lr, disp, W, H, params->median_k, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SGM_ERR_CUDA;
    }
    return SGM_OK;
}
