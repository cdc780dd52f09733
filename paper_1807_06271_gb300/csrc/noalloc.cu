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

#include "sgm_handle.cuh"

namespace {

// Scratch shared by every call of sgm_compute_static on a device.
static __device__ __align__(256) unsigned char g_static_scratch[SGM_STATIC_SCRATCH_BYTES];

// The device address of g_static_scratch is looked up with the device
// current and cached per (device, context): host code cannot use the
// symbol's host-side stand-in, and a context made again after
// cudaDeviceReset loads the module again, possibly at another address.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchAddr {
    void *ctx;
    unsigned char *addr;
};
ScratchAddr g_scratch[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);
CtxGetCurrentFn g_ctx_get_current = nullptr;  // cuCtxGetCurrent, through the runtime

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The current context of the calling thread, or null where it cannot be read.
void *current_context() {
    if (!g_ctx_get_current) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        g_ctx_get_current = (CtxGetCurrentFn)fn;
    }
    void *ctx = nullptr;
    return g_ctx_get_current(&ctx) == 0 ? ctx : nullptr;
}

// Device address of the scratch array on device dev, which is current.  The
// lookup (cudaGetSymbolAddress, which also makes the device's primary context
// current) runs on the first call on a device and again whenever the current
// context is not the one the cached address belongs to.
int scratch_for_device(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return SGM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr &c = g_scratch[dev];
    void *ctx = current_context();
    if (!c.addr || !ctx || c.ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SGM_ERR_CUDA;
        }
        c.addr = (unsigned char *)p;
        c.ctx = current_context();  // null (not readable): looked up again next call
    }
    *out = c.addr;
    return SGM_OK;
}

// The device that holds p, or -1 when p is not device (or managed) memory.
int device_of(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return -1;
    return a.device;
}

struct DeviceSwitch {
    int prev = -1;
    bool ok = true;
    explicit DeviceSwitch(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
        }
    }
    ~DeviceSwitch() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

sgm::StaticLayout sgm::static_layout(const ScratchSizes &sz) {
    StaticLayout l;
    l.codes = 0;
    l.cost = round_up(l.codes + sz.codes, 256);
    l.planes = round_up(l.cost + sz.cost, 256);
    l.job_state = round_up(l.planes + sz.planes, 256);
    l.disp_lr = round_up(l.job_state + sz.job_state, 256);
    l.end = l.disp_lr + sz.disp_lr;
    return l;
}

extern "C" int sgm_compute_static(int W, int H, int D, const sgm_params *params,
                                  const uint8_t *left, const uint8_t *right, uint8_t *disp,
                                  void *stream) {
    if (!left || !right || !disp) return SGM_ERR_INVALID_ARG;
    int rc = sgm::validate_params(W, H, D, params);
    if (rc != SGM_OK) return rc;
    const sgm::ScratchSizes sz = sgm::scratch_sizes(W, H, D, params);
    const sgm::StaticLayout at = sgm::static_layout(sz);
    if (at.end > (size_t)SGM_STATIC_SCRATCH_BYTES) return SGM_ERR_UNSUPPORTED;

    // The three buffers must be device memory of one device; the call runs on
    // that device, whichever is current.
    const int dev = device_of(left);
    if (dev < 0 || device_of(right) != dev || device_of(disp) != dev) return SGM_ERR_INVALID_ARG;
    DeviceSwitch on(dev);
    if (!on.ok) return SGM_ERR_CUDA;

    const bool wide = params->cost == SGM_COST_SAD;
    const int nbits = params->census_w * params->census_h - 1;
    const int code_bytes = wide ? 0 : (nbits <= 32 ? 4 : 8);
    const int npaths = __builtin_popcount((unsigned)params->path_mask);
    unsigned char *base = nullptr;
    rc = scratch_for_device(dev, &base);
    if (rc != SGM_OK) return rc;
    void *codes = base + at.codes;
    uint8_t *cost = base + at.cost;
    uint8_t *planes = base + at.planes;
    unsigned *counter = reinterpret_cast<unsigned *>(base + at.job_state);
    uint8_t *disp_lr = base + at.disp_lr;
    const int cpl = sgm::chunks_per_lane_max(D, wide);
    const sgm::PathJobs jobs = sgm::make_path_jobs(W, H, D, params->path_mask, cpl);

    // Every kernel below overwrites the scratch it later reads, and the cost
    // kernel clears the aggregation's work-queue state, so nothing left by an
    // earlier call needs clearing.
    cudaStream_t s = (cudaStream_t)stream;
    const int pitch = params->row_pitch ? params->row_pitch : W;
    const sgm::RectMaps no_maps{nullptr, nullptr, nullptr, nullptr};
    const size_t npx = (size_t)W * H;
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
                                  counter, 2, cpl, s);
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
