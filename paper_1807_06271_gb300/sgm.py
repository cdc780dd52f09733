"""Python binding of libsgm (ctypes).  Argument marshalling only: every step
of the method runs in the CUDA library; there is no CPU fallback.

Device buffers are torch CUDA tensors (uint8 images and disparities, uint16
maps, int64/uint64 census codes); the stream defaults to torch's current
stream.  Function names follow the C ABI in ``include/sgm.h``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import build as _build

SGM_OK = 0
SGM_ERR_INVALID_ARG = 1
SGM_ERR_UNSUPPORTED = 2
SGM_ERR_OOM = 3
SGM_ERR_CUDA = 4
SGM_ERR_TIMEOUT = 5
SGM_ERR_OVERRUN = 6
SGM_INVALID = 0xFF

SGM_PATHS_4 = 0x0F
SGM_PATHS_8 = 0xFF
SGM_PATHS_STREAM4 = 0x55
SGM_COST_CENSUS = 0  # Hamming distance of census codes over the window
SGM_COST_SAD = 1  # sum of absolute differences over the window (16-bit path costs)

# Kernels of the census Hamming cost (bit-identical results)
SGM_COST_KERNEL_AUTO = 0  # the faster one on GB300 (CUDA cores)
SGM_COST_KERNEL_CUDA_CORES = 1  # POPC of the XOR of two codes, any D
SGM_COST_KERNEL_TENSOR_CORES = 2  # +-1 inner products on tcgen05 (17 <= D <= 128)

STAGES = ("census", "cost", "aggregate", "wta_lr", "median", "uvmap", "sweep")

# Path schedules (see sgm_set_schedule in include/sgm.h)
SGM_SCHEDULE_AUTO = 0
SGM_SCHEDULE_PLANES = 1  # independent scanlines over a cost volume, one plane per direction
SGM_SCHEDULE_SWEEP = 2  # the paper's streaming set in one fused top-down sweep
SGM_AGG_CHUNKS_MIXED = 3  # sgm_set_aggregation: rows at 1 chunk per lane, other directions at 2


class SgmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class _Params(ctypes.Structure):
    _fields_ = [("census_w", ctypes.c_int), ("census_h", ctypes.c_int),
                ("path_mask", ctypes.c_int), ("P1", ctypes.c_int), ("P2", ctypes.c_int),
                ("lr_tolerance", ctypes.c_int), ("median_k", ctypes.c_int),
                ("row_pitch", ctypes.c_int), ("cost", ctypes.c_int)]


@dataclass
class SgmParams:
    census_w: int = 5
    census_h: int = 5
    path_mask: int = SGM_PATHS_8
    P1: int = 8
    P2: int = 32
    lr_tolerance: int = 1
    median_k: int = 5
    row_pitch: int = 0
    cost: int = SGM_COST_CENSUS

    def _c(self) -> _Params:
        return _Params(self.census_w, self.census_h, self.path_mask, self.P1, self.P2,
                       self.lr_tolerance, self.median_k, self.row_pitch, self.cost)


class _UvPost(ctypes.Structure):
    _fields_ = [("u_threshold", ctypes.c_int), ("v_threshold", ctypes.c_int),
                ("u_roi", ctypes.c_int * 4), ("v_roi", ctypes.c_int * 4), ("dilate_r", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int

_SIGNATURES = {
    "sgm_create": [_I, _I, _I, ctypes.POINTER(_Params), ctypes.POINTER(_P)],
    "sgm_destroy": [_P],
    "sgm_compute": [_P, _P, _P, _P, _P],
    "uvmap_compute": [_P, _P, _P, _P, _P],
    "sgm_compute_host": [_P, _P, _P, _P, _P, _P, _P],
    "sgm_compute_host_async": [_P, _P, _P, _P, _P, _P, _P, _P],
    "sgm_host_wait": [_P, ctypes.c_ulonglong],
    "sgm_batch_compute": [_I, _P, _P, _P, _P, _P, _P, _P],
    "sgm_get_shape": [_P, _P, _P, _P, _P],
    "sgm_debug_census": [_P, _P, _P, _P, _P, _P],
    "sgm_debug_path": [_P, _I, _P, _P, _P, _P],
    "sgm_debug_sum": [_P, _P, _P, _P, _P],
    "sgm_debug_raw": [_P, _P, _P, _P, _P, _P, _P],
    "sgm_set_timing": [_P, _I],
    "sgm_get_stage_times": [_P, _P, _P, _I, _P],
    "sgm_compute_static": [_I, _I, _I, ctypes.POINTER(_Params), _P, _P, _P, _P],
    "sgm_autotune": [_P, _P, _P, _P, _P, _P],
    "uvmap_postprocess": [_P, _P, _P, ctypes.POINTER(_UvPost), _P, _P, _P],
    "sgm_set_rectification": [_P, _P, _P, _P, _P],
    "sgm_debug_cost": [_P, _P, _P, _I, _P, _P],
    "sgm_set_cost_kernel": [_P, _I],
    "sgm_device_status": [_P],
    "sgm_debug_stalled_wait": [_P, _P, _P, _P],
    "sgm_debug_guard_hits": [ctypes.POINTER(ctypes.c_ulonglong), _I],
    "sgm_debug_fail_alloc": [_I],
    "sgm_debug_canaries": [_I],
    "sgm_debug_check_canaries": [_P],
    "sgm_debug_poke_canary": [_P, _I],
    "sgm_scratch_bytes": [_I, _I, _I, ctypes.POINTER(_Params), _P, _P, _P],
    "sgm_probe_int_rate": [_I, _I, _P, _P],
    "sgm_set_schedule": [_P, _I, _I],
    "sgm_set_aggregation": [_P, _I, _I],
    "sgm_get_aggregation": [_P, _P, _P],
    "sgm_batch_create": [_I, _P, _P, _P, ctypes.POINTER(_Params), ctypes.POINTER(_P)],
    "sgm_batch_destroy": [_P],
    "sgm_batch_run": [_P, _P, _P, _P, _P, _P, _P],
    "sgm_batch_set_tuning": [_P, _I, _I, _I],
    "sgm_batch_get_tuning": [_P, _P, _P, _P],
    "sgm_batch_autotune": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "sgm_batch_device_bytes": [_P, _P],
    "sgm_get_schedule": [_P, _P, _P],
}

SGM_STATIC_SCRATCH_BYTES = 32 << 20

# operation mixes of sgm_probe_int_rate
SGM_PROBE_INT32_ADD_MIN = 0
SGM_PROBE_U16X2_MIN_ADD = 1
SGM_PROBE_POPC_XOR = 2


def library_path() -> str:
    """libsgm.so, or the build named by SGM_LIBRARY (a test variant of this
    library such as libsgm_guarded.so; it must exist, nothing falls back)."""
    return os.environ.get("SGM_LIBRARY") or _build.LIB


def load(build_if_missing: bool = True):
    """Load libsgm.so (building it with nvcc when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and "SGM_LIBRARY" not in os.environ and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsgm.so not found at {path}; build it with "
                           "`python -m paper_1807_06271_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sgm_status_string.argtypes = [_I]
    lib.sgm_status_string.restype = ctypes.c_char_p
    lib.sgm_stage_name.argtypes = [_I]
    lib.sgm_stage_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().sgm_status_string(status).decode()


def _check(rc: int, what: str):
    if rc != SGM_OK:
        raise SgmError(rc, what)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype_names, shape, what):
    """Pointer of a contiguous CUDA tensor with the expected dtype and size."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what}: expected a CUDA tensor")
    if str(t.dtype).replace("torch.", "") not in dtype_names:
        raise ValueError(f"{what}: dtype {t.dtype} not in {dtype_names}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t.data_ptr()


class Handle:
    """Owns one sgm_handle (W x H images, D disparities, fixed parameters)."""

    def __init__(self, W: int, H: int, D: int, params: SgmParams | None = None):
        self.W, self.H, self.D = W, H, D
        self.params = params or SgmParams()
        self._h = sgm_create(W, H, D, self.params)

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            sgm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _img_shape(self):
        pitch = self.params.row_pitch or self.W
        return (self.H, pitch)

    def compute(self, left, right, disp, stream=None):
        sgm_compute(self, left, right, disp, stream)

    def uvmap(self, disp, umap, vmap, stream=None):
        uvmap_compute(self, disp, umap, vmap, stream)


def _hptr(h):
    return h.ptr if isinstance(h, Handle) else h


def sgm_create(W: int, H: int, D: int, params: SgmParams):
    out = _P()
    p = params._c()
    _check(load().sgm_create(W, H, D, ctypes.byref(p), ctypes.byref(out)), "sgm_create")
    return out.value


def sgm_destroy(h):
    _check(load().sgm_destroy(_hptr(h)), "sgm_destroy")


def sgm_compute(h: Handle, left, right, disp, stream=None):
    shp = h._img_shape()
    _check(load().sgm_compute(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(disp, ("uint8",), (h.H, h.W), "disp"), _stream(stream)), "sgm_compute")


def uvmap_compute(h: Handle, disp, umap, vmap, stream=None):
    _check(load().uvmap_compute(
        h.ptr, _dev(disp, ("uint8",), (h.H, h.W), "disp"),
        _dev(umap, ("uint16", "int16"), (h.D, h.W), "umap"),
        _dev(vmap, ("uint16", "int16"), (h.H, h.D), "vmap"), _stream(stream)), "uvmap_compute")


def _host(t, nbytes, what):
    """Pointer of a host buffer (numpy array or CPU tensor) of nbytes bytes."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if t.is_cuda or not t.is_contiguous() or t.numel() * t.element_size() != nbytes:
            raise ValueError(f"{what}: expected a contiguous host tensor of {nbytes} bytes")
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"] or t.nbytes != nbytes:
        raise ValueError(f"{what}: expected a contiguous array of {nbytes} bytes")
    return t.ctypes.data


def sgm_compute_host(h: Handle, left, right, disp, umap=None, vmap=None, stream=None):
    npx = h.W * h.H
    _check(load().sgm_compute_host(
        h.ptr, _host(left, npx, "left"), _host(right, npx, "right"), _host(disp, npx, "disp"),
        _host(umap, 2 * h.D * h.W, "umap"), _host(vmap, 2 * h.H * h.D, "vmap"),
        _stream(stream)), "sgm_compute_host")


def sgm_compute_host_async(h: Handle, left, right, disp, umap=None, vmap=None, stream=None) -> int:
    """Queue one frame from host buffers (pinned); returns its ticket.  The
    buffers belong to the frame until sgm_host_wait(h, ticket) returns."""
    npx = h.W * h.H
    t = ctypes.c_ulonglong()
    _check(load().sgm_compute_host_async(
        h.ptr, _host(left, npx, "left"), _host(right, npx, "right"), _host(disp, npx, "disp"),
        _host(umap, 2 * h.D * h.W, "umap"), _host(vmap, 2 * h.H * h.D, "vmap"),
        _stream(stream), ctypes.byref(t)), "sgm_compute_host_async")
    return t.value


def sgm_host_wait(h: Handle, ticket: int):
    _check(load().sgm_host_wait(h.ptr, ctypes.c_ulonglong(ticket)), "sgm_host_wait")


def sgm_batch_compute(handles, lefts, rights, disps, umaps=None, vmaps=None, stream=None):
    n = len(handles)
    arr = lambda T, xs: (T * n)(*xs)
    hs = arr(_P, [h.ptr for h in handles])
    L = arr(_P, [_dev(t, ("uint8",), h._img_shape(), "left") for h, t in zip(handles, lefts)])
    R = arr(_P, [_dev(t, ("uint8",), h._img_shape(), "right") for h, t in zip(handles, rights)])
    Dd = arr(_P, [_dev(t, ("uint8",), (h.H, h.W), "disp") for h, t in zip(handles, disps)])
    U = V = None
    if umaps is not None:
        U = arr(_P, [_dev(t, ("uint16", "int16"), (h.D, h.W), "umap") if t is not None else None
                     for h, t in zip(handles, umaps)])
        V = arr(_P, [_dev(t, ("uint16", "int16"), (h.H, h.D), "vmap") if t is not None else None
                     for h, t in zip(handles, vmaps)])
    _check(load().sgm_batch_compute(n, hs, L, R, Dd, U, V, _stream(stream)), "sgm_batch_compute")


def sgm_autotune(h: Handle, left, right, disp, stream=None) -> int:
    """Pick the aggregation kernel's resident blocks per SM for h's shape by
    timing the pipeline on this pair; returns the chosen value."""
    shp = h._img_shape()
    best = _I()
    _check(load().sgm_autotune(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(disp, ("uint8",), (h.H, h.W), "disp"), _stream(stream), ctypes.byref(best)),
        "sgm_autotune")
    return best.value


def sgm_get_shape(h: Handle):
    W, H, D, B = _I(), _I(), _I(), _I()
    _check(load().sgm_get_shape(h.ptr, ctypes.byref(W), ctypes.byref(H), ctypes.byref(D),
                                ctypes.byref(B)), "sgm_get_shape")
    return W.value, H.value, D.value, B.value


def sgm_debug_census(h: Handle, left, right, codes_left, codes_right, stream=None):
    shp = h._img_shape()
    _check(load().sgm_debug_census(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(codes_left, ("int64", "uint64"), (h.H, h.W), "codes_left"),
        _dev(codes_right, ("int64", "uint64"), (h.H, h.W), "codes_right"), _stream(stream)),
        "sgm_debug_census")


def sgm_debug_path(h: Handle, r: int, left, right, L, stream=None):
    shp = h._img_shape()
    _check(load().sgm_debug_path(
        h.ptr, r, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(L, ("uint16", "int16"), (h.H, h.W, h.D), "L"), _stream(stream)), "sgm_debug_path")


def sgm_debug_cost(h: Handle, left, right, C, kernel: int = SGM_COST_KERNEL_AUTO, stream=None):
    """Matching cost C (H x W x D uint16) from the given cost kernel."""
    shp = h._img_shape()
    _check(load().sgm_debug_cost(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"), kernel,
        _dev(C, ("uint16", "int16"), (h.H, h.W, h.D), "C"), _stream(stream)), "sgm_debug_cost")


class Batch:
    """Owns one sgm_batch: n pairs of sizes shapes[i] = (W, H, D), one set of
    parameters, one pooled device allocation (see sgm_batch_* in sgm.h)."""

    def __init__(self, shapes, params: SgmParams | None = None):
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.params = params or SgmParams()
        n = len(self.shapes)
        Ws = (ctypes.c_int * n)(*[sh[0] for sh in self.shapes])
        Hs = (ctypes.c_int * n)(*[sh[1] for sh in self.shapes])
        Ds = (ctypes.c_int * n)(*[sh[2] for sh in self.shapes])
        p = self.params._c()
        out = _P()
        _check(load().sgm_batch_create(n, Ws, Hs, Ds, ctypes.byref(p), ctypes.byref(out)), "sgm_batch_create")
        self._b = out.value

    @property
    def ptr(self):
        return self._b

    def close(self):
        if self._b:
            load().sgm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _arrays(self, left, right, disp, umap, vmap):
        n = len(self.shapes)
        if not (len(left) == len(right) == len(disp) == n):
            raise ValueError("one left, right and disp tensor per pair")
        L = (_P * n)(*[_dev(t, ("uint8",), (H, W), "left") for t, (W, H, D) in zip(left, self.shapes)])
        R = (_P * n)(*[_dev(t, ("uint8",), (H, W), "right") for t, (W, H, D) in zip(right, self.shapes)])
        O = (_P * n)(*[_dev(t, ("uint8",), (H, W), "disp") for t, (W, H, D) in zip(disp, self.shapes)])
        if umap is None:
            return L, R, O, None, None
        U = (_P * n)(*[_dev(t, ("uint16", "int16"), (D, W), "umap") for t, (W, H, D) in zip(umap, self.shapes)])
        V = (_P * n)(*[_dev(t, ("uint16", "int16"), (H, D), "vmap") for t, (W, H, D) in zip(vmap, self.shapes)])
        return L, R, O, U, V

    def run(self, left, right, disp, umap=None, vmap=None, stream=None):
        _check(load().sgm_batch_run(self._b, *self._arrays(left, right, disp, umap, vmap), _stream(stream)),
               "sgm_batch_run")

    def set_tuning(self, groups: int, blocks_per_sm: int, chunks_per_lane: int = 1):
        _check(load().sgm_batch_set_tuning(self._b, groups, blocks_per_sm, chunks_per_lane), "sgm_batch_set_tuning")

    def tuning(self):
        """(groups, blocks_per_sm, chunks_per_lane)"""
        g, b, c = _I(), _I(), _I()
        _check(load().sgm_batch_get_tuning(self._b, ctypes.byref(g), ctypes.byref(b), ctypes.byref(c)),
               "sgm_batch_get_tuning")
        return g.value, b.value, c.value

    def autotune(self, left, right, disp, umap=None, vmap=None, stream=None):
        """(groups, blocks_per_sm, chunks_per_lane) chosen."""
        g, b, c = _I(), _I(), _I()
        _check(load().sgm_batch_autotune(self._b, *self._arrays(left, right, disp, umap, vmap), _stream(stream),
                                         ctypes.byref(g), ctypes.byref(b), ctypes.byref(c)), "sgm_batch_autotune")
        return g.value, b.value, c.value

    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(load().sgm_batch_device_bytes(self._b, ctypes.byref(v)), "sgm_batch_device_bytes")
        return v.value


def sgm_batch_create(shapes, params: SgmParams | None = None) -> Batch:
    return Batch(shapes, params)


def sgm_batch_destroy(b: Batch):
    b.close()


def sgm_batch_run(b: Batch, left, right, disp, umap=None, vmap=None, stream=None):
    b.run(left, right, disp, umap, vmap, stream)


def sgm_batch_set_tuning(b: Batch, groups: int, blocks_per_sm: int, chunks_per_lane: int = 1):
    b.set_tuning(groups, blocks_per_sm, chunks_per_lane)


def sgm_batch_get_tuning(b: Batch):
    return b.tuning()


def sgm_batch_autotune(b: Batch, left, right, disp, umap=None, vmap=None, stream=None):
    return b.autotune(left, right, disp, umap, vmap, stream)


def sgm_batch_device_bytes(b: Batch) -> int:
    return b.device_bytes()


def sgm_set_aggregation(h: Handle, blocks_per_sm: int, chunks_per_lane: int):
    """Aggregation kernel shape of later calls on h (see sgm.h)."""
    _check(load().sgm_set_aggregation(h.ptr, blocks_per_sm, chunks_per_lane), "sgm_set_aggregation")


def sgm_get_aggregation(h: Handle):
    """(blocks_per_sm, chunks_per_lane) in use on h."""
    a, b = _I(), _I()
    _check(load().sgm_get_aggregation(h.ptr, ctypes.byref(a), ctypes.byref(b)), "sgm_get_aggregation")
    return a.value, b.value


def sgm_set_schedule(h: Handle, schedule: int, rows_per_cta: int = 4):
    """Path schedule of later calls on h (SGM_SCHEDULE_*)."""
    _check(load().sgm_set_schedule(h.ptr, schedule, rows_per_cta), "sgm_set_schedule")


def sgm_get_schedule(h: Handle):
    """(schedule, rows_per_cta) in use on h."""
    a, b = _I(), _I()
    _check(load().sgm_get_schedule(h.ptr, ctypes.byref(a), ctypes.byref(b)), "sgm_get_schedule")
    return a.value, b.value


def sgm_set_cost_kernel(h: Handle, kernel: int):
    _check(load().sgm_set_cost_kernel(h.ptr, kernel), "sgm_set_cost_kernel")


def sgm_device_status(h: Handle) -> int:
    """SGM_OK, or SGM_ERR_TIMEOUT if a bounded device wait of h gave up since the last call."""
    return load().sgm_device_status(h.ptr)


def sgm_debug_stalled_wait(h: Handle, left, right, stream=None):
    """Runs the tensor-core cost kernel with a wait that runs out (see sgm.h)."""
    shp = h._img_shape()
    _check(load().sgm_debug_stalled_wait(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"), _stream(stream)),
        "sgm_debug_stalled_wait")


def sgm_debug_guard_hits(reset: bool = False) -> int:
    """Index-check hits of a guarded build since the last reset (see sgm.h);
    SgmError(SGM_ERR_UNSUPPORTED) in the default build."""
    v = ctypes.c_ulonglong()
    _check(load().sgm_debug_guard_hits(ctypes.byref(v), 1 if reset else 0), "sgm_debug_guard_hits")
    return v.value


def sgm_debug_fail_alloc(n: int):
    """The n-th device allocation of the library from now on fails (0: none)."""
    _check(load().sgm_debug_fail_alloc(n), "sgm_debug_fail_alloc")


def sgm_debug_canaries(on: bool):
    """Handles created while on guard their device buffers with canary bytes."""
    _check(load().sgm_debug_canaries(1 if on else 0), "sgm_debug_canaries")


def sgm_debug_check_canaries(h: Handle) -> int:
    """SGM_OK, or SGM_ERR_OVERRUN if a guard byte of h changed."""
    return load().sgm_debug_check_canaries(h.ptr)


def sgm_debug_poke_canary(h: Handle, i: int):
    _check(load().sgm_debug_poke_canary(h.ptr, i), "sgm_debug_poke_canary")


def sgm_debug_sum(h: Handle, left, right, S, stream=None):
    shp = h._img_shape()
    _check(load().sgm_debug_sum(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(S, ("uint16", "int16"), (h.H, h.W, h.D), "S"), _stream(stream)), "sgm_debug_sum")


def sgm_debug_raw(h: Handle, left, right, disp_left=None, disp_right=None, disp_lr=None,
                  stream=None):
    shp = h._img_shape()
    px = (h.H, h.W)
    _check(load().sgm_debug_raw(
        h.ptr, _dev(left, ("uint8",), shp, "left"), _dev(right, ("uint8",), shp, "right"),
        _dev(disp_left, ("uint8",), px, "disp_left"), _dev(disp_right, ("uint8",), px, "disp_right"),
        _dev(disp_lr, ("uint8",), px, "disp_lr"), _stream(stream)), "sgm_debug_raw")


def sgm_set_timing(h: Handle, enable: bool):
    _check(load().sgm_set_timing(h.ptr, 1 if enable else 0), "sgm_set_timing")


def sgm_get_stage_times(h: Handle):
    """{stage: (total_ms, launches)} since the previous read."""
    n = len(STAGES)
    ms = (ctypes.c_float * n)()
    cnt = (ctypes.c_int * n)()
    ns = _I()
    _check(load().sgm_get_stage_times(h.ptr, ms, cnt, n, ctypes.byref(ns)), "sgm_get_stage_times")
    return {STAGES[i]: (ms[i], cnt[i]) for i in range(min(n, ns.value))}


def sgm_compute_static(W: int, H: int, D: int, params: SgmParams, left, right, disp, stream=None):
    """sgm_compute without a handle or any device allocation (scratch in a fixed
    device array of SGM_STATIC_SCRATCH_BYTES per GPU).  left, right and disp
    must live on one GPU; the call runs there.  Calls that overlap on the GPU
    race on that array; the first call on a device must not be made inside a
    stream capture."""
    shp = (H, params.row_pitch or W)
    devs = {t.device for t in (left, right, disp) if t is not None and getattr(t, "is_cuda", False)}
    if len(devs) > 1:
        raise ValueError(f"sgm_compute_static: left, right and disp are on different devices {sorted(map(str, devs))}")
    p = params._c()
    args = (W, H, D, ctypes.byref(p), _dev(left, ("uint8",), shp, "left"),
            _dev(right, ("uint8",), shp, "right"), _dev(disp, ("uint8",), (H, W), "disp"))
    import torch
    with torch.cuda.device(left.device):
        _check(load().sgm_compute_static(*args, _stream(stream)), "sgm_compute_static")


def sgm_probe_int_rate(kind: int, iters: int = 20000):
    """(lane instructions per second, launch ms) of the integer probe kernel
    for one operation mix (SGM_PROBE_*) on the current device."""
    r, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().sgm_probe_int_rate(kind, iters, ctypes.byref(r), ctypes.byref(ms)), "sgm_probe_int_rate")
    return r.value, ms.value


def sgm_scratch_bytes(W: int, H: int, D: int, params: SgmParams):
    """(handle_bytes, host_staging_bytes, static_bytes): the device memory
    sgm_create allocates, what the host-buffer entry points add, and what
    sgm_compute_static would use of its fixed array (no device call)."""
    p = params._c()
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().sgm_scratch_bytes(W, H, D, ctypes.byref(p), ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)), "sgm_scratch_bytes")
    return a.value, b.value, c.value


def uvmap_postprocess(h: Handle, umap, vmap, u_threshold: int, v_threshold: int, u_roi=None,
                      v_roi=None, dilate_r: int = 1, uout=None, vout=None, stream=None):
    """Thresholded, dilated and Gaussian-smoothed U-/V-maps (uint8) of Sec. 3.2."""
    u_roi = u_roi or (0, h.D, 0, h.W)
    v_roi = v_roi or (0, h.H, 0, h.D)
    p = _UvPost(u_threshold, v_threshold, (ctypes.c_int * 4)(*u_roi), (ctypes.c_int * 4)(*v_roi),
                dilate_r)
    _check(load().uvmap_postprocess(
        h.ptr, _dev(umap, ("uint16", "int16"), (h.D, h.W), "umap"),
        _dev(vmap, ("uint16", "int16"), (h.H, h.D), "vmap"), ctypes.byref(p),
        _dev(uout, ("uint8",), (h.D, h.W), "uout"), _dev(vout, ("uint8",), (h.H, h.D), "vout"),
        _stream(stream)), "uvmap_postprocess")


def sgm_set_rectification(h: Handle, left_x=None, left_y=None, right_x=None, right_y=None):
    """Rectify the inputs of later calls through integer maps (device uint16/int16
    tensors, H x W; keep them alive while h uses them); no arguments switch it off."""
    shp = (h.H, h.W)
    _check(load().sgm_set_rectification(
        h.ptr, _dev(left_x, ("uint16", "int16"), shp, "left_x"), _dev(left_y, ("uint16", "int16"), shp, "left_y"), _dev(right_x, ("uint16", "int16"), shp, "right_x"),
        _dev(right_y, ("uint16", "int16"), shp, "right_y")), "sgm_set_rectification")
    h._rect = (left_x, left_y, right_x, right_y)  # keep the tensors alive
