"""CPU oracle for SGM stereo and the U-/V-disparity maps.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library and
its Python binding never import this package; the two implementations share
no code.

The arithmetic lives in ``sgm_oracle.c`` (plain C, integer, stage by stage in
the order of the paper's Sec. 3.1 pipeline and Sec. 3.2 maps); this module
compiles it with gcc and wraps each stage for numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Bit r of a path mask enables direction r (dx, dy); same order as the C table.
DIRECTIONS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (-1, 1), (1, -1)]
PATHS_4 = 0x0F  # left->right, right->left, top->bottom, bottom->top
PATHS_8 = 0xFF  # all eight directions
PATHS_STREAM4 = 0x55  # 0, 45, 90, 135 degrees: the paper's four streaming paths
COST_CENSUS = 0  # Hamming distance of census codes
COST_SAD = 1  # sum of absolute differences over the support window


def build(force: bool = False) -> str:
    """Compile ``sgm_oracle.c`` into ``liboracle.so`` next to it."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_census.argtypes = [P, I, I, I, I, I, P]
        lib.oracle_cost_volume.argtypes = [P, P, I, I, I, I, P]
        lib.oracle_sad_cost_volume.argtypes = [P, P, I, I, I, I, I, I, P]
        lib.oracle_aggregate_path.argtypes = [P, I, I, I, I, I, I, P]
        lib.oracle_sum_paths.argtypes = [P, I, I, I, I, I, I, P]
        lib.oracle_wta_left.argtypes = [P, I, I, I, P]
        lib.oracle_wta_right.argtypes = [P, I, I, I, P]
        lib.oracle_lr_check.argtypes = [P, P, I, I, I, P]
        lib.oracle_median.argtypes = [P, I, I, I, P]
        lib.oracle_uvmap.argtypes = [P, I, I, I, P, P]
        lib.oracle_hamming.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_uv_post.argtypes = [P, I, I, I, I, I, I, I, I, P]
        lib.oracle_rectify.argtypes = [P, I, I, I, P, P, P]
        lib.oracle_sgm.argtypes = [P, P, I, I, I, I, I, I, I, I, I, I, I, I] + [P] * 9
        for name in ("oracle_census", "oracle_cost_volume", "oracle_sad_cost_volume",
                     "oracle_aggregate_path",
                     "oracle_sum_paths", "oracle_wta_left", "oracle_wta_right",
                     "oracle_lr_check", "oracle_median", "oracle_uvmap", "oracle_sgm",
                     "oracle_hamming", "oracle_uv_post", "oracle_rectify"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (status {rc})")


def census_bits(cw: int, ch: int) -> int:
    return cw * ch - 1


def hamming(a: int, b: int) -> int:
    return _load().oracle_hamming(ctypes.c_uint64(a), ctypes.c_uint64(b))


def census(img: np.ndarray, cw: int, ch: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), np.uint64)
    _check(_load().oracle_census(_p(img), W, H, W, cw, ch, _p(out)), "census")
    return out


def cost_volume(cl: np.ndarray, cr: np.ndarray, D: int, nbits: int) -> np.ndarray:
    cl = np.ascontiguousarray(cl, dtype=np.uint64)
    cr = np.ascontiguousarray(cr, dtype=np.uint64)
    H, W = cl.shape
    out = np.empty((H, W, D), np.uint16)
    _check(_load().oracle_cost_volume(_p(cl), _p(cr), W, H, D, nbits, _p(out)), "cost")
    return out


def sad_cost_volume(left: np.ndarray, right: np.ndarray, D: int, ww: int, wh: int) -> np.ndarray:
    """C[y, x, d] = SAD over a ww x wh window (clamped image reads); ww*wh*255 for x < d."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    out = np.empty((H, W, D), np.uint16)
    _check(_load().oracle_sad_cost_volume(_p(left), _p(right), W, H, W, D, ww, wh, _p(out)),
           "sad_cost")
    return out


def aggregate_path(C: np.ndarray, r: int, P1: int, P2: int) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.uint16)
    H, W, D = C.shape
    out = np.empty((H, W, D), np.uint16)
    _check(_load().oracle_aggregate_path(_p(C), W, H, D, r, P1, P2, _p(out)), "path")
    return out


def sum_paths(C: np.ndarray, path_mask: int, P1: int, P2: int) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.uint16)
    H, W, D = C.shape
    out = np.empty((H, W, D), np.uint16)
    _check(_load().oracle_sum_paths(_p(C), W, H, D, path_mask, P1, P2, _p(out)), "sum")
    return out


def wta_left(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.uint16)
    H, W, D = S.shape
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_wta_left(_p(S), W, H, D, _p(out)), "wta_left")
    return out


def wta_right(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.uint16)
    H, W, D = S.shape
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_wta_right(_p(S), W, H, D, _p(out)), "wta_right")
    return out


def lr_check(DL: np.ndarray, DR: np.ndarray, tol: int) -> np.ndarray:
    DL = np.ascontiguousarray(DL, dtype=np.uint8)
    DR = np.ascontiguousarray(DR, dtype=np.uint8)
    H, W = DL.shape
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_lr_check(_p(DL), _p(DR), W, H, tol, _p(out)), "lr_check")
    return out


def median(img: np.ndarray, k: int) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_median(_p(img), W, H, k, _p(out)), "median")
    return out


def uvmap(disp: np.ndarray, D: int):
    disp = np.ascontiguousarray(disp, dtype=np.uint8)
    H, W = disp.shape
    U = np.empty((D, W), np.uint16)
    V = np.empty((H, D), np.uint16)
    _check(_load().oracle_uvmap(_p(disp), W, H, D, _p(U), _p(V)), "uvmap")
    return U, V


def sgm(left: np.ndarray, right: np.ndarray, D: int, census_w: int, census_h: int,
        path_mask: int, P1: int, P2: int, lr_tol: int, median_k: int,
        stages: bool = False, uv: bool = True, cost: int = COST_CENSUS) -> dict:
    """Run the whole path on one pair.  Returns ``disp`` (and U, V when ``uv``);
    with ``stages`` also the census codes (census cost only), S, D_left,
    D_right and the LR map.  census_w x census_h is the support window of
    either cost."""
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    assert right.shape == (H, W)
    out = {"disp": np.empty((H, W), np.uint8)}
    if uv:
        out["U"] = np.empty((D, W), np.uint16)
        out["V"] = np.empty((H, D), np.uint16)
    if stages:
        if cost == COST_CENSUS:
            out["codes_l"] = np.empty((H, W), np.uint64)
            out["codes_r"] = np.empty((H, W), np.uint64)
        out["S"] = np.empty((H, W, D), np.uint16)
        out["DL"] = np.empty((H, W), np.uint8)
        out["DR"] = np.empty((H, W), np.uint8)
        out["lr"] = np.empty((H, W), np.uint8)
    g = out.get
    rc = _load().oracle_sgm(
        _p(left), _p(right), W, H, W, D, census_w, census_h, cost, path_mask, P1, P2,
        lr_tol, median_k, _p(g("codes_l")), _p(g("codes_r")), _p(g("S")),
        _p(g("DL")), _p(g("DR")), _p(g("lr")), _p(out["disp"]), _p(g("U")),
        _p(g("V")))
    _check(rc, "sgm")
    return out


def uv_post(m: np.ndarray, threshold: int, roi=None, dilate_r: int = 1) -> np.ndarray:
    """Binary map of counts >= threshold inside roi = (r0, r1, c0, c1), dilated by a
    (2r+1)^2 square, then 3x3 binomial Gaussian of 255 * binary (uint8)."""
    m = np.ascontiguousarray(m, dtype=np.uint16)
    rows, cols = m.shape
    r0, r1, c0, c1 = roi if roi is not None else (0, rows, 0, cols)
    out = np.empty((rows, cols), np.uint8)
    _check(_load().oracle_uv_post(_p(m), rows, cols, threshold, r0, r1, c0, c1, dilate_r, _p(out)),
           "uv_post")
    return out


def rectify(img: np.ndarray, mx: np.ndarray, my: np.ndarray) -> np.ndarray:
    """I_rect(x, y) = I(mx(x, y), my(x, y)); 0 where the map leaves the image."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    mx = np.ascontiguousarray(mx, dtype=np.uint16)
    my = np.ascontiguousarray(my, dtype=np.uint16)
    out = np.empty((H, W), np.uint8)
    _check(_load().oracle_rectify(_p(img), W, H, W, _p(mx), _p(my), _p(out)), "rectify")
    return out
