"""The C-ABI library builds, loads without a GPU, exports every symbol that
include/sgm.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

from paper_1807_06271_gb300 import sgm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?(?:int|char|void)\s*\*?\s*(\w+)\s*\(", text, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sgm_create", "sgm_compute", "uvmap_compute", "sgm_destroy",
                 "sgm_batch_compute", "sgm_status_string", "sgm_debug_path"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = sgm.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    assert sgm.status_string(sgm.SGM_OK) == "ok"
    assert "invalid" in sgm.status_string(sgm.SGM_ERR_INVALID_ARG)
    assert sgm.status_string(999) == "unknown status"


def _create(W, H, D, **kw):
    p = sgm.SgmParams(**kw)._c()
    out = ctypes.c_void_p()
    rc = sgm.load().sgm_create(W, H, D, ctypes.byref(p), ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("W,H,D,kw,want", [
    (0, 10, 16, {}, sgm.SGM_ERR_INVALID_ARG),             # empty image
    (10, 0, 16, {}, sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 0, {}, sgm.SGM_ERR_INVALID_ARG),              # no disparities
    (10, 10, 256, {}, sgm.SGM_ERR_UNSUPPORTED),            # d would collide with 0xFF
    (10, 10, 16, dict(census_w=4), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(census_w=9, census_h=9), sgm.SGM_ERR_UNSUPPORTED),  # 80 bits
    (10, 10, 16, dict(P1=9, P2=8), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(P1=-1), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(census_w=9, census_h=7, P2=200), sgm.SGM_ERR_UNSUPPORTED),  # 62+200 > 255
    (10, 10, 16, dict(path_mask=0), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(path_mask=0x100), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(median_k=4), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(median_k=9), sgm.SGM_ERR_UNSUPPORTED),
    (10, 10, 16, dict(row_pitch=5), sgm.SGM_ERR_INVALID_ARG),
    (9000, 10, 16, {}, sgm.SGM_ERR_UNSUPPORTED),
    (10, 10, 16, dict(cost=2), sgm.SGM_ERR_INVALID_ARG),  # no such cost
    # SAD: (25 * 255 + 800) * 8 paths = 57400 fits 16 bits; with P2 = 2000, 67000 does not
    (10, 10, 16, dict(cost=1, census_w=5, census_h=5, P1=200, P2=2000), sgm.SGM_ERR_UNSUPPORTED),
    # SAD: one path, 11 x 13 window: 36465 + 0 is above the 0x7FFF padding marker
    (10, 10, 16, dict(cost=1, census_w=11, census_h=13, P1=0, P2=0, path_mask=1), sgm.SGM_ERR_UNSUPPORTED),
    (10, 10, 16, dict(cost=1, census_w=17, census_h=1, P1=0, P2=0, path_mask=1), sgm.SGM_ERR_UNSUPPORTED),
    (10, 10, 16, dict(cost=1, census_w=4, census_h=5), sgm.SGM_ERR_INVALID_ARG),  # even window
    (10, 10, 16, dict(census_w=5, census_h=4), sgm.SGM_ERR_INVALID_ARG),
    (10, 10, 16, dict(census_w=-1), sgm.SGM_ERR_INVALID_ARG),
    (1, 65536, 1, dict(path_mask=1), sgm.SGM_ERR_UNSUPPORTED),     # rows index with 16 bits
    (8193, 1, 1, dict(path_mask=1), sgm.SGM_ERR_UNSUPPORTED),
    (10, 10, 16, dict(census_w=9, census_h=7, P1=0, P2=194), sgm.SGM_ERR_UNSUPPORTED),  # 62 + 194 = 256
    (10, 10, 16, dict(cost=1, census_w=5, census_h=5, P1=0, P2=26392, path_mask=1), sgm.SGM_ERR_UNSUPPORTED),
    # 32-bit lane-chunk indices of the planes: 8192 x 65535 x 8 paths x 32 lanes
    (8192, 65535, 255, dict(path_mask=0xFF), sgm.SGM_ERR_UNSUPPORTED),
])
def test_create_rejects_bad_arguments_on_host(W, H, D, kw, want):
    rc, h = _create(W, H, D, **kw)
    assert rc == want and h is None


@pytest.mark.parametrize("W,H,D,kw", [
    (1, 65535, 1, dict(path_mask=1)),                                 # largest height
    (8192, 1, 1, dict(path_mask=1)),                                  # largest width
    (4, 4, 255, {}),                                                  # largest D
    (10, 10, 16, dict(census_w=9, census_h=7, P1=0, P2=193)),         # 62 + 193 = 255
    (10, 10, 16, dict(median_k=7)),
    (10, 10, 16, dict(median_k=0)),
    (10, 10, 16, dict(median_k=1)),
    (10, 10, 16, dict(row_pitch=10)),
    (10, 10, 16, dict(cost=1, census_w=5, census_h=5, P1=0, P2=26391, path_mask=1)),  # 6375 + 26391 = 0x7FFE
    (10, 10, 16, dict(cost=1, census_w=15, census_h=1, P1=0, P2=0, path_mask=1)),     # widest SAD window
    (10, 10, 16, dict(census_w=1, census_h=1, P1=0, P2=0)),                           # 0-bit census
])
def test_create_accepts_the_limits(W, H, D, kw):
    """Values on the accepted side of each limit pass the host checks: without
    a GPU the call then fails at the device query (SGM_ERR_CUDA), with one it
    creates a (small) handle."""
    rc, h = _create(W, H, D, **kw)
    assert rc in (sgm.SGM_OK, sgm.SGM_ERR_CUDA), rc
    if h:
        assert sgm.load().sgm_destroy(h) == sgm.SGM_OK


def test_null_arguments_are_rejected():
    lib = sgm.load()
    assert lib.sgm_create(10, 10, 16, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_host_wait(None, 0) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_compute_host_async(None, None, None, None, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_compute(None, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.uvmap_compute(None, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_destroy(None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_batch_compute(-1, None, None, None, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_batch_compute(0, None, None, None, None, None, None, None) == sgm.SGM_OK
    assert lib.sgm_debug_cost(None, None, None, 0, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_set_cost_kernel(None, 0) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_device_status(None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_debug_stalled_wait(None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_stage_name(0) == b"census"
    assert lib.sgm_stage_name(99) is None


def test_binding_has_the_c_names():
    for n in declared_functions():
        if n in ("sgm_status_string", "sgm_stage_name"):
            continue
        assert hasattr(sgm, n), n


def test_product_code_never_reaches_the_oracle():
    """The package (binding, serving, build, generators) and the CUDA sources
    neither import, include nor load anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1807_06271_gb300")
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#\s*include\s*[<\"].*oracle)|liboracle|oracle[/\\]", re.M)
    checked = 0
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn), encoding="utf-8").read()
                assert not pat.search(text), os.path.join(dirpath, fn)
                checked += 1
    assert checked >= 10


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No fallback: with libsgm.so absent the first call raises."""
    monkeypatch.setattr(sgm, "_lib", None)
    monkeypatch.setattr(sgm, "library_path", lambda: str(tmp_path / "libsgm.so"))
    with pytest.raises(RuntimeError, match="libsgm.so not found"):
        sgm.load(build_if_missing=False)


def _handle_functions():
    """Declared functions whose first parameter is an sgm_handle."""
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
            names += re.findall(r"^\s*int\s+(\w+)\s*\(\s*sgm_handle\s+\w+\s*[,)]", text, re.M)
    return sorted(set(names))


def test_every_handle_entry_point_rejects_a_null_handle():
    """Null handle, zero or null everything else: SGM_ERR_INVALID_ARG before
    any device call (so this runs without a GPU)."""
    lib = sgm.load()
    names = _handle_functions()
    assert len(names) >= 20
    for n in names:
        fn = getattr(lib, n)
        numeric = (ctypes.c_int, ctypes.c_uint, ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_float, ctypes.c_size_t)
        args = [0 if t in numeric else None for t in fn.argtypes]
        assert fn(*args) == sgm.SGM_ERR_INVALID_ARG, n


def test_static_entry_point_checks_before_any_device_call():
    lib = sgm.load()
    bad = sgm.SgmParams(census_w=4)._c()
    assert lib.sgm_compute_static(10, 10, 16, ctypes.byref(bad), None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    good = sgm.SgmParams()._c()
    assert lib.sgm_compute_static(10, 10, 16, ctypes.byref(good), None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_compute_static(10, 10, 16, None, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_debug_fail_alloc(-1) == sgm.SGM_ERR_INVALID_ARG


def test_static_entry_point_rejects_memory_that_is_not_on_a_device():
    """Host buffers (or, on a machine without a GPU, any buffer) are not device
    memory of one device: SGM_ERR_INVALID_ARG, and nothing is launched."""
    lib = sgm.load()
    good = sgm.SgmParams(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_4)._c()
    img = (ctypes.c_uint8 * (32 * 16))()
    out = (ctypes.c_uint8 * (32 * 16))()
    rc = lib.sgm_compute_static(32, 16, 16, ctypes.byref(good), ctypes.addressof(img), ctypes.addressof(img),
                                ctypes.addressof(out), None)
    assert rc == sgm.SGM_ERR_INVALID_ARG


def _expected_bytes(W, H, D, cw, ch, mask, cost):
    """Scratch sizes written out from the layout the header documents."""
    lanes = 1
    while 8 * lanes < D:
        lanes *= 2
    Dp = 8 * lanes
    e = 2 if cost == sgm.SGM_COST_SAD else 1
    code = 0 if cost == sgm.SGM_COST_SAD else (4 if cw * ch - 1 <= 32 else 8)
    npx = W * H
    npaths = bin(mask).count("1")
    parts = [2 * npx * code, npx * Dp * e, npaths * npx * Dp * e, 4224 + 4, npx]
    handle = sum(parts)
    staging = 2 * (3 * npx + 2 * D * W + 2 * H * D)
    at = 0
    for i, b in enumerate((parts[0], parts[1], parts[2], parts[3])):
        at = (at + b + 255) // 256 * 256
    static = at + npx
    return handle, staging, static


@pytest.mark.parametrize("W,H,D,cw,ch,mask,cost", [
    (320, 240, 64, 5, 5, sgm.SGM_PATHS_4, sgm.SGM_COST_CENSUS),
    (1242, 375, 128, 9, 7, sgm.SGM_PATHS_8, sgm.SGM_COST_CENSUS),
    (640, 360, 60, 5, 5, sgm.SGM_PATHS_STREAM4, sgm.SGM_COST_SAD),
    (17, 3, 255, 3, 3, 0x01, sgm.SGM_COST_CENSUS),
])
def test_scratch_bytes_follow_the_documented_layout(W, H, D, cw, ch, mask, cost):
    p = sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=8 if cost == 0 else 200,
                      P2=32 if cost == 0 else 800, cost=cost)
    assert sgm.sgm_scratch_bytes(W, H, D, p) == _expected_bytes(W, H, D, cw, ch, mask, cost)


def test_scratch_bytes_checks_its_arguments():
    lib = sgm.load()
    bad = sgm.SgmParams(census_w=4)._c()
    assert lib.sgm_scratch_bytes(10, 10, 16, ctypes.byref(bad), None, None, None) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_scratch_bytes(10, 10, 16, None, None, None, None) == sgm.SGM_ERR_INVALID_ARG
    big = sgm.SgmParams(census_w=9, census_h=9)._c()
    assert lib.sgm_scratch_bytes(10, 10, 16, ctypes.byref(big), None, None, None) == sgm.SGM_ERR_UNSUPPORTED


def test_static_limit_follows_the_scratch_query():
    """The 320x240, D=64, 4-path workload fits the fixed array; the KITTI-shaped one does not."""
    small = sgm.SgmParams(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_4, P1=4, P2=24)
    big = sgm.SgmParams(census_w=9, census_h=7, path_mask=sgm.SGM_PATHS_8, P1=8, P2=96)
    assert sgm.sgm_scratch_bytes(320, 240, 64, small)[2] <= sgm.SGM_STATIC_SCRATCH_BYTES
    assert sgm.sgm_scratch_bytes(1242, 375, 128, big)[2] > sgm.SGM_STATIC_SCRATCH_BYTES


def test_batch_entry_points_check_their_arguments_on_the_host():
    """Null batch or null arrays: SGM_ERR_INVALID_ARG; bad shapes or
    parameters are refused before anything is allocated (no GPU needed)."""
    lib = sgm.load()
    for name in ("sgm_batch_destroy", "sgm_batch_run", "sgm_batch_set_tuning", "sgm_batch_get_tuning",
                 "sgm_batch_autotune", "sgm_batch_device_bytes"):
        fn = getattr(lib, name)
        args = [0 if t is ctypes.c_int else None for t in fn.argtypes]
        assert fn(*args) == sgm.SGM_ERR_INVALID_ARG, name
    p = sgm.SgmParams(census_w=9, census_h=7, path_mask=0xFF, P1=8, P2=96)._c()
    out = ctypes.c_void_p()
    W, H, D = (ctypes.c_int * 2)(64, 32), (ctypes.c_int * 2)(48, 16), (ctypes.c_int * 2)(64, 300)
    assert lib.sgm_batch_create(2, W, H, D, ctypes.byref(p), ctypes.byref(out)) == sgm.SGM_ERR_UNSUPPORTED
    assert lib.sgm_batch_create(0, W, H, D, ctypes.byref(p), ctypes.byref(out)) == sgm.SGM_ERR_INVALID_ARG
    assert lib.sgm_batch_create(2, W, H, None, ctypes.byref(p), ctypes.byref(out)) == sgm.SGM_ERR_INVALID_ARG
    pitched = sgm.SgmParams(row_pitch=128)._c()
    D2 = (ctypes.c_int * 2)(64, 64)
    assert lib.sgm_batch_create(2, W, H, D2, ctypes.byref(pitched), ctypes.byref(out)) == sgm.SGM_ERR_INVALID_ARG
    assert out.value is None


def test_guard_counter_is_a_guarded_build_feature():
    """The default library has no index checks: sgm_debug_guard_hits says
    so without touching the device."""
    if os.environ.get("SGM_LIBRARY"):
        pytest.skip("another build of the library is selected")
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_debug_guard_hits()
    assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
