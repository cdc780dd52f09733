"""The no-allocation entry point against the handle-based one.

sgm_compute_static serves callers that cannot call cudaMalloc (a hard-deadline
camera loop, a host framework that owns all device memory); it keeps its
scratch in one fixed device array per GPU.  Its results must equal
sgm_compute's bit for bit, also on consecutive calls that reuse the array
with different image sizes and parameters, and a call must allocate no
device memory.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes, sgm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

CASES = [
    # W, H, D, window, path mask, P1, P2, LR tol, median, cost
    (320, 240, 64, (5, 5), sgm.SGM_PATHS_4, 4, 24, 1, 5, sgm.SGM_COST_CENSUS),
    (200, 150, 32, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3, sgm.SGM_COST_CENSUS),
    (160, 120, 48, (5, 5), sgm.SGM_PATHS_STREAM4, 200, 800, 1, 5, sgm.SGM_COST_SAD),
]


def _run_both(W, H, D, cw_ch, mask, P1, P2, tol, k, cost, seed):
    s = scenes.boxes_scene(W, H, D, seed=seed, n_boxes=3, dlo=2, dhi=D - 2)
    p = sgm.SgmParams(census_w=cw_ch[0], census_h=cw_ch[1], path_mask=mask, P1=P1, P2=P2,
                      lr_tolerance=tol, median_k=k, cost=cost)
    left = torch.from_numpy(s.left).cuda()
    right = torch.from_numpy(s.right).cuda()
    want = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    with sgm.Handle(W, H, D, p) as h:
        h.compute(left, right, want)
    got = torch.full((H, W), 7, dtype=torch.uint8, device="cuda")
    sgm.sgm_compute_static(W, H, D, p, left, right, got)
    torch.cuda.synchronize()
    return s, p, got.cpu().numpy(), want.cpu().numpy()


def test_static_matches_handle_path_on_consecutive_calls():
    for i, case in enumerate(CASES + CASES[:1]):
        s, p, got, want = _run_both(*case, seed=90 + i)
        assert np.array_equal(got, want), f"call {i}: differs from sgm_compute"
        ref = oracle.sgm(s.left, s.right, case[2], p.census_w, p.census_h, p.path_mask, p.P1, p.P2,
                         p.lr_tolerance, p.median_k, uv=False, cost=p.cost)
        assert np.array_equal(got, ref["disp"]), f"call {i}: differs from the oracle"


def test_static_rejects_scratch_beyond_its_maximum():
    w = scenes.KITTI_1242  # 8 planes of 1242*375*128 bytes: far above the static maximum
    p = sgm.SgmParams(census_w=9, census_h=7, path_mask=w.path_mask, P1=8, P2=96,
                      lr_tolerance=1, median_k=3)
    left = torch.zeros((w.H, w.W), dtype=torch.uint8, device="cuda")
    disp = torch.zeros((w.H, w.W), dtype=torch.uint8, device="cuda")
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute_static(w.W, w.H, w.D, p, left, left, disp)
    assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
    pc = p._c()
    assert sgm.load().sgm_compute_static(w.W, w.H, w.D, ctypes.byref(pc), None, None, None,
                                         None) == sgm.SGM_ERR_INVALID_ARG


def test_static_allocates_nothing():
    """With the library's next device allocation set to fail, the static call
    still succeeds, and the device's free memory is the same before and after
    it (outputs and inputs are allocated up front)."""
    W, H, D = 320, 240, 64
    s = scenes.boxes_scene(W, H, D, seed=97, n_boxes=3, dlo=2, dhi=D - 2)
    p = sgm.SgmParams(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_4, P1=4, P2=24,
                      lr_tolerance=1, median_k=5)
    left = torch.from_numpy(s.left).cuda()
    right = torch.from_numpy(s.right).cuda()
    got = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    sgm.sgm_compute_static(W, H, D, p, left, right, got)  # first call: device address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sgm.sgm_debug_fail_alloc(1)
    try:
        for _ in range(2):
            sgm.sgm_compute_static(W, H, D, p, left, right, got)
        torch.cuda.synchronize()
    finally:
        sgm.sgm_debug_fail_alloc(0)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = oracle.sgm(s.left, s.right, D, 5, 5, p.path_mask, p.P1, p.P2, p.lr_tolerance, p.median_k, uv=False)
    assert np.array_equal(got.cpu().numpy(), ref["disp"])


def test_static_without_median_on_a_side_stream():
    """median_k = 1 (the LR map is copied out) and a tolerance of 0, on a
    non-default stream, twice in a row: equal to the handle path and the oracle."""
    W, H, D = 256, 200, 48
    p = sgm.SgmParams(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_8, P1=8, P2=32,
                      lr_tolerance=0, median_k=1)
    st = torch.cuda.Stream()
    for seed in (101, 102):
        s = scenes.boxes_scene(W, H, D, seed=seed, n_boxes=3, dlo=2, dhi=D - 2)
        left = torch.from_numpy(s.left).cuda()
        right = torch.from_numpy(s.right).cuda()
        want = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        with sgm.Handle(W, H, D, p) as h:
            h.compute(left, right, want)
        torch.cuda.synchronize()
        got = torch.full((H, W), 7, dtype=torch.uint8, device="cuda")
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            sgm.sgm_compute_static(W, H, D, p, left, right, got, st)
        st.synchronize()
        assert np.array_equal(got.cpu().numpy(), want.cpu().numpy())
        ref = oracle.sgm(s.left, s.right, D, 5, 5, p.path_mask, p.P1, p.P2, 0, 1, uv=False)
        assert np.array_equal(got.cpu().numpy(), ref["disp"])


def test_static_rejects_a_host_buffer():
    W, H, D = 64, 32, 16
    p = sgm.SgmParams(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_4)
    img = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    host = torch.zeros((H, W), dtype=torch.uint8).pin_memory()
    pc = p._c()
    rc = sgm.load().sgm_compute_static(W, H, D, ctypes.byref(pc), img.data_ptr(), img.data_ptr(),
                                       host.data_ptr(), None)
    assert rc == sgm.SGM_ERR_INVALID_ARG
