"""The no-allocation entry point against the handle-based one.

sgm_compute_static serves callers that cannot call cudaMalloc (a hard-deadline
camera loop, a host framework that owns all device memory); it keeps its
scratch in one fixed device array per GPU.  Its results must equal
sgm_compute's bit for bit, also on consecutive calls that reuse the array
with different image sizes and parameters.  This file is collected last."""
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
