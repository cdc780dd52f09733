"""The fused streaming sweep (SGM_SCHEDULE_SWEEP) against the CPU oracle.

The sweep computes the matching cost, the paths of the paper's streaming set
(Sec. 3.1.3, Fig. 2), S, both winners and the LR check in one top-down pass;
its raw left/right maps, its checked map and the median-filtered result must
equal the oracle's bit for bit, for every subset of the streaming set, ragged
and full disparity ranges, 32- and 64-bit codes, single rows and columns,
and each rows-per-block setting (which moves the hand-overs between thread
blocks)."""
import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes, sgm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_pair(W, H, seed):
    rng = scenes.Rng(seed)
    left = rng.integers(0, 255, W * H).astype(np.uint8).reshape(H, W)
    right = np.roll(left, 3, axis=1) // 2 + rng.integers(0, 127, W * H).astype(np.uint8).reshape(H, W)
    return left, right


def run_sweep(left, right, D, p, rows):
    H, W = left.shape
    with sgm.Handle(W, H, D, p) as h:
        sgm.sgm_set_schedule(h, sgm.SGM_SCHEDULE_SWEEP, rows)
        assert sgm.sgm_get_schedule(h) == (sgm.SGM_SCHEDULE_SWEEP, rows)
        L, R = cuda(left), cuda(right)
        dl, dr, lr = (torch.full((H, W), 77, dtype=torch.uint8, device="cuda") for _ in range(3))
        sgm.sgm_debug_raw(h, L, R, dl, dr, lr)
        disp = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
        h.compute(L, R, disp)
        torch.cuda.synchronize()
        assert sgm.sgm_device_status(h) == sgm.SGM_OK
        return dl.cpu().numpy(), dr.cpu().numpy(), lr.cpu().numpy(), disp.cpu().numpy()


def check(left, right, D, cw, ch, mask, P1, P2, tol, k, rows):
    p = sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=P1, P2=P2, lr_tolerance=tol, median_k=k)
    dl, dr, lr, disp = run_sweep(left, right, D, p, rows)
    ref = oracle.sgm(left, right, D, cw, ch, mask, P1, P2, tol, k, stages=True, uv=False)
    for name, got in (("DL", dl), ("DR", dr), ("lr", lr), ("disp", disp)):
        want = ref[name]
        if not np.array_equal(got, want):
            bad = np.argwhere(got != want)
            y, x = bad[0]
            raise AssertionError(f"{name} differs at {len(bad)} pixels, first (y={y}, x={x}): "
                                 f"got {got[y, x]} want {want[y, x]}")


# W, H, D, window, mask, P1, P2, LR tol, median, rows per block
CASES = [
    (160, 48, 60, (5, 5), 0x55, 8, 32, 1, 5, 4),      # the paper's set, ragged D (Dp 64)
    (160, 48, 64, (5, 5), 0x55, 8, 32, 1, 5, 2),      # full D = 64
    (128, 40, 128, (9, 7), 0x55, 8, 96, 1, 3, 8),     # 64-bit codes, D = 128
    (133, 37, 100, (9, 7), 0x55, 8, 96, 0, 0, 4),     # ragged everything, tolerance 0, no median
    (97, 29, 65, (5, 5), 0x55, 10, 40, -1, 3, 2),     # D just past 64, LR check off
    (70, 33, 7, (3, 3), 0x55, 2, 6, 1, 1, 8),         # small D
    (64, 20, 1, (5, 5), 0x55, 8, 32, 1, 0, 4),        # one disparity
    (90, 30, 32, (5, 5), 0x01, 8, 32, 1, 0, 2),       # horizontal only: rows independent
    (90, 30, 32, (5, 5), 0x04, 8, 32, 1, 0, 4),       # vertical only
    (90, 30, 32, (5, 5), 0x10, 8, 32, 1, 0, 4),       # 45 degrees only
    (90, 30, 32, (5, 5), 0x40, 8, 32, 1, 0, 8),       # 135 degrees only
    (90, 30, 48, (5, 5), 0x05, 8, 32, 1, 3, 2),       # L->R and T->B
    (90, 30, 48, (5, 5), 0x50, 8, 32, 1, 3, 4),       # both diagonals
    (90, 30, 48, (7, 5), 0x15, 8, 32, 2, 5, 8),       # three of four
    (1, 23, 16, (5, 5), 0x55, 8, 32, 1, 3, 2),        # a single column
    (200, 1, 64, (5, 5), 0x55, 8, 32, 1, 3, 2),       # a single row
    (3, 3, 8, (3, 3), 0x55, 8, 32, 1, 3, 4),          # smaller than a block of rows
    (257, 9, 128, (9, 7), 0x55, 8, 96, 1, 3, 2),      # W past a multiple of the rings' slots
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}d{c[2]}m{c[4]:02x}r{c[9]}" for c in CASES])
def test_sweep_matches_oracle(case):
    W, H, D, (cw, ch), mask, P1, P2, tol, k, rows = case
    left, right = random_pair(W, H, seed=W * 31 + H * 7 + D)
    check(left, right, D, cw, ch, mask, P1, P2, tol, k, rows)


@pytest.mark.parametrize("rows", [2, 4, 8])
def test_sweep_on_a_scene_at_each_block_size(rows):
    s = scenes.boxes_scene(240, 100, 60, seed=1807 + rows, n_boxes=4, dlo=4, dhi=56)
    check(s.left, s.right, 60, 5, 5, 0x55, 8, 32, 1, 5, rows)


def test_sweep_full_size_paper_setting():
    """The paper's own setting: 640x360, D = 60, 5x5 census, the streaming set,
    P1 = 8, P2 = 32, LR tolerance 1, 5x5 median (one CTA boundary every few rows)."""
    w = scenes.PAPER_640
    s = scenes.scene_for(w, scenes.workload_seed(5, 0))
    for rows in (2, 8):
        check(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol, w.median_k, rows)


def test_sweep_equals_planes_and_the_tuner_keeps_results():
    """Both schedules give the same maps, and sgm_autotune (which now also
    tries the sweep) leaves the results unchanged whichever it picks."""
    w = scenes.PAPER_640
    s = scenes.scene_for(w, 77)
    p = sgm.SgmParams(census_w=5, census_h=5, path_mask=0x55, P1=8, P2=32, lr_tolerance=1, median_k=5)
    L, R = cuda(s.left), cuda(s.right)
    outs = []
    with sgm.Handle(w.W, w.H, w.D, p) as h:
        for sched in (sgm.SGM_SCHEDULE_PLANES, sgm.SGM_SCHEDULE_SWEEP):
            sgm.sgm_set_schedule(h, sched, 4)
            d = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
            h.compute(L, R, d)
            outs.append(d)
        d = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
        sgm.sgm_autotune(h, L, R, d)
        sched, rows = sgm.sgm_get_schedule(h)
        assert sched in (sgm.SGM_SCHEDULE_PLANES, sgm.SGM_SCHEDULE_SWEEP)
        h.compute(L, R, d)
        outs.append(d)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_sweep_is_refused_where_it_does_not_apply():
    with sgm.Handle(64, 32, 32, sgm.SgmParams(census_w=5, census_h=5, path_mask=0xFF, P1=8, P2=32)) as h:
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_schedule(h, sgm.SGM_SCHEDULE_SWEEP, 4)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
        assert sgm.sgm_get_schedule(h)[0] == sgm.SGM_SCHEDULE_PLANES
    with sgm.Handle(64, 32, 200, sgm.SgmParams(census_w=5, census_h=5, path_mask=0x55, P1=8, P2=32)) as h:
        with pytest.raises(sgm.SgmError):
            sgm.sgm_set_schedule(h, sgm.SGM_SCHEDULE_SWEEP, 4)   # D > 128
    with sgm.Handle(64, 32, 32, sgm.SgmParams(census_w=5, census_h=5, path_mask=0x55, P1=8, P2=32)) as h:
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_schedule(h, sgm.SGM_SCHEDULE_SWEEP, 9)
        assert e.value.status == sgm.SGM_ERR_INVALID_ARG


def test_sweep_wait_that_runs_out_is_reported_and_the_handle_recovers():
    """The fused sweep's bounded waits: with row 1 waiting for a pixel that is
    never published, the wait gives up after 2 ms, every other row stops, the
    timeout is reported once, and the next frames are bit-exact again."""
    W, H, D = 160, 48, 60
    s = scenes.boxes_scene(W, H, D, seed=5, n_boxes=3, dlo=4, dhi=56)
    p = sgm.SgmParams(census_w=5, census_h=5, path_mask=0x55, P1=8, P2=32, lr_tolerance=1, median_k=5)
    ref = oracle.sgm(s.left, s.right, D, 5, 5, 0x55, 8, 32, 1, 5, uv=False)
    with sgm.Handle(W, H, D, p) as h:
        sgm.sgm_set_schedule(h, sgm.SGM_SCHEDULE_SWEEP, 4)
        L, R = cuda(s.left), cuda(s.right)
        sgm.sgm_debug_stalled_wait(h, L, R)
        assert sgm.sgm_device_status(h) == sgm.SGM_ERR_TIMEOUT
        assert sgm.sgm_device_status(h) == sgm.SGM_OK  # reported once
        for _ in range(2):
            d = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            h.compute(L, R, d)
            torch.cuda.synchronize()
            assert np.array_equal(d.cpu().numpy(), ref["disp"])
        assert sgm.sgm_device_status(h) == sgm.SGM_OK
