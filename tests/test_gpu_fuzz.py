"""Randomised parity sweep (GPU): seeded draws of shape, disparity range, cost
kind and window, path set, penalties, LR tolerance, median size, Hamming
kernel, row pitch and rectification maps, each compared with the oracle
element by element: the cost volume, the sum S, the final disparity map and
the U-/V-maps, through the device entry points and, for some draws, the
host-buffer one."""
import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes, sgm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u16(t):
    return t.cpu().numpy().view(np.uint16)


def draw_case(seed):
    r = np.random.default_rng(9000 + seed)
    if r.random() < 0.1:  # wide and short, up to the largest width the library takes
        W, H = int(r.integers(1000, 8193)), int(r.integers(1, 9))
    else:
        W, H = int(r.integers(1, 301)), int(r.integers(1, 81))
    D = int(r.integers(1, 256))
    sad = r.random() < 0.3
    mask = int(r.integers(1, 256))
    npaths = bin(mask).count("1")
    while True:
        cw, ch = int(r.choice([1, 3, 5, 7, 9])), int(r.choice([1, 3, 5, 7]))
        if sad:
            cmax = cw * ch * 255
            P2max = min(32766 - cmax, 65535 // npaths - cmax)
            if P2max >= 0:
                break
        elif cw * ch - 1 <= 64:
            P2max = 255 - (cw * ch - 1)
            break
    P2 = int(r.integers(0, P2max + 1))
    P1 = int(r.integers(0, P2 + 1))
    tol = int(r.choice([-1, 0, 1, 2]))
    k = int(r.choice([0, 1, 3, 5, 7]))
    kernel = sgm.SGM_COST_KERNEL_AUTO
    if not sad and 16 < D <= 128 and r.random() < 0.5:
        kernel = sgm.SGM_COST_KERNEL_TENSOR_CORES
    elif not sad:
        kernel = sgm.SGM_COST_KERNEL_CUDA_CORES
    if min(W, H) >= 8 and r.random() < 0.7:
        s = scenes.boxes_scene(W, H, D, seed=seed, n_boxes=3, dlo=min(1, D - 1), dhi=max(1, D - 1))
        left, right = s.left, s.right
    else:
        left = r.integers(0, 256, (H, W)).astype(np.uint8)
        right = np.roll(left, int(r.integers(0, max(1, min(D, W)))), axis=1)
    return W, H, D, sad, cw, ch, mask, P1, P2, tol, k, kernel, left, right


def draw_extras(seed, W, H):
    """Row pitch, rectification maps (or None) and whether to also run the
    host-buffer entry point; from a stream of its own, so that the draws
    above stay as they are."""
    r = np.random.default_rng(19000 + seed)
    pitch = W + int(r.integers(1, 70)) if r.random() < 0.3 else 0
    maps = None
    if r.random() < 0.25:
        y, x = np.mgrid[0:H, 0:W]
        # a mostly smooth warp with a few wild entries, some of them outside the image
        dx = int(r.integers(-3, 4)) + (y // max(1, H // 4)) % 2
        dy = int(r.integers(-2, 3))
        maps = []
        for base, off, n in ((x, 0, W), (y, 0, H), (x, dx, W), (y, dy, H)):
            m = np.clip(base + off, 0, 0xFFFF).astype(np.uint16)
            wild = r.random(m.shape) < 0.02
            m[wild] = r.integers(0, n + 8, int(wild.sum()))
            maps.append(m)
    host = r.random() < 0.3
    return pitch, maps, host


@pytest.mark.parametrize("seed", range(100))
def test_random_configuration_matches_oracle(seed):
    W, H, D, sad, cw, ch, mask, P1, P2, tol, k, kernel, left, right = draw_case(seed)
    pitch, maps, host = draw_extras(seed, W, H)
    cost = sgm.SGM_COST_SAD if sad else sgm.SGM_COST_CENSUS
    p = sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=P1, P2=P2, lr_tolerance=tol,
                      median_k=k, cost=cost, row_pitch=pitch)
    what = (f"W={W} H={H} D={D} {'sad' if sad else 'census'} {cw}x{ch} mask={mask:#x} P={P1}/{P2} tol={tol} "
            f"k={k} kernel={kernel} pitch={pitch} rect={maps is not None} host={host}")
    lo, ro = left, right
    if maps is not None:
        lo, ro = oracle.rectify(left, maps[0], maps[1]), oracle.rectify(right, maps[2], maps[3])
    o = oracle.sgm(lo, ro, D, cw, ch, mask, P1, P2, tol, k, stages=True, cost=cost)
    if sad:
        C_want = oracle.sad_cost_volume(lo, ro, D, cw, ch)
    else:
        C_want = oracle.cost_volume(o["codes_l"], o["codes_r"], D, cw * ch - 1)
    with sgm.Handle(W, H, D, p) as h:
        sgm.sgm_set_cost_kernel(h, kernel)
        if maps is not None:
            dev_maps = [cuda(m.view(np.int16)) for m in maps]
            sgm.sgm_set_rectification(h, *dev_maps)
        if pitch:  # rows of `pitch` bytes, the bytes past W filled with a value the path must not read
            pl, pr = np.full((H, pitch), 77, np.uint8), np.full((H, pitch), 201, np.uint8)
            pl[:, :W], pr[:, :W] = left, right
            L, R = cuda(pl), cuda(pr)
        else:
            L, R = cuda(left), cuda(right)
        C = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        sgm.sgm_debug_cost(h, L, R, C, kernel)
        S = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        sgm.sgm_debug_sum(h, L, R, S)
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        h.compute(L, R, disp)
        U = torch.empty((D, W), dtype=torch.int16, device="cuda")
        V = torch.empty((H, D), dtype=torch.int16, device="cuda")
        h.uvmap(disp, U, V)
        torch.cuda.synchronize()
        assert sgm.sgm_device_status(h) == sgm.SGM_OK, what
        for name, got, want in (("cost", u16(C), C_want), ("S", u16(S), o["S"]), ("disp", disp.cpu().numpy(), o["disp"]),
                                ("U", u16(U), o["U"]), ("V", u16(V), o["V"])):
            assert got.shape == want.shape, (what, name)
            assert np.array_equal(got, want), f"{what}: {name} differs at {np.argwhere(got != want)[:3].tolist()}"
        if host:  # packed host rows (the handle's pitch applies to device inputs only)
            hd = np.empty((H, W), np.uint8)
            hu = np.empty((D, W), np.uint16)
            hv = np.empty((H, D), np.uint16)
            sgm.sgm_compute_host(h, left, right, hd, hu, hv)
            assert sgm.sgm_device_status(h) == sgm.SGM_OK, what
            for name, got, want in (("host disp", hd, o["disp"]), ("host U", hu, o["U"]), ("host V", hv, o["V"])):
                assert np.array_equal(got, want), f"{what}: {name} differs at {np.argwhere(got != want)[:3].tolist()}"
