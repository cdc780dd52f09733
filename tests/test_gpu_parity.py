"""CUDA path vs the CPU oracle, element by element, through the C ABI.

All arithmetic is integer, so every stage must match bit-exactly: census
codes, each path's L_r, the sum S, the left/right winners, the LR-checked map,
the median-filtered map and the U-/V-maps."""
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


def params(cw, ch, mask, P1, P2, tol, k, pitch=0, cost=sgm.SGM_COST_CENSUS):
    return sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=P1, P2=P2,
                         lr_tolerance=tol, median_k=k, row_pitch=pitch, cost=cost)


def gpu_all(left, right, D, p):
    H, W = left.shape
    out = {}
    with sgm.Handle(W, H, D, p) as h:
        L, R = cuda(left), cuda(right)
        if p.cost == sgm.SGM_COST_CENSUS:
            cl = torch.empty((H, W), dtype=torch.int64, device="cuda")
            cr = torch.empty_like(cl)
            sgm.sgm_debug_census(h, L, R, cl, cr)
            out["codes_l"] = cl.cpu().numpy().view(np.uint64)
            out["codes_r"] = cr.cpu().numpy().view(np.uint64)
        out["paths"] = {}
        for r in range(8):
            if (p.path_mask >> r) & 1:
                Lr = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
                sgm.sgm_debug_path(h, r, L, R, Lr)
                out["paths"][r] = u16(Lr)
        S = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        sgm.sgm_debug_sum(h, L, R, S)
        out["S"] = u16(S)
        dl, dr, lr = (torch.empty((H, W), dtype=torch.uint8, device="cuda") for _ in range(3))
        sgm.sgm_debug_raw(h, L, R, dl, dr, lr)
        out["DL"], out["DR"], out["lr"] = dl.cpu().numpy(), dr.cpu().numpy(), lr.cpu().numpy()
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        h.compute(L, R, disp)
        U = torch.empty((D, W), dtype=torch.int16, device="cuda")
        V = torch.empty((H, D), dtype=torch.int16, device="cuda")
        h.uvmap(disp, U, V)
        torch.cuda.synchronize()
        out["disp"], out["U"], out["V"] = disp.cpu().numpy(), u16(U), u16(V)
    return out


def oracle_all(left, right, D, p):
    o = oracle.sgm(left, right, D, p.census_w, p.census_h, p.path_mask, p.P1, p.P2,
                   p.lr_tolerance, p.median_k, stages=True, cost=p.cost)
    if p.cost == sgm.SGM_COST_CENSUS:
        C = oracle.cost_volume(o["codes_l"], o["codes_r"], D, p.census_w * p.census_h - 1)
    else:
        C = oracle.sad_cost_volume(left, right, D, p.census_w, p.census_h)
    o["paths"] = {r: oracle.aggregate_path(C, r, p.P1, p.P2)
                  for r in range(8) if (p.path_mask >> r) & 1}
    return o


def assert_same(g, o, what):
    assert g.shape == o.shape, (what, g.shape, o.shape)
    if not np.array_equal(g, o):
        bad = np.argwhere(g != o)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {i}: gpu {g[i]} oracle {o[i]}")


def compare_all(left, right, D, p):
    g, o = gpu_all(left, right, D, p), oracle_all(left, right, D, p)
    if p.cost == sgm.SGM_COST_CENSUS:
        assert_same(g["codes_l"], o["codes_l"], "census left")
        assert_same(g["codes_r"], o["codes_r"], "census right")
    for r in o["paths"]:
        assert_same(g["paths"][r], o["paths"][r], f"path {r}")
    for k in ("S", "DL", "DR", "lr", "disp", "U", "V"):
        assert_same(g[k], o[k], k)


CASES = [
    # W, H, D, cw, ch, mask, P1, P2, tol, k
    (37, 23, 16, 5, 5, 0x0F, 4, 24, 1, 5),
    (64, 33, 64, 9, 7, 0xFF, 8, 96, 1, 3),
    (100, 7, 13, 3, 3, 0x55, 2, 9, 0, 0),
    (5, 100, 33, 7, 9, 0xFF, 10, 60, 2, 7),
    (129, 40, 128, 9, 7, 0xFF, 8, 96, 1, 3),
    (70, 45, 129, 5, 5, 0xAA, 3, 30, 1, 5),
    (300, 20, 255, 5, 5, 0x0F, 1, 200, 1, 3),
    (1, 1, 1, 1, 1, 0x01, 0, 0, -1, 0),
    (8, 8, 64, 5, 5, 0xFF, 4, 24, 1, 3),
    (200, 1, 32, 5, 5, 0x0F, 4, 24, 1, 3),
    (1, 50, 8, 5, 5, 0x0F, 4, 24, 1, 3),
    (33, 17, 60, 5, 5, 0x55, 8, 32, 1, 5),
    (97, 61, 100, 9, 7, 0x3C, 7, 50, 1, 1),
    (45, 31, 2, 3, 5, 0x81, 1, 1, 0, 3),
    # P2 on both sides of the code width (24 bits): with P2 >= the largest
    # cost the P2 term of Eq. 2 can never win over L(d*) + C for the previous
    # minimum's disparity d*, below it it can
    (150, 40, 128, 5, 5, 0xFF, 4, 23, 1, 3),
    (150, 40, 128, 5, 5, 0xFF, 4, 24, 1, 3),
    (90, 30, 64, 5, 5, 0xFF, 2, 23, 1, 3),
    (90, 30, 64, 5, 5, 0xFF, 2, 24, 1, 3),
    # widths that are not a multiple of a warp's pixel group, 64 disparities
    (301, 9, 60, 5, 5, 0xFF, 4, 24, 1, 3),
    (150, 12, 64, 9, 7, 0x0F, 8, 96, 2, 3),
    # more rows than 3 WTA CTAs per SM hold on 152 SMs but fewer than 4: the
    # WTA launcher takes its one-group-ahead variant (other cases take two)
    (48, 500, 64, 9, 7, 0xFF, 8, 96, 1, 3),
    (33, 700, 128, 5, 5, 0x0F, 4, 24, 1, 3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:3])) + f"-m{c[5]:02x}")
def test_stage_parity_textured(case):
    W, H, D, cw, ch, mask, P1, P2, tol, k = case
    s = scenes.boxes_scene(W, H, D, seed=W * 131 + H, n_boxes=3,
                           dlo=min(2, D - 1), dhi=max(2, D - 1)) if min(W, H) >= 8 else None
    if s is None:
        r = np.random.default_rng(W + H + D)
        left = r.integers(0, 256, (H, W)).astype(np.uint8)
        right = r.integers(0, 256, (H, W)).astype(np.uint8)
    else:
        left, right = s.left, s.right
    compare_all(left, right, D, params(cw, ch, mask, P1, P2, tol, k))


@pytest.mark.parametrize("seed", range(6))
def test_stage_parity_random_masks_and_noise(seed):
    r = np.random.default_rng(seed)
    W, H = int(r.integers(20, 90)), int(r.integers(10, 60))
    D = int(r.integers(1, 140))
    cw, ch = [(3, 3), (5, 5), (9, 7), (7, 9), (5, 3)][seed % 5]
    nb = cw * ch - 1
    P2 = int(r.integers(0, 255 - nb))
    P1 = int(r.integers(0, P2 + 1))
    mask = int(r.integers(1, 256))
    left = r.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, 3, axis=1) ^ (r.random((H, W)) < 0.1).astype(np.uint8)
    compare_all(left, right, D, params(cw, ch, mask, P1, P2, int(r.integers(-1, 3)),
                                       [0, 1, 3, 5, 7][seed % 5]))


def test_constant_images_degenerate_case():
    left = np.full((30, 40), 90, np.uint8)
    compare_all(left, left.copy(), 24, params(5, 5, 0xFF, 4, 24, 1, 3))


def test_max_width_row():
    W, H, D = 8192, 3, 64
    r = np.random.default_rng(1)
    left = r.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, -5, axis=1)
    p = params(5, 5, 0x0F, 4, 24, 1, 3)
    o = oracle.sgm(left, right, D, 5, 5, 0x0F, 4, 24, 1, 3)
    with sgm.Handle(W, H, D, p) as h:
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        h.compute(cuda(left), cuda(right), disp)
        assert_same(disp.cpu().numpy(), o["disp"], "disp")


def test_row_pitch_and_side_stream():
    W, H, D, pitch = 50, 20, 32, 64
    s = scenes.boxes_scene(W, H, D, seed=3, n_boxes=2, dlo=2, dhi=30)
    big_l = np.zeros((H, pitch), np.uint8)
    big_r = np.full((H, pitch), 200, np.uint8)
    big_l[:, :W], big_r[:, :W] = s.left, s.right
    p = params(5, 5, 0xFF, 4, 24, 1, 3, pitch=pitch)
    o = oracle.sgm(s.left, s.right, D, 5, 5, 0xFF, 4, 24, 1, 3)
    st = torch.cuda.Stream()
    with sgm.Handle(W, H, D, p) as h, torch.cuda.stream(st):
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        h.compute(cuda(big_l), cuda(big_r), disp, stream=st)
        st.synchronize()
        assert_same(disp.cpu().numpy(), o["disp"], "disp with pitch")


# ---------------------------------------------------------------------------
# Full-size workloads, in the configuration the benchmark times.
# ---------------------------------------------------------------------------

def _workload_params(w):
    return params(w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol, w.median_k, cost=w.cost)


@pytest.mark.parametrize("name,idx", [("SMALL_320", 0), ("KITTI_1242", 1), ("HD_1280", 2),
                                      ("PAPER_640", 5), ("PAPER_640_SAD", 6)])
def test_full_size_workloads_bit_exact(name, idx):
    w = getattr(scenes, name)
    s = scenes.scene_for(w, scenes.workload_seed(idx))
    p = _workload_params(w)
    o = oracle.sgm(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2,
                   w.lr_tol, w.median_k, stages=True, cost=w.cost)
    with sgm.Handle(w.W, w.H, w.D, p) as h:
        L, R = cuda(s.left), cuda(s.right)
        disp = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
        U = torch.empty((w.D, w.W), dtype=torch.int16, device="cuda")
        V = torch.empty((w.H, w.D), dtype=torch.int16, device="cuda")
        h.compute(L, R, disp)
        h.uvmap(disp, U, V)
        S = torch.empty((w.H, w.W, w.D), dtype=torch.int16, device="cuda")
        sgm.sgm_debug_sum(h, L, R, S)
        torch.cuda.synchronize()
        assert_same(u16(S), o["S"], "S")
        assert_same(disp.cpu().numpy(), o["disp"], "disp")
        assert_same(u16(U), o["U"], "U")
        assert_same(u16(V), o["V"], "V")


def test_host_entry_point_matches_device_path():
    w = scenes.SMALL_320
    s = scenes.scene_for(w, scenes.workload_seed(0))
    o = oracle.sgm(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2,
                   w.lr_tol, w.median_k)
    with sgm.Handle(w.W, w.H, w.D, _workload_params(w)) as h:
        disp = np.empty((w.H, w.W), np.uint8)
        U = np.empty((w.D, w.W), np.uint16)
        V = np.empty((w.H, w.D), np.uint16)
        for _ in range(2):
            sgm.sgm_compute_host(h, s.left, s.right, disp, U, V)
            assert_same(disp, o["disp"], "disp")
            assert_same(U, o["U"], "U")
            assert_same(V, o["V"], "V")


def test_host_async_pipeline_matches_oracle_per_frame():
    """Five different frames queued back to back through the two staging slots
    (each slot reused), a synchronous call in between, then every frame
    collected by its ticket."""
    W, H, D = 160, 96, 48
    p = params(5, 5, sgm.SGM_PATHS_8, 4, 24, 1, 3)
    frames = [scenes.boxes_scene(W, H, D, seed=300 + i, n_boxes=3, dlo=2, dhi=D - 2) for i in range(5)]
    want = [oracle.sgm(f.left, f.right, D, 5, 5, sgm.SGM_PATHS_8, 4, 24, 1, 3) for f in frames]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ins = [(pin(f.left), pin(f.right)) for f in frames]
    outs = [(torch.empty((H, W), dtype=torch.uint8).pin_memory(),
             torch.empty((D, W), dtype=torch.int16).pin_memory(),
             torch.empty((H, D), dtype=torch.int16).pin_memory()) for _ in frames]
    with sgm.Handle(W, H, D, p) as h:
        tickets = []
        for i, ((l, r), (d, u, v)) in enumerate(zip(ins, outs)):
            tickets.append(sgm.sgm_compute_host_async(h, l.numpy(), r.numpy(), d.numpy(),
                                                       u.numpy().view(np.uint16), v.numpy().view(np.uint16)))
            if i == 2:  # a synchronous frame between queued ones
                d2 = np.empty((H, W), np.uint8)
                sgm.sgm_compute_host(h, frames[0].left, frames[0].right, d2)
                assert_same(d2, want[0]["disp"], "sync frame")
        assert tickets == list(range(tickets[0], tickets[0] + 5))
        for i, t in enumerate(tickets):
            sgm.sgm_host_wait(h, t)
            d, u, v = outs[i]
            assert_same(d.numpy(), want[i]["disp"], f"disp {i}")
            assert_same(u.numpy().view(np.uint16), want[i]["U"], f"U {i}")
            assert_same(v.numpy().view(np.uint16), want[i]["V"], f"V {i}")
        with pytest.raises(sgm.SgmError):
            sgm.sgm_host_wait(h, tickets[-1] + 1)


def test_batch_of_mixed_sizes_matches_oracle():
    specs = [(320, 240, 64), (160, 120, 32), (200, 90, 128), (64, 64, 16)]
    hs, Ls, Rs, Ds, Us, Vs, want = [], [], [], [], [], [], []
    p = params(9, 7, 0xFF, 8, 96, 1, 3)
    for i, (W, H, D) in enumerate(specs):
        s = scenes.ground_scene(W, H, D, seed=40 + i, n_obstacles=3, dlo=D // 6, dhi=(D * 6) // 7)
        want.append(oracle.sgm(s.left, s.right, D, 9, 7, 0xFF, 8, 96, 1, 3))
        hs.append(sgm.Handle(W, H, D, p))
        Ls.append(cuda(s.left))
        Rs.append(cuda(s.right))
        Ds.append(torch.empty((H, W), dtype=torch.uint8, device="cuda"))
        Us.append(torch.empty((D, W), dtype=torch.int16, device="cuda"))
        Vs.append(torch.empty((H, D), dtype=torch.int16, device="cuda"))
    sgm.sgm_batch_compute(hs, Ls, Rs, Ds, Us, Vs)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        assert_same(Ds[i].cpu().numpy(), want[i]["disp"], f"disp {i}")
        assert_same(u16(Us[i]), want[i]["U"], f"U {i}")
        assert_same(u16(Vs[i]), want[i]["V"], f"V {i}")
    for h in hs:
        h.close()


def test_stage_timing_counts_launches():
    w = scenes.SMALL_320
    s = scenes.scene_for(w, scenes.workload_seed(0))
    with sgm.Handle(w.W, w.H, w.D, _workload_params(w)) as h:
        L, R = cuda(s.left), cuda(s.right)
        disp = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
        sgm.sgm_set_timing(h, True)
        for _ in range(3):
            h.compute(L, R, disp)
        t = sgm.sgm_get_stage_times(h)
        assert t["census"][1] == 3 and t["aggregate"][1] == 3 and t["wta_lr"][1] == 3
        assert all(ms > 0 for ms, n in t.values() if n)
        assert sgm.sgm_get_stage_times(h)["aggregate"][1] == 0


# ---------------------------------------------------------------------------
# Next rows: map post-processing (Sec. 3.2) and rectification (Sec. 3.1.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("thr,rad,roi_frac", [(3, 1, None), (8, 2, (0.2, 0.9, 0.1, 0.8)), (1, 0, (0.5, 1.0, 0.0, 0.5))])
def test_uv_postprocess_matches_oracle(thr, rad, roi_frac):
    w = scenes.HD_1280
    s = scenes.scene_for(w, scenes.workload_seed(2))
    o = oracle.sgm(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2,
                   w.lr_tol, w.median_k)
    def roi(rows, cols):
        if roi_frac is None:
            return (0, rows, 0, cols)
        a, b, c, d = roi_frac
        return (int(a * rows), int(b * rows), int(c * cols), int(d * cols))
    uroi, vroi = roi(w.D, w.W), roi(w.H, w.D)
    with sgm.Handle(w.W, w.H, w.D, _workload_params(w)) as h:
        disp = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
        U = torch.empty((w.D, w.W), dtype=torch.int16, device="cuda")
        V = torch.empty((w.H, w.D), dtype=torch.int16, device="cuda")
        h.compute(cuda(s.left), cuda(s.right), disp)
        h.uvmap(disp, U, V)
        uo = torch.empty((w.D, w.W), dtype=torch.uint8, device="cuda")
        vo = torch.empty((w.H, w.D), dtype=torch.uint8, device="cuda")
        sgm.uvmap_postprocess(h, U, V, thr, 2 * thr, uroi, vroi, rad, uo, vo)
        torch.cuda.synchronize()
        assert_same(uo.cpu().numpy(), oracle.uv_post(o["U"], thr, uroi, rad), "U post")
        assert_same(vo.cpu().numpy(), oracle.uv_post(o["V"], 2 * thr, vroi, rad), "V post")


def _distorted_pair(W, H, D, seed):
    """Left image as is; right image moved down 3 rows with a per-row shear,
    and the integer maps that undo it."""
    s = scenes.boxes_scene(W, H, D, seed=seed, n_boxes=3, dlo=2, dhi=D - 2)
    y, x = np.mgrid[0:H, 0:W]
    shear = (y // 8) % 3
    raw = np.zeros_like(s.right)
    ys, xs = y + 3, x + shear
    ok = (ys < H) & (xs < W)
    raw[ys[ok], xs[ok]] = s.right[ok]
    maps = (x.astype(np.uint16), y.astype(np.uint16),
            np.minimum(x + shear, 0xFFFF).astype(np.uint16), (y + 3).astype(np.uint16))
    return s.left, raw, maps


@pytest.mark.parametrize("W,H,D,cw,ch,cost", [(96, 64, 32, 5, 5, 0), (160, 90, 64, 9, 7, 0),
                                              (77, 41, 16, 7, 9, 0), (96, 64, 32, 5, 5, 1),
                                              (83, 47, 24, 3, 7, 1)])
def test_rectified_pipeline_matches_oracle(W, H, D, cw, ch, cost):
    left, raw, (lx, ly, rx, ry) = _distorted_pair(W, H, D, seed=W + D)
    P1, P2 = (4, 24) if cost == sgm.SGM_COST_CENSUS else (100, 400)
    p = params(cw, ch, 0xFF, P1, P2, 1, 3, cost=cost)
    lr = oracle.rectify(left, lx, ly)
    rr = oracle.rectify(raw, rx, ry)
    o = oracle.sgm(lr, rr, D, cw, ch, 0xFF, P1, P2, 1, 3, stages=True, cost=cost)
    with sgm.Handle(W, H, D, p) as h:
        maps = [cuda(m.view(np.int16)) for m in (lx, ly, rx, ry)]
        sgm.sgm_set_rectification(h, *maps)
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        if cost == sgm.SGM_COST_CENSUS:
            cl = torch.empty((H, W), dtype=torch.int64, device="cuda")
            cr = torch.empty_like(cl)
            sgm.sgm_debug_census(h, cuda(left), cuda(raw), cl, cr)
            torch.cuda.synchronize()
            assert_same(cl.cpu().numpy().view(np.uint64), o["codes_l"], "census left")
            assert_same(cr.cpu().numpy().view(np.uint64), o["codes_r"], "census right")
        S = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        sgm.sgm_debug_sum(h, cuda(left), cuda(raw), S)
        h.compute(cuda(left), cuda(raw), disp)
        torch.cuda.synchronize()
        assert_same(u16(S), o["S"], "S")
        assert_same(disp.cpu().numpy(), o["disp"], "disp")
        sgm.sgm_set_rectification(h)  # off again: plain images
        h.compute(cuda(lr), cuda(rr), disp)
        torch.cuda.synchronize()
        assert_same(disp.cpu().numpy(), o["disp"], "disp without maps")


# --------------------------------------------------------------------------
# SAD matching cost (16-bit costs and path costs)
# --------------------------------------------------------------------------

SAD_CASES = [
    # W, H, D, window, path mask, P1, P2, LR tol, median
    (37, 23, 16, 5, 5, 0x0F, 200, 800, 1, 5),
    (64, 33, 60, 5, 5, 0x55, 200, 800, 1, 5),     # the paper's paths, ragged D
    (129, 40, 128, 5, 5, 0xFF, 200, 800, 1, 3),   # S up to 8 * 7175 = 57400
    (70, 45, 100, 3, 3, 0xAA, 50, 300, 1, 3),
    (5, 100, 33, 7, 5, 0x0F, 10, 60, 2, 7),
    (300, 20, 255, 5, 5, 0x03, 200, 800, 1, 3),   # D = 255: 32 lanes per pixel
    (1, 1, 1, 1, 1, 0x01, 0, 0, -1, 0),
    (200, 1, 32, 5, 5, 0x0F, 200, 800, 1, 3),
    (45, 31, 2, 11, 11, 0x01, 0, 0, 0, 3),        # costs up to 30855
    (97, 61, 100, 1, 1, 0x3C, 20, 100, 1, 1),
]


@pytest.mark.parametrize("case", SAD_CASES, ids=lambda c: "x".join(map(str, c[:3])) + f"-w{c[3]}x{c[4]}")
def test_sad_stage_parity(case):
    W, H, D, ww, wh, mask, P1, P2, tol, k = case
    if min(W, H) >= 8:
        s = scenes.boxes_scene(W, H, D, seed=W * 7 + H, n_boxes=3, dlo=min(2, D - 1), dhi=max(2, D - 1))
        left, right = s.left, s.right
    else:
        r = np.random.default_rng(W + 3 * H + D)
        left = r.integers(0, 256, (H, W)).astype(np.uint8)
        right = r.integers(0, 256, (H, W)).astype(np.uint8)
    compare_all(left, right, D, params(ww, wh, mask, P1, P2, tol, k, cost=sgm.SGM_COST_SAD))


# Cost volumes of both Hamming-cost kernels: 128-pixel segments with ragged
# last ones, every padded width Dp (8 .. 256), codes of 0 to 62 bits.
COST_SHAPES = [
    # W, H, D, cw, ch
    (1242, 3, 128, 9, 7),
    (1242, 40, 128, 9, 7),
    (640, 100, 60, 5, 5),
    (300, 4, 60, 5, 5),
    (129, 5, 100, 9, 7),
    (128, 2, 64, 7, 9),
    (257, 3, 33, 5, 5),
    (40, 6, 16, 3, 3),
    (5, 4, 8, 1, 1),
    (77, 3, 1, 5, 3),
    (1, 7, 3, 5, 5),
    (3, 2, 17, 5, 5),
    (200, 3, 129, 9, 7),
    (90, 2, 255, 5, 5),
]


@pytest.mark.parametrize("case", COST_SHAPES, ids=lambda c: "x".join(map(str, c)))
def test_cost_volume_of_each_kernel_matches_oracle(case):
    W, H, D, cw, ch = case
    r = np.random.default_rng(W * 7 + D)
    left = r.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, min(D - 1, 9), axis=1) ^ (r.random((H, W)) < 0.2).astype(np.uint8) * 29
    nbits = cw * ch - 1
    want = oracle.cost_volume(oracle.census(left, cw, ch), oracle.census(right, cw, ch), D, nbits)
    with sgm.Handle(W, H, D, params(cw, ch, 0x0F, 1, 255 - nbits, 1, 0)) as h:
        L, R = cuda(left), cuda(right)
        for kernel in (sgm.SGM_COST_KERNEL_AUTO, sgm.SGM_COST_KERNEL_CUDA_CORES, sgm.SGM_COST_KERNEL_TENSOR_CORES):
            C = torch.full((H, W, D), -1, dtype=torch.int16, device="cuda")
            if kernel == sgm.SGM_COST_KERNEL_TENSOR_CORES and not 16 < D <= 128:
                with pytest.raises(sgm.SgmError) as e:
                    sgm.sgm_debug_cost(h, L, R, C, kernel)
                assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
                continue
            sgm.sgm_debug_cost(h, L, R, C, kernel)
            torch.cuda.synchronize()
            assert_same(u16(C), want, f"cost volume, kernel {kernel}")
        assert sgm.sgm_device_status(h) == sgm.SGM_OK


@pytest.mark.parametrize("kernel", [sgm.SGM_COST_KERNEL_CUDA_CORES, sgm.SGM_COST_KERNEL_TENSOR_CORES])
def test_pipeline_with_each_cost_kernel(kernel):
    s = scenes.boxes_scene(300, 60, 128, seed=11, n_boxes=4, dlo=4, dhi=120)
    p = params(9, 7, 0xFF, 8, 96, 1, 3)
    o = oracle.sgm(s.left, s.right, 128, 9, 7, 0xFF, 8, 96, 1, 3, uv=False)["disp"]
    with sgm.Handle(300, 60, 128, p) as h:
        sgm.sgm_set_cost_kernel(h, kernel)
        disp = torch.empty((60, 300), dtype=torch.uint8, device="cuda")
        h.compute(cuda(s.left), cuda(s.right), disp)
        torch.cuda.synchronize()
        assert_same(disp.cpu().numpy(), o, "disparity")
        assert sgm.sgm_device_status(h) == sgm.SGM_OK


def test_bounded_wait_reports_timeout_and_handle_recovers():
    """The tensor-core cost kernel's first wait runs out on an mbarrier nothing
    arrives at: the call records SGM_ERR_TIMEOUT, the matrix products still
    drain, and the next frame on the same handle is bit-exact again."""
    s = scenes.boxes_scene(700, 40, 128, seed=5, n_boxes=3, dlo=4, dhi=120)
    p = params(9, 7, 0xFF, 8, 96, 1, 3)
    o = oracle.sgm(s.left, s.right, 128, 9, 7, 0xFF, 8, 96, 1, 3, uv=False)["disp"]
    with sgm.Handle(700, 40, 128, p) as h:
        L, R = cuda(s.left), cuda(s.right)
        assert sgm.sgm_device_status(h) == sgm.SGM_OK
        sgm.sgm_debug_stalled_wait(h, L, R)
        assert sgm.sgm_device_status(h) == sgm.SGM_ERR_TIMEOUT
        assert sgm.sgm_device_status(h) == sgm.SGM_OK  # the record was cleared
        for kernel in (sgm.SGM_COST_KERNEL_TENSOR_CORES, sgm.SGM_COST_KERNEL_CUDA_CORES):
            sgm.sgm_set_cost_kernel(h, kernel)
            disp = torch.empty((40, 700), dtype=torch.uint8, device="cuda")
            h.compute(L, R, disp)
            torch.cuda.synchronize()
            assert_same(disp.cpu().numpy(), o, f"disparity after the timeout, kernel {kernel}")
        assert sgm.sgm_device_status(h) == sgm.SGM_OK
    with sgm.Handle(64, 8, 200, params(5, 5, 0x0F, 4, 24, 1, 3)) as h:
        img = torch.zeros((8, 64), dtype=torch.uint8, device="cuda")
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_debug_stalled_wait(h, img, img)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED


def test_cost_kernel_choice_is_checked():
    with sgm.Handle(64, 8, 200, params(5, 5, 0x0F, 4, 24, 1, 3)) as h:
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_cost_kernel(h, sgm.SGM_COST_KERNEL_TENSOR_CORES)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_cost_kernel(h, 7)
        assert e.value.status == sgm.SGM_ERR_INVALID_ARG
    with sgm.Handle(16, 8, 8, params(5, 5, 0x0F, 200, 800, 1, 3, cost=sgm.SGM_COST_SAD)) as h:
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_cost_kernel(h, sgm.SGM_COST_KERNEL_CUDA_CORES)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
        sgm.sgm_set_cost_kernel(h, sgm.SGM_COST_KERNEL_AUTO)


def test_sad_handle_has_no_census_codes():
    p = params(5, 5, 0x0F, 200, 800, 1, 3, cost=sgm.SGM_COST_SAD)
    with sgm.Handle(16, 8, 8, p) as h:
        img = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
        c = torch.empty((8, 16), dtype=torch.int64, device="cuda")
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_debug_census(h, img, img, c, c)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Every blocks-per-SM setting the tuner tries: the aggregation places one
# long-axis job per (SM, scheduler) slot, so its schedule changes with the
# number of resident blocks, and its results must not.
# ---------------------------------------------------------------------------

_TUNE_CASES = {
    "kitti": lambda: (scenes.scene_for(scenes.KITTI_1242, scenes.workload_seed(1)), scenes.KITTI_1242),
    "tall": lambda: (scenes.boxes_scene(160, 600, 64, seed=77, n_boxes=5, dlo=2, dhi=60), None),
}
_tune_oracle = {}


def _tune_case(name):
    if name not in _tune_oracle:
        s, w = _TUNE_CASES[name]()
        if w is None:  # columns are the long axis: 5x5 census, 8 paths
            cfg = dict(D=64, cw=5, ch=5, mask=0xFF, P1=4, P2=24, tol=1, k=3)
        else:
            cfg = dict(D=w.D, cw=w.census_w, ch=w.census_h, mask=w.path_mask, P1=w.P1, P2=w.P2, tol=w.lr_tol,
                       k=w.median_k)
        o = oracle.sgm(s.left, s.right, cfg["D"], cfg["cw"], cfg["ch"], cfg["mask"], cfg["P1"], cfg["P2"],
                       cfg["tol"], cfg["k"], stages=True)
        _tune_oracle[name] = (s, cfg, o)
    return _tune_oracle[name]


@pytest.mark.parametrize("name", sorted(_TUNE_CASES))
@pytest.mark.parametrize("bps", [1, 2, 3, 4, 6])
def test_every_tuner_setting_is_bit_exact(name, bps, monkeypatch):
    s, c, o = _tune_case(name)
    H, W = s.left.shape
    monkeypatch.setenv("SGM_AGG_BLOCKS_PER_SM", str(bps))  # read when the handle is created
    with sgm.Handle(W, H, c["D"], params(c["cw"], c["ch"], c["mask"], c["P1"], c["P2"], c["tol"], c["k"])) as h:
        L, R = cuda(s.left), cuda(s.right)
        S = torch.empty((H, W, c["D"]), dtype=torch.int16, device="cuda")
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        sgm.sgm_debug_sum(h, L, R, S)
        h.compute(L, R, disp)
        torch.cuda.synchronize()
        assert sgm.sgm_device_status(h) == sgm.SGM_OK
        assert_same(u16(S), o["S"], f"S at {bps} blocks/SM")
        assert_same(disp.cpu().numpy(), o["disp"], f"disp at {bps} blocks/SM")


# W, H, D, window, mask, P1, P2, LR tol, median
CPL_CASES = [
    (150, 70, 128, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),    # 4 lanes of 4 chunks per scanline
    (131, 57, 100, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),    # ragged: padding inside the last lane's chunks
    (97, 45, 64, (5, 5), sgm.SGM_PATHS_4, 4, 24, 1, 5),      # 2 lanes per scanline
    (60, 80, 33, (5, 5), sgm.SGM_PATHS_STREAM4, 8, 32, 0, 0),  # one 4-chunk lane per scanline, ragged
    (40, 30, 255, (3, 3), sgm.SGM_PATHS_8, 2, 10, 1, 3),     # 32 chunks: 8 lanes of 4
]


@pytest.mark.parametrize("cpl", [1, 2, 3, 4])
@pytest.mark.parametrize("case", CPL_CASES, ids=[f"{c[0]}x{c[1]}d{c[2]}" for c in CPL_CASES])
def test_every_chunks_per_lane_setting_is_bit_exact(case, cpl):
    """Each path's L_r, S and the disparity map equal the oracle's with 1, 2
    and 4 chunks of 8 disparities per lane (sgm_set_aggregation)."""
    W, H, D, (cw, ch), mask, P1, P2, tol, k = case
    s = scenes.boxes_scene(W, H, D, seed=W + 7 * cpl, n_boxes=3, dlo=1, dhi=D - 1)
    o = oracle.sgm(s.left, s.right, D, cw, ch, mask, P1, P2, tol, k, stages=True, uv=False)
    with sgm.Handle(W, H, D, params(cw, ch, mask, P1, P2, tol, k)) as h:
        sgm.sgm_set_aggregation(h, 3, cpl)
        assert sgm.sgm_get_aggregation(h) == (3, cpl)
        L, R = cuda(s.left), cuda(s.right)
        S = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
        disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        sgm.sgm_debug_sum(h, L, R, S)
        h.compute(L, R, disp)
        for r in (0, 3, 4, 7):
            if (mask >> r) & 1:
                Lr = torch.empty((H, W, D), dtype=torch.int16, device="cuda")
                sgm.sgm_debug_path(h, r, L, R, Lr)
                torch.cuda.synchronize()
                cv = oracle.cost_volume(o["codes_l"], o["codes_r"], D, oracle.census_bits(cw, ch))
                assert_same(u16(Lr), oracle.aggregate_path(cv, r, P1, P2), f"L_{r} with {cpl} chunks per lane")
        torch.cuda.synchronize()
        assert_same(u16(S), o["S"], f"S with {cpl} chunks per lane")
        assert_same(disp.cpu().numpy(), o["disp"], f"disp with {cpl} chunks per lane")


def test_chunks_per_lane_limits():
    with sgm.Handle(64, 32, 16, params(5, 5, sgm.SGM_PATHS_8, 8, 32, 1, 3)) as h:   # D = 16: two chunks per pixel
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_aggregation(h, 3, 4)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_set_aggregation(h, 3, 5)
        assert e.value.status == sgm.SGM_ERR_INVALID_ARG
        assert sgm.sgm_get_aggregation(h)[1] == 1
    sad = params(5, 5, sgm.SGM_PATHS_STREAM4, 200, 800, 1, 5, cost=sgm.SGM_COST_SAD)
    with sgm.Handle(64, 32, 64, sad) as h:   # 16-bit costs: one chunk per lane
        with pytest.raises(sgm.SgmError):
            sgm.sgm_set_aggregation(h, 3, 2)
