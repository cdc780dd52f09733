"""Pins for the CPU oracle: hand-worked fixtures, brute force on tiny inputs,
closed forms and invariants.  None of these re-types the oracle's own
formulas; each checks it against something it does not share."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes
from tests.conftest import golden


def rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# Census transform (Sec. 3.1.2)
# --------------------------------------------------------------------------

def test_census_hand_worked_3x3():
    g = golden("census_3x3.json")
    img = np.array(g["image"], np.uint8)
    codes = oracle.census(img, *g["window"])
    assert codes.tolist() == g["codes"]


def test_census_bit_order_5x3():
    g = golden("census_bit_order_5x3.json")
    cw, ch = g["window"]
    for wx, wy, bit in g["bits"]:
        img = np.full((7, 9), 100, np.uint8)
        img[3 + wy, 4 + wx] = 40
        assert int(oracle.census(img, cw, ch)[3, 4]) == 1 << bit


@pytest.mark.parametrize("cw,ch", [(3, 3), (5, 5), (9, 7), (7, 9), (1, 3)])
def test_census_constant_image_is_zero(cw, ch):
    img = np.full((11, 13), 77, np.uint8)
    assert not oracle.census(img, cw, ch).any()


@pytest.mark.parametrize("cw,ch", [(5, 5), (9, 7)])
def test_census_invariant_under_increasing_map(cw, ch):
    img = rng(1).integers(0, 128, (20, 24)).astype(np.uint8)
    lut = np.cumsum(rng(2).integers(1, 3, 256))  # strictly increasing
    lut = (lut - lut[0]).clip(0, 255).astype(np.uint8)
    mapped = lut[img]
    assert np.array_equal(oracle.census(img, cw, ch), oracle.census(mapped, cw, ch))


def test_census_codes_fit_their_bits_and_borders_are_zero_bits():
    img = rng(3).integers(0, 256, (16, 16)).astype(np.uint8)
    codes = oracle.census(img, 9, 7)
    assert (codes < np.uint64(1 << 62)).all()
    # top-left pixel: the window rows above and columns to the left are outside,
    # so at most the neighbours right of / below the centre can be set.
    c = int(codes[0, 0])
    for wy in range(-3, 4):
        for wx in range(-4, 5):
            if (wx, wy) == (0, 0):
                continue
            k = (wy + 3) * 9 + (wx + 4)
            k -= 1 if (wy, wx) > (0, 0) else 0
            if wx < 0 or wy < 0:
                assert not (c >> k) & 1


def test_census_translation_equivariance_interior():
    img = rng(4).integers(0, 256, (30, 40)).astype(np.uint8)
    a = oracle.census(img, 5, 5)
    b = oracle.census(np.roll(img, (2, 3), axis=(0, 1)), 5, 5)
    assert np.array_equal(a[2:-4, 2:-5], b[4:-2, 5:-2])


# --------------------------------------------------------------------------
# Matching cost, Eq. 1
# --------------------------------------------------------------------------

def test_hamming_matches_python_bit_count():
    r = rng(5)
    for _ in range(200):
        a, b = (int(v) for v in r.integers(0, 2**63, 2, dtype=np.uint64))
        assert oracle.hamming(a, b) == (a ^ b).bit_count()
        assert oracle.hamming(a, b) == oracle.hamming(b, a)


def test_cost_volume_definition_brute_force():
    r = rng(6)
    H, W, D = 5, 9, 6
    cl = r.integers(0, 2**62, (H, W), dtype=np.uint64)
    cr = r.integers(0, 2**62, (H, W), dtype=np.uint64)
    C = oracle.cost_volume(cl, cr, D, 62)
    for y in range(H):
        for x in range(W):
            for d in range(D):
                want = (int(cl[y, x]) ^ int(cr[y, x - d])).bit_count() if x - d >= 0 else 62
                assert C[y, x, d] == want


def test_cost_zero_for_identical_images_at_d0():
    img = rng(7).integers(0, 256, (8, 10)).astype(np.uint8)
    c = oracle.census(img, 5, 5)
    C = oracle.cost_volume(c, c, 4, 24)
    assert not C[:, :, 0].any()


# --------------------------------------------------------------------------
# Path aggregation, Eq. 2
# --------------------------------------------------------------------------

def test_scanline_hand_worked():
    g = golden("sgm_scanline_4px.json")
    C = np.array(g["cost"], np.uint8)[None]  # 1 x 4 x 3
    L0 = oracle.aggregate_path(C, 0, g["P1"], g["P2"])
    L1 = oracle.aggregate_path(C, 1, g["P1"], g["P2"])
    assert L0[0].tolist() == g["L_left_to_right"]
    assert L1[0].tolist() == g["L_right_to_left"]
    S = oracle.sum_paths(C, 0x03, g["P1"], g["P2"])
    assert S[0].tolist() == g["S"]
    DL, DR = oracle.wta_left(S), oracle.wta_right(S)
    assert DL[0].tolist() == g["D_left"]
    assert DR[0].tolist() == g["D_right"]
    assert oracle.lr_check(DL, DR, g["lr_tol"])[0].tolist() == g["lr"]


def _path_pixels(x, y, dx, dy, W, H):
    """Pixels of the path through (x, y) from its start to (x, y)."""
    seq = [(x, y)]
    while 0 <= seq[0][0] - dx < W and 0 <= seq[0][1] - dy < H:
        seq.insert(0, (seq[0][0] - dx, seq[0][1] - dy))
    return seq


def _brute_min_energy(C, seq, D, P1, P2):
    """min over all disparity sequences ending in d of sum C + penalties (0 / P1 / P2)."""
    best = [None] * D
    for ds in itertools.product(range(D), repeat=len(seq)):
        e = sum(int(C[py, px, dd]) for (px, py), dd in zip(seq, ds))
        for a, b in zip(ds, ds[1:]):
            e += 0 if a == b else (P1 if abs(a - b) == 1 else P2)
        if best[ds[-1]] is None or e < best[ds[-1]]:
            best[ds[-1]] = e
    return best


@pytest.mark.parametrize("r", range(8))
@pytest.mark.parametrize("P1,P2", [(1, 3), (2, 2), (0, 5), (3, 9)])
def test_aggregation_equals_exhaustive_minimisation(r, P1, P2):
    """L_r(p,d) = BF(p,d) - min_k BF(q,k) with BF the exhaustive minimum over all
    disparity sequences along the path (q = predecessor of p)."""
    W, H, D = 5, 4, 3
    C = rng(100 + r).integers(0, 9, (H, W, D)).astype(np.uint8)
    L = oracle.aggregate_path(C, r, P1, P2)
    dx, dy = oracle.DIRECTIONS[r]
    for y in range(H):
        for x in range(W):
            seq = _path_pixels(x, y, dx, dy, W, H)
            bf = _brute_min_energy(C, seq, D, P1, P2)
            off = 0
            if len(seq) > 1:
                off = min(_brute_min_energy(C, seq[:-1], D, P1, P2))
            assert [b - off for b in bf] == L[y, x].tolist(), (x, y)


def test_aggregation_exhaustive_long_scanline_d4():
    W, D, P1, P2 = 6, 4, 2, 5
    C = rng(9).integers(0, 12, (1, W, D)).astype(np.uint8)
    for r in (0, 1):
        L = oracle.aggregate_path(C, r, P1, P2)
        dx, dy = oracle.DIRECTIONS[r]
        for x in range(W):
            seq = _path_pixels(x, 0, dx, dy, W, 1)
            bf = _brute_min_energy(C, seq, D, P1, P2)
            off = min(_brute_min_energy(C, seq[:-1], D, P1, P2)) if len(seq) > 1 else 0
            assert [b - off for b in bf] == L[0, x].tolist()


@pytest.mark.parametrize("r", range(8))
def test_zero_penalties_reduce_to_cost(r):
    C = rng(10 + r).integers(0, 63, (9, 11, 7)).astype(np.uint8)
    assert np.array_equal(oracle.aggregate_path(C, r, 0, 0), C)


@pytest.mark.parametrize("r", range(8))
def test_aggregation_bounds(r):
    C = rng(20 + r).integers(0, 63, (12, 15, 16)).astype(np.uint8)
    L = oracle.aggregate_path(C, r, 8, 96)
    assert L.min() >= 0 and L.max() <= 62 + 96


@pytest.mark.parametrize("a,b", [(2, 3), (4, 7), (6, 5), (0, 0)])
def test_aggregation_flip_symmetry(a, b):
    """Path a on the vertically flipped volume = flipped path b (b = mirror of a)."""
    C = rng(30).integers(0, 40, (7, 9, 5)).astype(np.uint8)
    La = oracle.aggregate_path(C[::-1].copy(), a, 4, 20)
    Lb = oracle.aggregate_path(C, b, 4, 20)
    assert np.array_equal(La, Lb[::-1])


def test_horizontal_paths_are_row_local():
    C = rng(31).integers(0, 40, (6, 10, 5)).astype(np.uint8)
    L = oracle.aggregate_path(C, 0, 3, 11)
    for y in range(6):
        assert np.array_equal(L[y], oracle.aggregate_path(C[y:y + 1], 0, 3, 11)[0])


# --------------------------------------------------------------------------
# WTA, right disparity and LR check (Sec. 3.1.3, 3.1.4)
# --------------------------------------------------------------------------

def test_wta_left_is_first_argmin():
    S = rng(40).integers(0, 6, (5, 7, 9)).astype(np.uint16)  # many ties
    assert np.array_equal(oracle.wta_left(S), np.argmin(S, axis=2))


def test_wta_right_brute_force():
    S = rng(41).integers(0, 6, (4, 12, 5)).astype(np.uint16)
    DR = oracle.wta_right(S)
    H, W, D = S.shape
    for y in range(H):
        for x in range(W):
            cands = [(int(S[y, x + d, d]), d) for d in range(D) if x + d < W]
            assert DR[y, x] == min(cands)[1]


def test_lr_check_brute_force_and_disabled():
    r = rng(42)
    DL = r.integers(0, 6, (6, 20)).astype(np.uint8)
    DR = r.integers(0, 6, (6, 20)).astype(np.uint8)
    for tol in (0, 1, 2):
        out = oracle.lr_check(DL, DR, tol)
        for y in range(6):
            for x in range(20):
                d = int(DL[y, x])
                ok = x - d >= 0 and abs(d - int(DR[y, x - d])) <= tol
                assert out[y, x] == (d if ok else 255)
    assert np.array_equal(oracle.lr_check(DL, DR, -1), DL)


# --------------------------------------------------------------------------
# Median (Sec. 3.1.5) and U-/V-maps (Sec. 3.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [3, 5, 7])
def test_median_matches_numpy_window_median(k):
    img = rng(50 + k).integers(0, 40, (13, 17)).astype(np.uint8)
    img[rng(60).random(img.shape) < 0.2] = 255
    out = oracle.median(img, k)
    r = k // 2
    pad = np.pad(img, r, mode="edge")
    for y in range(13):
        for x in range(17):
            win = pad[y:y + k, x:x + k].ravel()
            assert out[y, x] == int(np.median(win))


def test_median_off_copies():
    img = rng(61).integers(0, 256, (5, 6)).astype(np.uint8)
    assert np.array_equal(oracle.median(img, 0), img)
    assert np.array_equal(oracle.median(img, 1), img)


def test_uvmap_brute_force_and_totals():
    D = 10
    disp = rng(70).integers(0, D, (9, 14)).astype(np.uint8)
    disp[rng(71).random(disp.shape) < 0.3] = 255
    U, V = oracle.uvmap(disp, D)
    valid = disp != 255
    for d in range(D):
        assert np.array_equal(U[d], (disp == d).sum(axis=0))
        assert np.array_equal(V[:, d], (disp == d).sum(axis=1))
    assert U.sum() == V.sum() == valid.sum()
    assert np.array_equal(V.sum(axis=1), valid.sum(axis=1))
    assert np.array_equal(U.sum(axis=0), valid.sum(axis=0))


def test_vmap_shows_ground_plane_line():
    """A ground-plane scene puts the V-map maximum of each low row at the
    ground disparity of that row (Sec. 3.2: the V-map reveals the ground plane)."""
    s = scenes.ground_scene(200, 120, 32, seed=5, n_obstacles=0, texture="blur", sigma=0.0)
    out = oracle.sgm(s.left, s.right, 32, 5, 5, oracle.PATHS_4, 4, 24, 1, 5)
    V = out["V"].astype(int)
    hz = int(round(0.4 * 120))
    rows = range(hz + 10, 115)
    hits = sum(abs(int(np.argmax(V[y])) - int(s.gt[y, 100])) <= 1 for y in rows)
    assert hits >= 0.9 * len(rows)


# --------------------------------------------------------------------------
# End to end
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [0, 5, 11])
def test_constant_shift_recovers_disparity(d):
    s = scenes.shifted_pair(64, 32, d, seed=8 + d)
    out = oracle.sgm(s.left, s.right, 16, 5, 5, oracle.PATHS_4, 4, 24, 1, 5, stages=True)
    disp = out["disp"]
    assert (disp[3:-3, d + 3:-3] == d).all()
    # without the median every LR-valid pixel with x >= d carries d in the interior
    assert (out["lr"][3:-3, d + 3:-3] == d).mean() > 0.97


@pytest.mark.parametrize("mask", [oracle.PATHS_4, oracle.PATHS_8])
def test_vertical_flip_symmetry_end_to_end(mask):
    s = scenes.boxes_scene(48, 40, 16, seed=12, n_boxes=2, dlo=2, dhi=12)
    a = oracle.sgm(s.left, s.right, 16, 5, 5, mask, 4, 24, 1, 3)
    b = oracle.sgm(s.left[::-1], s.right[::-1], 16, 5, 5, mask, 4, 24, 1, 3)
    assert np.array_equal(a["disp"][::-1], b["disp"])
    assert np.array_equal(a["V"][::-1], b["V"])


def test_stage_chain_is_consistent():
    s = scenes.boxes_scene(40, 24, 12, seed=13, n_boxes=2, dlo=2, dhi=10)
    o = oracle.sgm(s.left, s.right, 12, 5, 5, oracle.PATHS_8, 6, 40, 1, 3, stages=True)
    cl = oracle.census(s.left, 5, 5)
    assert np.array_equal(cl, o["codes_l"])
    C = oracle.cost_volume(cl, oracle.census(s.right, 5, 5), 12, 24)
    S = sum(oracle.aggregate_path(C, r, 6, 40).astype(np.int64) for r in range(8))
    assert np.array_equal(S, o["S"])
    assert np.array_equal(np.argmin(S, axis=2), o["DL"])
    assert np.array_equal(oracle.median(o["lr"], 3), o["disp"])


def test_oracle_rejects_bad_arguments():
    img = np.zeros((4, 4), np.uint8)
    with pytest.raises(ValueError):
        oracle.census(img, 4, 3)  # even window
    with pytest.raises(ValueError):
        oracle.census(img, 9, 9)  # 80 bits
    with pytest.raises(ValueError):
        oracle.aggregate_path(np.zeros((2, 2, 2), np.uint8), 0, 5, 2)  # P1 > P2
    with pytest.raises(ValueError):
        oracle.median(img, 4)


# --------------------------------------------------------------------------
# U-/V-map post-processing (Sec. 3.2): threshold, RoI, dilation, Gaussian
# --------------------------------------------------------------------------

def test_uv_post_single_cell_gives_dilated_binomial_footprint():
    m = np.zeros((9, 11), np.uint16)
    m[4, 5] = 7
    out = oracle.uv_post(m, threshold=5, dilate_r=0)
    k = np.outer([1, 2, 1], [1, 2, 1])
    want = np.zeros((9, 11), np.int64)
    want[3:6, 4:7] = (k * 255 + 8) // 16
    assert np.array_equal(out, want)
    # below threshold: nothing
    assert not oracle.uv_post(m, threshold=8, dilate_r=1).any()


def test_uv_post_matches_scipy_morphology_and_convolution():
    ndi = pytest.importorskip("scipy.ndimage")
    r = rng(80)
    m = r.integers(0, 12, (40, 57)).astype(np.uint16)
    for thr, rad, roi in [(9, 1, (5, 35, 3, 50)), (6, 2, (0, 40, 0, 57)), (11, 0, (10, 20, 10, 20))]:
        b = np.zeros(m.shape, bool)
        r0, r1, c0, c1 = roi
        b[r0:r1, c0:c1] = m[r0:r1, c0:c1] >= thr
        d = ndi.binary_dilation(b, structure=np.ones((2 * rad + 1,) * 2, bool)) if rad else b
        g = ndi.convolve(d.astype(np.int64) * 255, np.outer([1, 2, 1], [1, 2, 1]), mode="constant")
        assert np.array_equal(oracle.uv_post(m, thr, roi, rad), (g + 8) // 16)


# --------------------------------------------------------------------------
# Rectification (Sec. 3.1.1)
# --------------------------------------------------------------------------

def test_rectify_identity_shift_and_outside():
    img = rng(90).integers(0, 256, (20, 30)).astype(np.uint8)
    y, x = np.mgrid[0:20, 0:30]
    assert np.array_equal(oracle.rectify(img, x, y), img)
    # rows shifted by 3 and columns by 2: a plain numpy slice
    out = oracle.rectify(img, np.minimum(x + 2, 29), np.minimum(y + 3, 19))
    assert np.array_equal(out[:17, :28], img[3:, 2:])
    # map entries outside the source image give 0
    mx = x.copy()
    mx[5, 7] = 30
    out = oracle.rectify(img, mx, y)
    assert out[5, 7] == 0 and np.array_equal(np.delete(out.ravel(), 5 * 30 + 7), np.delete(img.ravel(), 5 * 30 + 7))


def test_rectify_undoes_a_known_distortion():
    """A right image moved down 3 rows with a per-row horizontal shear is put
    back exactly (away from the borders) by the inverse maps."""
    s = scenes.boxes_scene(64, 48, 16, seed=91, n_boxes=2, dlo=2, dhi=12)
    H, W = s.right.shape
    y, x = np.mgrid[0:H, 0:W]
    shear = (y // 8) % 3
    raw = np.zeros_like(s.right)
    ys, xs = y + 3, x + shear
    ok = (ys < H) & (xs < W)
    raw[ys[ok], xs[ok]] = s.right[ok]
    back = oracle.rectify(raw, np.minimum(x + shear, 0xFFFF), y + 3)
    assert np.array_equal(back[: H - 3, : W - 2], s.right[: H - 3, : W - 2])


# --------------------------------------------------------------------------
# SAD matching cost (Sec. 3.1.2, 5 x 5 support of Sec. 4.1; reading R13)
# --------------------------------------------------------------------------

def _sad_by_padded_box_filter(left, right, D, ww, wh):
    """Independent construction: edge-pad both images (the clamped reads),
    form |L - R shifted by d| on the padded grid and box-filter it with a
    library 2-D convolution; x < d takes the maximum cost."""
    signal = pytest.importorskip("scipy.signal")
    H, W = left.shape
    rw, rh = ww // 2, wh // 2
    Lp = np.pad(left.astype(np.int64), ((rh, rh), (rw, rw)), mode="edge")
    Rp = np.pad(right.astype(np.int64), ((rh, rh), (rw, rw)), mode="edge")
    out = np.full((H, W, D), ww * wh * 255, np.int64)
    for d in range(min(D, W)):
        A = np.abs(Lp[:, d:] - Rp[:, : Rp.shape[1] - d])  # padded columns j >= d
        out[:, d:, d] = signal.convolve2d(A, np.ones((wh, ww), np.int64), mode="valid")
    return out


@pytest.mark.parametrize("W,H,D,ww,wh", [(13, 9, 6, 5, 5), (21, 7, 9, 3, 5), (8, 11, 12, 1, 1),
                                         (30, 12, 16, 7, 3)])
def test_sad_cost_matches_padded_box_filter(W, H, D, ww, wh):
    r = rng(90 + W)
    left = r.integers(0, 256, (H, W)).astype(np.uint8)
    right = r.integers(0, 256, (H, W)).astype(np.uint8)
    got = oracle.sad_cost_volume(left, right, D, ww, wh)
    assert np.array_equal(got, _sad_by_padded_box_filter(left, right, D, ww, wh))


def test_sad_cost_special_cases():
    r = rng(91)
    img = r.integers(0, 256, (10, 17)).astype(np.uint8)
    C = oracle.sad_cost_volume(img, img, 5, 5, 5)
    assert (C[:, :, 0] == 0).all()                      # identical images at d = 0
    for d in range(5):
        assert (C[:, :d, d] == 25 * 255).all()          # x - d < 0: the maximum
    flat = np.full((6, 9), 77, np.uint8)
    C = oracle.sad_cost_volume(flat, flat, 4, 5, 5)
    for d in range(4):
        assert (C[:, d:, d] == 0).all()                 # constant images: 0 wherever x >= d
    # a brightness offset of k adds exactly 25 k to every in-range cost
    C = oracle.sad_cost_volume(flat + 3, flat, 4, 5, 5)
    for d in range(4):
        assert (C[:, d:, d] == 75).all()


def test_sad_constant_shift_recovers_disparity():
    d = 7
    s = scenes.shifted_pair(72, 36, d, seed=92)
    out = oracle.sgm(s.left, s.right, 16, 5, 5, oracle.PATHS_STREAM4, 200, 800, 1, 5,
                     stages=True, cost=oracle.COST_SAD)
    assert (out["disp"][3:-3, d + 3:-3] == d).all()
    assert "codes_l" not in out


def test_sad_stage_chain_is_consistent():
    s = scenes.boxes_scene(40, 24, 12, seed=93, n_boxes=2, dlo=2, dhi=10)
    o = oracle.sgm(s.left, s.right, 12, 5, 5, oracle.PATHS_8, 200, 800, 1, 3, stages=True,
                   cost=oracle.COST_SAD)
    C = oracle.sad_cost_volume(s.left, s.right, 12, 5, 5)
    S = sum(oracle.aggregate_path(C, r, 200, 800).astype(np.int64) for r in range(8))
    assert S.max() < 65536
    assert np.array_equal(S, o["S"])
    assert np.array_equal(np.argmin(S, axis=2), o["DL"])
    assert np.array_equal(oracle.median(o["lr"], 3), o["disp"])


@pytest.mark.parametrize("r", [0, 3, 4, 7])
def test_aggregation_exhaustive_with_sad_range_costs(r):
    """16-bit costs of the SAD range with the paper's SAD penalties (200, 800)."""
    W, H, D, P1, P2 = 4, 3, 3, 200, 800
    C = rng(110 + r).integers(0, 25 * 255 + 1, (H, W, D)).astype(np.uint16)
    L = oracle.aggregate_path(C, r, P1, P2)
    dx, dy = oracle.DIRECTIONS[r]
    for y in range(H):
        for x in range(W):
            seq = _path_pixels(x, y, dx, dy, W, H)
            bf = _brute_min_energy(C, seq, D, P1, P2)
            off = min(_brute_min_energy(C, seq[:-1], D, P1, P2)) if len(seq) > 1 else 0
            assert [b - off for b in bf] == L[y, x].tolist(), (x, y)
