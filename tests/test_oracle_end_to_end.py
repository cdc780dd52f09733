"""End-to-end pin of the oracle (CPU): on tiny images, every stage of
``oracle.sgm`` equals a second composition written here from the paper's
definitions in plain Python loops, sharing nothing with the oracle's C code:

- census (Sec. 3.1.2, reading R1) by comparing every window neighbour;
- the Hamming cost of Eq. 1 (R2 outside the image) by counting bits, or the
  SAD cost (R13) as a clamped window sum of absolute differences;
- each path of Eq. 2 (R3) as the exhaustive minimum over all disparity
  sequences along the path, minus the predecessor's minimum;
- S, both winners-take-all (R4, R5), the LR check (R6), the median (R7) and
  the U-/V-maps (R8) by direct search, sort and count.
"""
import itertools

import numpy as np
import pytest

import oracle


def bf_census(img, cw, ch):
    H, W = img.shape
    codes = np.zeros((H, W), np.uint64)
    for y in range(H):
        for x in range(W):
            bits, k = 0, 0
            for v in range(-(ch // 2), ch // 2 + 1):
                for u in range(-(cw // 2), cw // 2 + 1):
                    if u == 0 and v == 0:
                        continue
                    yy, xx = y + v, x + u
                    if 0 <= yy < H and 0 <= xx < W and img[yy, xx] < img[y, x]:
                        bits |= 1 << k
                    k += 1
            codes[y, x] = bits
    return codes


def bf_cost(cl, cr, D, nbits):
    H, W = cl.shape
    C = np.zeros((H, W, D), np.int64)
    for y in range(H):
        for x in range(W):
            for d in range(D):
                C[y, x, d] = bin(int(cl[y, x]) ^ int(cr[y, x - d])).count("1") if x - d >= 0 else nbits
    return C


def bf_sad(left, right, D, ww, wh):
    H, W = left.shape
    C = np.zeros((H, W, D), np.int64)
    for y in range(H):
        for x in range(W):
            for d in range(D):
                if x - d < 0:
                    C[y, x, d] = ww * wh * 255
                    continue
                tot = 0
                for v in range(-(wh // 2), wh // 2 + 1):
                    for u in range(-(ww // 2), ww // 2 + 1):
                        yy = min(max(y + v, 0), H - 1)
                        xl = min(max(x + u, 0), W - 1)
                        xr = min(max(x - d + u, 0), W - 1)
                        tot += abs(int(left[yy, xl]) - int(right[yy, xr]))
                C[y, x, d] = tot
    return C


def bf_path(C, dx, dy, P1, P2):
    """L_r(p, d) = min over disparity sequences along the path ending at p with
    d of (sum of costs + 0 / P1 / P2 per step), minus the same minimum over all
    d at the predecessor (0 at the path's first pixel)."""
    H, W, D = C.shape

    def energies(seq):
        best = [None] * D
        for ds in itertools.product(range(D), repeat=len(seq)):
            e = sum(int(C[py, px, dd]) for (px, py), dd in zip(seq, ds))
            e += sum(0 if a == b else (P1 if abs(a - b) == 1 else P2) for a, b in zip(ds, ds[1:]))
            if best[ds[-1]] is None or e < best[ds[-1]]:
                best[ds[-1]] = e
        return best

    L = np.zeros((H, W, D), np.int64)
    for y in range(H):
        for x in range(W):
            seq = [(x, y)]
            while 0 <= seq[0][0] - dx < W and 0 <= seq[0][1] - dy < H:
                seq.insert(0, (seq[0][0] - dx, seq[0][1] - dy))
            e = energies(seq)
            off = min(energies(seq[:-1])) if len(seq) > 1 else 0
            L[y, x] = [v - off for v in e]
    return L


def bf_pipeline(left, right, D, cw, ch, mask, P1, P2, tol, k, sad=False):
    H, W = left.shape
    if sad:
        cl = cr = None
        C = bf_sad(left, right, D, cw, ch)
    else:
        cl, cr = bf_census(left, cw, ch), bf_census(right, cw, ch)
        C = bf_cost(cl, cr, D, cw * ch - 1)
    S = np.zeros((H, W, D), np.int64)
    for r, (dx, dy) in enumerate(oracle.DIRECTIONS):
        if (mask >> r) & 1:
            S += bf_path(C, dx, dy, P1, P2)
    DL = np.zeros((H, W), np.int64)
    DR = np.zeros((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            DL[y, x] = min(range(D), key=lambda d: (S[y, x, d], d))
            ds = [d for d in range(D) if x + d < W]
            DR[y, x] = min(ds, key=lambda d: (S[y, x + d, d], d))
    lr = np.full((H, W), 0xFF, np.int64)
    for y in range(H):
        for x in range(W):
            d = DL[y, x]
            if tol < 0:
                lr[y, x] = d
            elif x - d >= 0 and abs(d - DR[y, x - d]) <= tol:
                lr[y, x] = d
    if k <= 1:
        disp = lr.copy()
    else:
        disp = np.zeros((H, W), np.int64)
        for y in range(H):
            for x in range(W):
                win = sorted(lr[min(max(y + v, 0), H - 1), min(max(x + u, 0), W - 1)]
                             for v in range(-(k // 2), k // 2 + 1) for u in range(-(k // 2), k // 2 + 1))
                disp[y, x] = win[(k * k + 1) // 2 - 1]
    U = np.zeros((D, W), np.int64)
    V = np.zeros((H, D), np.int64)
    for y in range(H):
        for x in range(W):
            if disp[y, x] < D:
                U[disp[y, x], x] += 1
                V[y, disp[y, x]] += 1
    return dict(codes_l=cl, codes_r=cr, C=C, S=S, D_left=DL, D_right=DR, lr=lr, disp=disp, U=U, V=V)


CASES = [
    # W, H, D, census window, path mask, P1, P2, LR tolerance, median size, seed
    (6, 4, 3, 3, 3, 0xFF, 2, 7, 1, 3, 1),
    (5, 5, 3, 3, 3, 0x55, 1, 4, 0, 3, 2),     # the paper's streaming set
    (7, 3, 4, 5, 3, 0x0F, 3, 9, 1, 1, 3),
    (6, 4, 2, 3, 5, 0xAA, 0, 0, 2, 0, 4),     # no penalties
    (4, 6, 3, 1, 3, 0x33, 5, 5, -1, 5, 5),    # P1 = P2, LR check off, 5x5 median
    (5, 4, 3, 5, 5, 0xC3, 2, 30, 1, 3, 6),    # P2 above every cost
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:3])) + f"-m{c[5]:02x}")
def test_oracle_equals_brute_force_composition(case):
    W, H, D, cw, ch, mask, P1, P2, tol, k, seed = case
    r = np.random.default_rng(4200 + seed)
    left = r.integers(0, 8, (H, W)).astype(np.uint8)   # few levels: many census ties and cost ties
    right = np.roll(left, 1, axis=1)
    right[:, 0] = r.integers(0, 8, H)
    want = bf_pipeline(left, right, D, cw, ch, mask, P1, P2, tol, k)
    got = oracle.sgm(left, right, D, cw, ch, mask, P1, P2, tol, k, stages=True)
    assert np.array_equal(got["codes_l"].astype(np.uint64), want["codes_l"])
    assert np.array_equal(got["codes_r"].astype(np.uint64), want["codes_r"])
    assert np.array_equal(oracle.cost_volume(got["codes_l"], got["codes_r"], D, cw * ch - 1), want["C"])
    assert np.array_equal(got["S"].astype(np.int64), want["S"])
    assert np.array_equal(got["DL"].astype(np.int64), want["D_left"])
    assert np.array_equal(got["DR"].astype(np.int64), want["D_right"])
    assert np.array_equal(got["lr"].astype(np.int64), want["lr"])
    assert np.array_equal(got["disp"].astype(np.int64), want["disp"])
    assert np.array_equal(got["U"].astype(np.int64), want["U"])
    assert np.array_equal(got["V"].astype(np.int64), want["V"])


SAD_CASES = [
    # W, H, D, window, path mask, P1, P2, LR tolerance, median size, seed
    (6, 4, 3, 3, 3, 0x0F, 200, 800, 1, 3, 11),   # the paper's SAD penalties
    (5, 5, 3, 5, 5, 0x55, 50, 400, 0, 3, 12),
    (7, 3, 2, 3, 1, 0xFF, 0, 0, -1, 1, 13),
]


@pytest.mark.parametrize("case", SAD_CASES, ids=lambda c: "x".join(map(str, c[:3])) + f"-m{c[5]:02x}")
def test_sad_oracle_equals_brute_force_composition(case):
    W, H, D, ww, wh, mask, P1, P2, tol, k, seed = case
    r = np.random.default_rng(4300 + seed)
    left = r.integers(0, 256, (H, W)).astype(np.uint8)
    right = np.roll(left, 1, axis=1)
    right[:, 0] = r.integers(0, 256, H)
    want = bf_pipeline(left, right, D, ww, wh, mask, P1, P2, tol, k, sad=True)
    got = oracle.sgm(left, right, D, ww, wh, mask, P1, P2, tol, k, stages=True, cost=oracle.COST_SAD)
    assert np.array_equal(oracle.sad_cost_volume(left, right, D, ww, wh).astype(np.int64), want["C"])
    for key, gkey in (("S", "S"), ("D_left", "DL"), ("D_right", "DR"), ("lr", "lr"), ("disp", "disp"),
                      ("U", "U"), ("V", "V")):
        assert np.array_equal(got[gkey].astype(np.int64), want[key]), key
