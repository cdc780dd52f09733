"""Runs the plane path of a guarded build of the library (selected with
SGM_LIBRARY) over shapes that reach every edge case of its indexing, checks
each result against the CPU oracle and prints one JSON line with the number
of index-check hits.  Started by tests/test_gpu_guarded.py in a process of its
own, so that the guarded library is the only one loaded."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_1807_06271_gb300 import scenes, sgm  # noqa: E402

# W, H, D, census window, path mask, P1, P2, LR tolerance, median
CASES = [
    (160, 96, 64, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),
    (131, 57, 100, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),     # ragged D, odd sizes
    (97, 45, 64, (5, 5), sgm.SGM_PATHS_4, 4, 24, 1, 5),
    (60, 80, 33, (5, 5), sgm.SGM_PATHS_STREAM4, 8, 32, 0, 0),  # W < H: columns are the long axis
    (40, 30, 255, (3, 3), sgm.SGM_PATHS_8, 2, 10, 1, 3),      # 32 lanes per pixel
    (300, 20, 40, (9, 7), sgm.SGM_PATHS_8, 8, 96, -1, 5),     # LR check off
    (20, 200, 48, (5, 5), sgm.SGM_PATHS_8, 8, 32, 2, 0),
    (1, 9, 33, (5, 5), sgm.SGM_PATHS_4, 8, 32, 1, 3),         # one column
    (70, 1, 16, (5, 5), sgm.SGM_PATHS_8, 8, 32, 1, 3),        # one row
    (1, 1, 1, (3, 3), sgm.SGM_PATHS_8, 0, 0, 1, 3),           # one pixel, one disparity
    (257, 33, 128, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),
    (1242, 375, 128, (9, 7), sgm.SGM_PATHS_8, 8, 96, 1, 3),   # the full KITTI-shaped frame
]


def pair(W, H, D, seed):
    if min(W, H) >= 8:
        s = scenes.boxes_scene(W, H, D, seed=seed, n_boxes=3, dlo=min(1, D - 1), dhi=max(1, D - 1))
        return s.left, s.right
    r = np.random.default_rng(seed)
    return r.integers(0, 256, (H, W)).astype(np.uint8), r.integers(0, 256, (H, W)).astype(np.uint8)


def main():
    sgm.sgm_debug_guard_hits(reset=True)
    bad = []
    for n, (W, H, D, (cw, ch), mask, P1, P2, tol, k) in enumerate(CASES):
        left, right = pair(W, H, D, 40 + n)
        p = sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=P1, P2=P2, lr_tolerance=tol, median_k=k)
        o = oracle.sgm(left, right, D, cw, ch, mask, P1, P2, tol, k)
        with sgm.Handle(W, H, D, p) as h:
            for cpl in (1, 2, 4):
                try:
                    sgm.sgm_set_aggregation(h, 3, cpl)
                except sgm.SgmError:
                    continue
                L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
                d = torch.empty((H, W), dtype=torch.uint8, device="cuda")
                U = torch.empty((D, W), dtype=torch.int16, device="cuda")
                V = torch.empty((H, D), dtype=torch.int16, device="cuda")
                h.compute(L, R, d)
                h.uvmap(d, U, V)
                torch.cuda.synchronize()
                ok = (np.array_equal(d.cpu().numpy(), o["disp"])
                      and np.array_equal(U.cpu().numpy().view(np.uint16), o["U"])
                      and np.array_equal(V.cpu().numpy().view(np.uint16), o["V"]))
                if not ok:
                    bad.append(f"{W}x{H}d{D} cpl {cpl}")
    # the batch engine: one group per pair and one shared aggregation launch
    specs = [(160, 96, 64), (97, 61, 128), (64, 40, 32), (45, 45, 100), (1, 9, 33)]
    p8 = sgm.SgmParams(census_w=9, census_h=7, path_mask=sgm.SGM_PATHS_8, P1=8, P2=96, lr_tolerance=1, median_k=3)
    pairs = [pair(W, H, D, 90 + i) for i, (W, H, D) in enumerate(specs)]
    b = sgm.Batch(specs, p8)
    Ls = [torch.from_numpy(a).cuda() for a, _ in pairs]
    Rs = [torch.from_numpy(c).cuda() for _, c in pairs]
    Ds = [torch.empty((H, W), dtype=torch.uint8, device="cuda") for W, H, D in specs]
    for groups in (len(specs), 1):
        b.set_tuning(groups, 3)
        b.run(Ls, Rs, Ds)
        torch.cuda.synchronize()
        for i, (W, H, D) in enumerate(specs):
            o = oracle.sgm(pairs[i][0], pairs[i][1], D, 9, 7, sgm.SGM_PATHS_8, 8, 96, 1, 3, uv=False)
            if not np.array_equal(Ds[i].cpu().numpy(), o["disp"]):
                bad.append(f"batch {W}x{H}d{D} groups {groups}")
    b.close()
    torch.cuda.synchronize()
    print(json.dumps({"library": os.path.basename(sgm.library_path()), "hits": sgm.sgm_debug_guard_hits(),
                      "cases": len(CASES), "mismatches": bad}))


if __name__ == "__main__":
    main()
