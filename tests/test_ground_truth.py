"""The path as a stereo matcher (CPU): on every workload's synthetic scene the
disparity map (the oracle's, which the GPU tests show equals the CUDA path's
bit for bit) is dense and agrees with the scene's ground truth.

- density: the share of pixels that survive the LR check and the median;
- bad-3: among valid pixels whose ground truth is a match, the share more
  than 3 disparities off (the KITTI error measure of the paper's Sec. 4; the
  figures are not comparable with Table 3, which needs the real dataset);
- the LR check (Sec. 3.1.4) removes mostly wrong pixels: the pixels it keeps
  are wrong less than half as often as the raw left winners.
"""
import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes

NAMES = list(scenes.WORKLOADS)


@pytest.mark.parametrize("name", NAMES)
def test_dense_and_close_to_ground_truth(name):
    w = scenes.WORKLOADS[name]
    s = scenes.scene_for(w, scenes.workload_seed(NAMES.index(name)))
    o = oracle.sgm(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol,
                   w.median_k, stages=True, uv=False, cost=w.cost)
    disp, raw, gt = o["disp"].astype(int), o["DL"].astype(int), s.gt.astype(int)
    matched = gt >= 0
    valid = disp != 0xFF
    density = valid.mean()
    bad3 = (np.abs(disp - gt)[valid & matched] > 3).mean()
    kept = o["lr"] != 0xFF
    raw_bad3 = (np.abs(raw - gt)[matched] > 3).mean()
    kept_bad3 = (np.abs(raw - gt)[matched & kept] > 3).mean()
    assert density >= 0.85, (name, density)
    assert bad3 <= 0.03, (name, bad3)
    assert kept_bad3 < 0.5 * raw_bad3, (name, kept_bad3, raw_bad3)
