"""Batched execution (one captured CUDA graph per batch) and the autotuner,
against the single-pair entry point and the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes, sgm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

P8 = dict(census_w=9, census_h=7, path_mask=sgm.SGM_PATHS_8, P1=8, P2=96, lr_tolerance=1, median_k=3)


def u16(t):
    return t.cpu().numpy().view(np.uint16)


def make_pair(W, H, D, seed):
    return scenes.ground_scene(W, H, D, seed=seed, n_obstacles=3, dlo=max(1, D // 6),
                               dhi=(D * 6) // 7, texture="value", sigma=2.0, occlusion=0.05)


class Batch:
    def __init__(self, specs, params=P8, seed0=300):
        self.specs = specs
        self.hs, self.L, self.R, self.Dd, self.U, self.V, self.scenes = [], [], [], [], [], [], []
        for i, (W, H, D) in enumerate(specs):
            s = make_pair(W, H, D, seed0 + i)
            self.scenes.append(s)
            self.hs.append(sgm.Handle(W, H, D, sgm.SgmParams(**params)))
            self.L.append(torch.from_numpy(s.left).cuda())
            self.R.append(torch.from_numpy(s.right).cuda())
            self.Dd.append(torch.empty((H, W), dtype=torch.uint8, device="cuda"))
            self.U.append(torch.empty((D, W), dtype=torch.int16, device="cuda"))
            self.V.append(torch.empty((H, D), dtype=torch.int16, device="cuda"))

    def run(self):
        sgm.sgm_batch_compute(self.hs, self.L, self.R, self.Dd, self.U, self.V)
        torch.cuda.synchronize()

    def single(self, i):
        W, H, D = self.specs[i]
        d = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        u = torch.empty((D, W), dtype=torch.int16, device="cuda")
        v = torch.empty((H, D), dtype=torch.int16, device="cuda")
        self.hs[i].compute(self.L[i], self.R[i], d)
        self.hs[i].uvmap(d, u, v)
        torch.cuda.synchronize()
        return d.cpu().numpy(), u16(u), u16(v)

    def close(self):
        for h in self.hs:
            h.close()


def test_graph_replay_follows_new_input_contents():
    b = Batch([(160, 96, 64), (97, 61, 128), (64, 40, 32)])
    b.run()
    first = [d.cpu().numpy().copy() for d in b.Dd]
    # new contents in the same buffers: the replayed graph must read them
    for i, (W, H, D) in enumerate(b.specs):
        s = make_pair(W, H, D, 900 + i)
        b.L[i].copy_(torch.from_numpy(s.left))
        b.R[i].copy_(torch.from_numpy(s.right))
        b.scenes[i] = s
    b.run()
    for i, (W, H, D) in enumerate(b.specs):
        s = b.scenes[i]
        o = oracle.sgm(s.left, s.right, D, 9, 7, sgm.SGM_PATHS_8, 8, 96, 1, 3)
        assert np.array_equal(b.Dd[i].cpu().numpy(), o["disp"]), i
        assert np.array_equal(u16(b.U[i]), o["U"]) and np.array_equal(u16(b.V[i]), o["V"]), i
    assert any(not np.array_equal(f, d.cpu().numpy()) for f, d in zip(first, b.Dd))
    b.close()


def test_timing_path_and_graph_path_agree():
    b = Batch([(120, 80, 64), (80, 50, 16)])
    b.run()
    graph_out = [d.cpu().numpy().copy() for d in b.Dd]
    for h in b.hs:
        sgm.sgm_set_timing(h, True)
    b.run()
    for i in range(2):
        assert np.array_equal(graph_out[i], b.Dd[i].cpu().numpy())
    assert sgm.sgm_get_stage_times(b.hs[0])["aggregate"][1] == 1
    b.close()


def test_destroyed_handles_drop_their_graphs():
    for rep in range(3):  # new handles may reuse freed addresses
        b = Batch([(100, 60, 32), (60, 100, 64)], seed0=40 + rep)
        b.run()
        for i in range(2):
            assert np.array_equal(b.Dd[i].cpu().numpy(), b.single(i)[0])
        b.close()


def test_autotune_keeps_results_and_is_reused():
    W, H, D = 320, 240, 64
    s = make_pair(W, H, D, 5)
    L, R = torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda()
    d0 = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    d1 = torch.empty_like(d0)
    h = sgm.Handle(W, H, D, sgm.SgmParams(**P8))
    h.compute(L, R, d0)
    best = sgm.sgm_autotune(h, L, R, d1)
    assert best in (1, 2, 3, 4, 6)
    h.compute(L, R, d1)
    torch.cuda.synchronize()
    assert np.array_equal(d0.cpu().numpy(), d1.cpu().numpy())
    h.close()


def test_64_pair_mixed_batch_equals_single_pair_launches():
    """Batched workload: 64 pairs with sizes drawn from {320x240, 640x480,
    1242x375, 1280x720} and D from {64, 128}, 9x7 census, 8 paths; every pair
    of the graph-replayed batch is byte-identical to its own single launch,
    and the smallest pairs match the oracle."""
    rng = scenes.Rng(1807 + 3)
    sizes = [(320, 240), (640, 480), (1242, 375), (1280, 720)]
    si = rng.integers(0, 3, 64)
    di = rng.integers(0, 1, 64)
    specs = [(sizes[a][0], sizes[a][1], (64, 128)[b]) for a, b in zip(si, di)]
    b = Batch(specs, seed0=1807 + 3)
    b.run()
    b.run()  # replay
    for i in range(len(specs)):
        d, u, v = b.single(i)
        assert np.array_equal(b.Dd[i].cpu().numpy(), d), i
        assert np.array_equal(u16(b.U[i]), u) and np.array_equal(u16(b.V[i]), v), i
    small = [i for i, sp in enumerate(specs) if sp[:2] == (320, 240)][:2]
    for i in small:
        D = specs[i][2]
        s = b.scenes[i]
        o = oracle.sgm(s.left, s.right, D, 9, 7, sgm.SGM_PATHS_8, 8, 96, 1, 3)
        assert np.array_equal(b.Dd[i].cpu().numpy(), o["disp"]), i
    b.close()
