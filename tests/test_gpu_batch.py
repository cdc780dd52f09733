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


# ---- the batch engine (sgm_batch_*): pooled scratch, one persistent
# aggregation launch per group over all its pairs' jobs ----------------------

class Engine:
    """The same pairs through sgm_batch_*; reference maps from single handles."""

    def __init__(self, specs, params=P8, seed0=300):
        self.specs, self.params = specs, sgm.SgmParams(**params)
        self.scenes = [make_pair(W, H, D, seed0 + i) for i, (W, H, D) in enumerate(specs)]
        self.L = [torch.from_numpy(s.left).cuda() for s in self.scenes]
        self.R = [torch.from_numpy(s.right).cuda() for s in self.scenes]
        self.Dd = [torch.full((H, W), 7, dtype=torch.uint8, device="cuda") for W, H, D in specs]
        self.U = [torch.empty((D, W), dtype=torch.int16, device="cuda") for W, H, D in specs]
        self.V = [torch.empty((H, D), dtype=torch.int16, device="cuda") for W, H, D in specs]
        self.b = sgm.Batch(specs, self.params)

    def run(self, maps=True):
        self.b.run(self.L, self.R, self.Dd, self.U if maps else None, self.V if maps else None)
        torch.cuda.synchronize()

    def single(self, i):
        W, H, D = self.specs[i]
        with sgm.Handle(W, H, D, self.params) as h:
            d = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            u = torch.empty((D, W), dtype=torch.int16, device="cuda")
            v = torch.empty((H, D), dtype=torch.int16, device="cuda")
            h.compute(self.L[i], self.R[i], d)
            h.uvmap(d, u, v)
            torch.cuda.synchronize()
            return d.cpu().numpy(), u16(u), u16(v)

    def check_all(self, maps=True):
        for i in range(len(self.specs)):
            d, u, v = self.single(i)
            assert np.array_equal(self.Dd[i].cpu().numpy(), d), f"pair {i} {self.specs[i]}"
            if maps:
                assert np.array_equal(u16(self.U[i]), u) and np.array_equal(u16(self.V[i]), v), i


@pytest.mark.parametrize("groups,bps,cpl", [(1, 3, 1), (2, 2, 1), (4, 4, 1), (8, 1, 1), (9, 3, 1), (1, 2, 4), (4, 3, 4),
                                             (9, 2, 4)])
def test_engine_matches_single_pairs_at_each_tuning(groups, bps, cpl):
    specs = [(160, 96, 64), (97, 61, 128), (64, 40, 32), (300, 20, 40), (20, 200, 48), (257, 33, 128),
             (45, 45, 100), (128, 64, 255), (1, 9, 33)]
    e = Engine(specs, seed0=500 + groups)
    e.b.set_tuning(groups, bps, cpl)
    assert e.b.tuning() == (min(groups, len(specs)), bps, cpl)
    e.run()
    e.check_all()
    for i in (0, 2, 6):  # and the oracle, on a few
        W, H, D = specs[i]
        s = e.scenes[i]
        o = oracle.sgm(s.left, s.right, D, 9, 7, sgm.SGM_PATHS_8, 8, 96, 1, 3)
        assert np.array_equal(e.Dd[i].cpu().numpy(), o["disp"]), i
        assert np.array_equal(u16(e.U[i]), o["U"]) and np.array_equal(u16(e.V[i]), o["V"]), i
    e.b.close()


def test_engine_groupings_that_are_accepted():
    """Groups: a power of two up to 64, or exactly one per pair (any count);
    anything else is refused and leaves the tuning as it was."""
    specs = [(60, 40, 32), (50, 30, 16), (40, 20, 64)]
    e = Engine(specs, seed0=40)
    assert e.b.tuning() == (3, 3, 1)  # starts with one group per pair
    for g in (1, 2, 4, 3):
        e.b.set_tuning(g, 2)
        assert e.b.tuning()[0] == min(g, 3)
    for bad in (0, 5, 6, 65):
        with pytest.raises(sgm.SgmError) as err:
            e.b.set_tuning(bad, 2)
        assert err.value.status == sgm.SGM_ERR_INVALID_ARG
    assert e.b.tuning()[0] == 3
    e.run()
    e.check_all()
    e.b.close()


def test_engine_replays_with_new_contents_and_without_maps():
    specs = [(120, 80, 64), (80, 50, 16), (150, 40, 128)]
    e = Engine(specs, seed0=70)
    e.run()
    for i, (W, H, D) in enumerate(specs):  # new contents, same buffers: the replay reads them
        s = make_pair(W, H, D, 970 + i)
        e.L[i].copy_(torch.from_numpy(s.left))
        e.R[i].copy_(torch.from_numpy(s.right))
    e.run()
    e.check_all()
    e.run(maps=False)  # a second graph, without the maps
    e.check_all(maps=False)
    e.b.close()


def test_engine_other_parameter_sets():
    """4-path 5x5 census with no median, and the SAD cost with the paper's
    penalties on the streaming set: each pair equal to its single launch."""
    specs = [(130, 70, 64), (90, 40, 60), (200, 30, 128)]
    for params in (dict(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_4, P1=4, P2=24, lr_tolerance=0, median_k=0),
                   dict(census_w=5, census_h=5, path_mask=sgm.SGM_PATHS_STREAM4, P1=200, P2=800, lr_tolerance=1,
                        median_k=5, cost=sgm.SGM_COST_SAD)):
        e = Engine(specs, params=params, seed0=20)
        assert e.b.tuning()[0] == len(specs)  # one group per pair: the single-pair chain
        e.run()
        e.check_all()
        e.b.set_tuning(1, 3)  # all pairs in one persistent aggregation launch
        e.run()
        e.check_all()
        e.b.close()


def test_engine_64_mixed_pairs_autotuned():
    """The batched workload through the engine: 64 pairs of sizes from
    {320x240, 640x480, 1242x375, 1280x720} and D from {64, 128}; autotuned,
    then every pair byte-identical to its single launch; the pool's size is
    reported."""
    rng = scenes.Rng(1807 + 3)
    sizes = [(320, 240), (640, 480), (1242, 375), (1280, 720)]
    si = rng.integers(0, 3, 64)
    di = rng.integers(0, 1, 64)
    specs = [(sizes[a][0], sizes[a][1], (64, 128)[b]) for a, b in zip(si, di)]
    e = Engine(specs, seed0=1807 + 3)
    g, bps, cpl = e.b.autotune(e.L, e.R, e.Dd, e.U, e.V)
    assert g in (1, 2, 4, 8, 16, 32, 64) and bps in (2, 3, 4) and cpl in (1, 4)
    e.run()
    e.check_all()
    # each handle would also hold its own work-queue state (4228 bytes); the
    # engine keeps one per group
    per_pair = sum(sgm.sgm_scratch_bytes(W, H, D, e.params)[0] - 4228 for W, H, D in specs)
    assert per_pair <= e.b.device_bytes() < per_pair + (1 << 20)
    e.b.close()
