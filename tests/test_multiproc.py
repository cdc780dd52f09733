"""Host logic of the multi-replica benchmark path on CPU: two gloo ranks,
one pair each, max-over-ranks timing and whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    seconds = 1.0 + r  # rank 1 is slower
    smax = bench.reduce_max(seconds, w)
    rate = bench.whole_job_rate(100.0, w, smax)
    q.put((r, bench.rank_seed(1, r), smax, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_distinct_pairs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out[0][1] != out[1][1]          # each rank draws its own pair
    assert out[0][2] == out[1][2] == 2.0   # max over ranks
    assert out[0][3] == out[1][3] == 100.0  # 2 ranks x 100 units / 2 s


def test_oracle_pool_runs_one_band_per_process():
    """The all-cores CPU baseline: spawned processes each run the unchanged
    oracle on the same band and report the work done."""
    import bench
    from paper_1807_06271_gb300 import scenes
    w = scenes.SMALL_320
    scene = scenes.scene_for(w, scenes.workload_seed(0))
    pool = bench.OraclePool(procs=2)
    try:
        dt, de = pool.run(w, scene, 16, 1)
    finally:
        pool.close()
    assert pool.procs == 2 and dt > 0
    assert de == 2 * w.W * 16 * w.D


def test_reference_arm_prints_the_contract_line(capsys):
    """`bench.py --impl reference` times the oracle on the host cores and prints
    one JSON line with the arm's workload keys and a zero-copy e2e."""
    import json
    import bench
    from paper_1807_06271_gb300 import scenes
    wl = "pair-320x240-d64-census5x5-4path"
    assert bench.main(["--impl", "reference", "--workload", wl, "--steps", "2", "--warmup", "3",
                       "--reference-seconds", "3"]) == 0
    out = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["metric"] == "MDE/s" and d["unit"] == "MDE/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 3, 1)
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic" and d["dtype"] == "u8"
    want = bench.workload_config(scenes.WORKLOADS[wl])
    assert {k: d["config"][k] for k in want} == want
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MDE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out.strip() == ""


def test_roofline_host_arithmetic():
    """Ops per estimate of the aggregation kernel (7 per path), of the cost
    and of the whole path (72 for the 8-path 9x7 workload, 37 for the 4-path
    5x5 ones, counted per estimate as the roofline model does), the HBM bytes the path must move,
    and the path roofline as min(integer bound, HBM bound)."""
    import bench
    from paper_1807_06271_gb300 import scenes
    assert bench.aggregation_ops(scenes.KITTI_1242)["per_de"] == 7 * 8 == 56
    assert bench.aggregation_ops(scenes.SMALL_320)["per_de"] == 28
    assert bench.cost_ops(scenes.KITTI_1242) == 5 and bench.cost_ops(scenes.SMALL_320) == 2
    assert bench.cost_ops(scenes.PAPER_640_SAD) == 2 * 5 + 5
    assert bench.popc_per_de(scenes.KITTI_1242) == 2 and bench.popc_per_de(scenes.PAPER_640_SAD) == 0
    assert bench.path_ops(scenes.KITTI_1242) == 72
    assert bench.path_ops(scenes.SMALL_320) == bench.path_ops(scenes.HD_1280) == 37
    # both ways along the scanlines: one 16-bit partial written and read (4 B);
    # the paper's streaming set is causal in one sweep: images in, map out
    assert bench.path_hbm_bytes_per_de(scenes.KITTI_1242) == 4.0
    assert bench.path_hbm_bytes_per_de(scenes.SMALL_320) == 4.0
    assert bench.path_hbm_bytes_per_de(scenes.PAPER_640) == 3.0 / 60
    peaks = {"int32_tops": 40.0, "u16x2_tops": 80.0, "popc_tops": 5.0}
    r = bench.path_roofline(scenes.KITTI_1242, 200000.0, peaks, 6700.0)
    assert r["int_bound_mde_s"] == 40e12 / 72 / 1e6 and r["hbm_bound_mde_s"] == 6700e9 / 4 / 1e6
    assert r["bound"] == "alu" and abs(r["frac"] - 200000.0 / (40e12 / 72 / 1e6)) < 1e-12
    k = bench.kernel_rooflines(scenes.KITTI_1242, {"aggregate": (1.0, 10), "cost": (0.3, 10), "wta_lr": (0.8, 10)},
                               peaks, 6700.0)
    de = 1242 * 375 * 128
    assert abs(k["aggregate"]["achieved_tops"] - 56 * de / 1e-4 / 1e12) < 1e-6
    assert abs(k["cost"]["achieved_tpopc"] - 2 * de / 3e-5 / 1e12) < 1e-6
    assert k["wta_lr"]["bytes"] == 1242 * 375 * (8 * 128 + 1)


def test_hbm_peak_comes_from_the_measured_file(tmp_path, monkeypatch):
    import json
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6700.8}))
    assert bench.measured_hbm_gbs() == (6700.8, "measured")


def test_profiled_traffic_needs_the_current_source(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "PROFILE_DIR", str(tmp_path))
    (tmp_path / "aggregate_w.md").write_text("# x\n\nsource-digest: 0123abcd\ndram-bytes-per-launch: 636939264\n")
    assert bench.profiled_traffic("aggregate", "w", "0123abcd") == 636939264.0
    assert bench.profiled_traffic("aggregate", "w", "ffffffff") is None   # kernel changed since the capture
    assert bench.profiled_traffic("aggregate", "other", "0123abcd") is None  # no capture for this workload
