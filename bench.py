#!/usr/bin/env python
"""Throughput of the SGM stereo path on GB300, in MDE/s (million disparity
estimates W*H*D per second).

One step = the whole path on one stereo pair already resident in HBM:
census + Hamming cost, path aggregation, WTA + right WTA + LR check, median,
U-/V-maps.  The workload is the KITTI-shaped pair (1242x375, D=128, 9x7
census, 8 paths, P1=8, P2=96, LR tolerance 1, 3x3 median) on a seeded
synthetic scene.  L2 is flushed (256 MiB write) between timed steps; each step
is timed with CUDA events on the launching stream and the flush is outside the
events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own pair (independent replicas, weak
scaling); rank 0 prints one JSON line.  ``--impl reference`` times the CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_06271_gb300 import scenes  # noqa: E402

WORKLOAD_INDEX = {"pair-320x240-d64-census5x5-4path": 0, "kitti-1242x375-d128-census9x7-8path": 1,
                  "hd-1280x720-d128-census5x5-4path-uv": 2, "paper-640x360-d60-census5x5-stream4": 5,
                  "paper-640x360-d60-sad5x5-stream4": 6}
FLUSH_BYTES = 256 << 20
PROFILE_DIR = os.path.join(ROOT, "profiles")


# ---------------------------------------------------------------------------
# host-side helpers (also exercised by the CPU multi-process tests)
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(workload_index: int, rank: int) -> int:
    """Each rank works on its own pair: seed 1807 + workload index + pair index."""
    return scenes.workload_seed(workload_index, rank)


def reduce_max(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    return units_per_rank * world / seconds_max


def aggregation_ops(w) -> dict:
    """Algorithmic integer operations per disparity estimate of the
    aggregation kernel alone: per enabled path 3 min + 2 add + 1 sub + 1
    running min = 7 (Eq. 2).  The matching cost runs in its own kernel."""
    npaths = bin(w.path_mask).count("1")
    return {"per_path": 7, "paths": npaths, "per_de": 7 * npaths}


def cost_ops(w) -> int:
    """Operations per estimate of the matching cost (Eq. 1): XOR + POPC for
    codes of up to 32 bits (2), two of each plus an add for 64-bit codes (5);
    the SAD cost, separable, an absolute difference and an add per window row
    plus an add per window column (2 wh + ww)."""
    if w.cost == 1:
        return 2 * w.census_h + w.census_w
    return 2 if w.census_w * w.census_h - 1 <= 32 else 5


def popc_per_de(w) -> int:
    return 0 if w.cost == 1 else (1 if w.census_w * w.census_h - 1 <= 32 else 2)


def path_ops(w) -> int:
    """Whole-path integer operations per estimate: the aggregation (7 per
    path), the cost once, R - 1 adds summing the paths and about 4 for the two
    winner-takes-all searches (72 for the 8-path 9x7 workload, 37 for the
    4-path 5x5 ones)."""
    npaths = bin(w.path_mask).count("1")
    return 7 * npaths + cost_ops(w) + (npaths - 1) + 4


def path_hbm_bytes_per_de(w) -> float:
    """Bytes per estimate that the path must move through HBM at the least.
    When the enabled directions run both ways along a scanline, one sweep's
    16-bit partial sum has to be written and read back once (4 B); when all of
    them are causal in one top-down sweep, only the images in and the map out
    (3 bytes per pixel)."""
    fwd = w.path_mask & 0x55
    bwd = w.path_mask & 0xAA
    return 4.0 if (fwd and bwd) else 3.0 / w.D


def measured_hbm_gbs():
    """(GB/s, basis): the measured copy bandwidth of this GPU type from
    MEASURED_PEAKS.json beside the repository, else a 6.8 TB/s fallback (one
    earlier GB300 measurement)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["hbm_gbs"])
        if v > 0:
            return v, "measured"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "fallback"


def int_peaks(sgm) -> dict:
    """Measured integer issue rates (best of three launches of the library's
    probe kernel): the add/min mix in lane operations per second, the packed
    16-bit min/add mix counted per 16-bit operation (two per instruction), and
    POPC (one of the two operations of the xor/popc mix)."""
    best = {}
    for name, kind in (("int32", sgm.SGM_PROBE_INT32_ADD_MIN), ("u16x2", sgm.SGM_PROBE_U16X2_MIN_ADD),
                       ("popc_xor", sgm.SGM_PROBE_POPC_XOR)):
        best[name] = max(sgm.sgm_probe_int_rate(kind)[0] for _ in range(3))
    return {"int32_tops": best["int32"] / 1e12, "u16x2_tops": 2 * best["u16x2"] / 1e12,
            "popc_tops": best["popc_xor"] / 2 / 1e12,
            "basis": "sgm_probe_int_rate: 8 blocks x 256 threads per SM, 8 independent chains per thread"}


def kernel_source_digest(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, digest: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; None otherwise."""
    path = os.path.join(PROFILE_DIR, f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_d = re.search(r"source-digest:\s*([0-9a-f]+)", text)
    m_t = re.search(r"dram-bytes-per-launch:\s*([0-9.eE+]+)", text)
    if not m_d or not m_t or m_d.group(1) != digest:
        return None
    return float(m_t.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def mark(self):
        self.marks.append(time.perf_counter())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (0, 1e30)
        inside = [s for t, s in self.samples if t0 <= t <= t1 + 0.06] or [s for _, s in self.samples]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in inside:
            f = [x.strip() for x in s.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_band(scene, w, rows):
    """A row band of the workload's pair (the first ``rows`` rows)."""
    return scene.left[:rows].copy(), scene.right[:rows].copy()


def time_oracle(w, scene, rows, reps):
    import oracle
    left, right = oracle_band(scene, w, rows)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.sgm(left, right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol,
                   w.median_k, uv=w.uv, cost=w.cost)
    dt = time.perf_counter() - t0
    return dt, w.W * rows * w.D * reps


def _oracle_worker(task):
    """One process of the all-cores oracle run: the plain oracle, unchanged,
    on one band of the pair (spawned process; no CUDA)."""
    import oracle
    left, right, w_fields, reps = task
    D, cw, ch, mask, P1, P2, tol, k, uv, cost = w_fields
    for _ in range(reps):
        oracle.sgm(left, right, D, cw, ch, mask, P1, P2, tol, k, uv=uv, cost=cost)
    return reps


def _oracle_warm(_):
    import oracle
    oracle._load()
    return os.getpid()


def _oracle_pair(task):
    """One whole pair through the plain oracle (spawned process; no CUDA)."""
    import oracle
    left, right, fields = task
    D, cw, ch, mask, P1, P2, tol, k, uv, cost = fields
    oracle.sgm(left, right, D, cw, ch, mask, P1, P2, tol, k, uv=uv, cost=cost)
    return left.shape[0] * left.shape[1] * D


class OraclePool:
    """The oracle on every host core at once: one spawned process per core,
    each running whole bands of the pair (the oracle itself stays single
    threaded and unchanged)."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        import oracle
        oracle.build()  # built once here, before the workers load it
        try:
            avail = len(os.sched_getaffinity(0))
        except AttributeError:
            avail = os.cpu_count() or 1
        self.procs = procs or avail
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_warm, range(self.procs))

    def run(self, w, scene, rows, reps):
        """Wall time of procs x reps bands of ``rows`` rows, and the DE done."""
        left, right = oracle_band(scene, w, rows)
        fields = (w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol, w.median_k, w.uv,
                  w.cost)
        tasks = [(left, right, fields, reps)] * self.procs
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, tasks, chunksize=1)
        dt = time.perf_counter() - t0
        return dt, w.W * rows * w.D * reps * self.procs

    def run_pairs(self, tasks):
        """Wall time of whole pairs (left, right, fields) spread over the
        processes, and the DE done."""
        t0 = time.perf_counter()
        de = sum(self.pool.map(_oracle_pair, tasks, chunksize=1))
        return time.perf_counter() - t0, de

    def close(self):
        self.pool.close()
        self.pool.join()


def workload_config(w):
    """The workload keys of the bench line, the same for both arms."""
    return {"workload": w.name, "W": w.W, "H": w.H, "D": w.D,
            "cost": "sad" if w.cost == 1 else "census",
            "census": f"{w.census_w}x{w.census_h}", "path_mask": w.path_mask,
            "P1": w.P1, "P2": w.P2, "lr_tol": w.lr_tol, "median_k": w.median_k,
            "uv_maps": w.uv}


def run_reference(args, w, windex):
    rank = dist_env()[0]
    if rank != 0:
        return 0
    scene = scenes.scene_for(w, rank_seed(windex, 0))
    # Size each step's sample (a band of rows of the pair) so that warm-up plus
    # the timed steps take about --reference-seconds (two minutes) of host time.
    probe_rows = min(w.H, 16)
    t_probe, _ = time_oracle(w, scene, probe_rows, 1)
    per_row = t_probe / probe_rows
    budget = args.reference_seconds / max(1, args.steps + args.warmup)
    rows = int(min(w.H, max(8, budget / max(per_row, 1e-9))))
    # every step runs the band once on each host core (one process per core)
    pool = OraclePool()
    for _ in range(args.warmup):
        pool.run(w, scene, rows, 1)
    dt, de = pool.run(w, scene, rows, args.steps)
    pool.close()
    value = de / dt / 1e6
    sample = (f"first {rows} of {w.H} rows of the {w.W}x{w.H} pair per step (all paths, WTA, LR, "
              f"median, U/V) in each of {pool.procs} processes, one per host core")
    line = {
        "impl": "reference", "metric": "MDE/s", "value": value, "unit": "MDE/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": dict(workload_config(w), parallelism=f"{pool.procs} host processes"),
        "cpu_baseline": {"value": value, "unit": "MDE/s", "cores": pool.procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MDE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------

def sgm_params_of(sgm, w):
    return sgm.SgmParams(census_w=w.census_w, census_h=w.census_h, path_mask=w.path_mask,
                         P1=w.P1, P2=w.P2, lr_tolerance=w.lr_tol, median_k=w.median_k, cost=w.cost)


class FramePair:
    """One workload's pair resident on the device, its handle and outputs."""

    def __init__(self, sgm, torch, w, seed, autotune):
        self.w = w
        self.scene = scenes.scene_for(w, seed)
        self.params = sgm_params_of(sgm, w)
        self.h = sgm.Handle(w.W, w.H, w.D, self.params)
        self.left = torch.from_numpy(self.scene.left).cuda()
        self.right = torch.from_numpy(self.scene.right).cuda()
        self.disp = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
        self.umap = torch.empty((w.D, w.W), dtype=torch.int16, device="cuda")
        self.vmap = torch.empty((w.H, w.D), dtype=torch.int16, device="cuda")
        # the aggregation kernel's resident blocks per SM, chosen by the
        # library's own tuner for this shape (a user calls the same entry point)
        self.bps = (sgm.sgm_autotune(self.h, self.left, self.right, self.disp,
                                     torch.cuda.current_stream()) if autotune else None)

    def step(self, stream):
        self.h.compute(self.left, self.right, self.disp, stream)
        if self.w.uv:
            self.h.uvmap(self.disp, self.umap, self.vmap, stream)

    def close(self):
        self.h.close()


def stream_rate(torch, sgm, fp, ns, pairs, stream):
    """Consecutive pairs spread round-robin over ns handles on ns streams
    (fp's handle plus ns - 1 new ones of the same shape, which start from the
    tuner's choice for it): one pair's HBM-bound WTA overlaps other pairs'
    aggregation, as a stream of frames is best run.  No L2 flush between
    pairs.  Returns ms per pair."""
    w = fp.w
    extra = [sgm.Handle(w.W, w.H, w.D, fp.params) for _ in range(ns - 1)]
    try:
        hs = [fp.h] + extra
        ss = [torch.cuda.Stream() for _ in range(ns)]
        ds = [fp.disp] + [torch.empty_like(fp.disp) for _ in extra]
        us = [fp.umap] + [torch.empty_like(fp.umap) for _ in extra]
        vs = [fp.vmap] + [torch.empty_like(fp.vmap) for _ in extra]

        def one(i):
            k = i % ns
            hs[k].compute(fp.left, fp.right, ds[k], ss[k])
            if w.uv:
                hs[k].uvmap(ds[k], us[k], vs[k], ss[k])

        for i in range(2 * ns):
            one(i)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for st in ss:
            st.wait_event(c0)
        for i in range(pairs):
            one(i)
        for st in ss:
            ev = torch.cuda.Event()
            ev.record(st)
            stream.wait_event(ev)
        c1.record(stream)
        torch.cuda.synchronize()
        return c0.elapsed_time(c1) / pairs
    finally:
        for h in extra:
            h.close()


def timed_steps(torch, fp, stream, flush, steps):
    """CUDA-event time of each of `steps` steps, L2 flushed before each
    (outside the events)."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        fp.step(stream)
        stops[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, stops)]


def stage_pass(sgm, fp, stream, flush, n):
    """Per-stage kernel times from a separate pass with stage events recorded
    around every kernel (the timed steps run without them)."""
    sgm.sgm_set_timing(fp.h, True)
    sgm.sgm_get_stage_times(fp.h)  # reset
    for i in range(n):
        flush.fill_(i & 0xFF)
        fp.step(stream)
    stage = sgm.sgm_get_stage_times(fp.h)
    sgm.sgm_set_timing(fp.h, False)
    return stage


def e2e_run(torch, sgm, fp, stream, steps, world=1):
    """End to end through the pipelined host-buffer entry point, as a camera
    loop uses it: two pinned host buffer sets in turn, a set reused once the
    frame that last used it has been collected.  Every step uploads its pair
    and downloads its disparity map (and U/V maps); frames run back to back."""
    w, h = fp.w, fp.h
    sets = []
    for _ in range(2):
        sets.append((torch.from_numpy(fp.scene.left).pin_memory(), torch.from_numpy(fp.scene.right).pin_memory(),
                     torch.empty((w.H, w.W), dtype=torch.uint8).pin_memory(),
                     torch.empty((w.D, w.W), dtype=torch.int16).pin_memory() if w.uv else None,
                     torch.empty((w.H, w.D), dtype=torch.int16).pin_memory() if w.uv else None))
    for i in range(2):
        sgm.sgm_host_wait(h, sgm.sgm_compute_host_async(h, *sets[i], stream))
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    tickets = []
    for i in range(steps):
        if i >= 2:
            sgm.sgm_host_wait(h, tickets[i - 2])
        tickets.append(sgm.sgm_compute_host_async(h, *sets[i & 1], stream))
    sgm.sgm_host_wait(h, tickets[-2])
    sgm.sgm_host_wait(h, tickets[-1])
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    return {"value": whole_job_rate(w.de_per_frame * steps, world, e2e_s) / 1e6, "unit": "MDE/s",
            "h2d_bytes_per_step": 2 * w.W * w.H,
            "d2h_bytes_per_step": w.W * w.H + (2 * w.D * w.W + 2 * w.H * w.D if w.uv else 0),
            "steps": steps, "api": "sgm_compute_host_async + sgm_host_wait"}


def kernel_rooflines(w, stage, peaks, hbm_gbs):
    """Each kernel of the path against the resource that bounds it, from the
    stage pass's mean event times."""
    de = w.de_per_frame
    npaths = bin(w.path_mask).count("1")
    lanes = 1
    while 8 * lanes < w.D:
        lanes *= 2
    Dp, eb = 8 * lanes, (2 if w.cost == 1 else 1)
    out = {}

    def mean_s(k):
        t, n = stage.get(k, (0.0, 0))
        return t / n / 1e3 if n else None

    t = mean_s("aggregate")
    if t:
        ops = aggregation_ops(w)["per_de"]
        a = ops * de / t / 1e12
        out["aggregate"] = {"bound": "alu", "ops_per_de": ops, "achieved_tops": a, "frac": a / peaks["int32_tops"],
                            "frac_packed": a / peaks["u16x2_tops"], "us": t * 1e6}
    t = mean_s("cost")
    if t:
        if w.cost == 1:
            ops = cost_ops(w)
            a = ops * de / t / 1e12
            out["cost"] = {"bound": "alu", "ops_per_de": ops, "achieved_tops": a, "frac": a / peaks["int32_tops"],
                           "us": t * 1e6}
        else:
            pc = popc_per_de(w)
            a = pc * de / t / 1e12
            out["cost"] = {"bound": "popc", "popc_per_de": pc, "achieved_tpopc": a, "frac": a / peaks["popc_tops"],
                           "us": t * 1e6}
    t = mean_s("sweep")
    if t:
        # the fused sweep does the cost, every path, the sums and both winners
        ops = path_ops(w)
        a = ops * de / t / 1e12
        out["sweep"] = {"bound": "alu", "ops_per_de": ops, "achieved_tops": a, "frac": a / peaks["int32_tops"],
                        "us": t * 1e6}
    t = mean_s("wta_lr")
    if t:
        byts = w.W * w.H * (npaths * Dp * eb + 1)
        a = byts / t / 1e9
        out["wta_lr"] = {"bound": "hbm", "bytes": byts, "achieved_gbs": a, "frac": a / hbm_gbs, "us": t * 1e6}
    return out


def path_roofline(w, value_mde, peaks, hbm_gbs):
    """The whole per-frame path: min(integer bound, HBM bound) in MDE/s and
    the fraction the measured throughput reaches."""
    ops = path_ops(w)
    byts = path_hbm_bytes_per_de(w)
    int_bound = peaks["int32_tops"] * 1e12 / ops / 1e6
    hbm_bound = hbm_gbs * 1e9 / byts / 1e6
    roof = min(int_bound, hbm_bound)
    return {"ops_per_de": ops, "hbm_bytes_per_de": byts, "int_bound_mde_s": int_bound,
            "hbm_bound_mde_s": hbm_bound, "bound": "alu" if int_bound <= hbm_bound else "hbm",
            "roofline_mde_s": roof, "achieved_mde_s": value_mde, "frac": value_mde / roof}


def per_config_line(torch, sgm, w, windex, steps, stream, flush, peaks, hbm_gbs):
    """One workload timed as the headline is (L2 flushed between steps, CUDA
    events on the stream), plus a short end-to-end run and its stage times."""
    fp = FramePair(sgm, torch, w, rank_seed(windex, 0), autotune=True)
    for _ in range(3):
        fp.step(stream)
    torch.cuda.synchronize()
    ms = timed_steps(torch, fp, stream, flush, steps)
    ms_per_step = sum(ms) / len(ms)
    value = w.de_per_frame / (ms_per_step / 1e3) / 1e6
    stage = stage_pass(sgm, fp, stream, flush, min(steps, 50))
    e2e = e2e_run(torch, sgm, fp, stream, max(3, min(steps, 50)))
    ms4 = stream_rate(torch, sgm, fp, 4, 200, stream)
    line = {"config": workload_config(w), "value": value, "unit": "MDE/s", "ms_per_step": ms_per_step,
            "fps": 1e3 / ms_per_step, "steps": steps, "e2e": e2e, "agg_blocks_per_sm": fp.bps,
            "stage_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in stage.items() if v[1]},
            "kernels": kernel_rooflines(w, stage, peaks, hbm_gbs),
            "path_roofline": path_roofline(w, value, peaks, hbm_gbs),
            "four_streams": {"ms_per_pair": ms4, "value": w.de_per_frame / (ms4 / 1e3) / 1e6, "unit": "MDE/s",
                             "pairs": 200}}
    fp.close()
    return line


def run_ours(args, w, windex):
    import numpy as np
    import torch

    from paper_1807_06271_gb300 import sgm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    stream = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peaks = int_peaks(sgm)
    hbm_gbs, hbm_of = measured_hbm_gbs()
    fp = FramePair(sgm, torch, w, rank_seed(windex, rank), autotune=not args.no_autotune)
    h, left, right, disp, umap, vmap = fp.h, fp.left, fp.right, fp.disp, fp.umap, fp.vmap
    # optional overrides of what the tuner chose (for profiling one kernel)
    if args.schedule != "auto":
        sgm.sgm_set_schedule(h, {"planes": sgm.SGM_SCHEDULE_PLANES, "sweep": sgm.SGM_SCHEDULE_SWEEP}[args.schedule],
                             args.sweep_rows)
    if args.cost_kernel != "auto":
        sgm.sgm_set_cost_kernel(h, {"cuda_cores": sgm.SGM_COST_KERNEL_CUDA_CORES,
                                    "tensor_cores": sgm.SGM_COST_KERNEL_TENSOR_CORES}[args.cost_kernel])
    params, scene, bps = fp.params, fp.scene, fp.bps
    for _ in range(args.warmup):
        fp.step(stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.mark()
    wall0 = time.perf_counter()
    step_ms = timed_steps(torch, fp, stream, flush, args.steps)
    wall = time.perf_counter() - wall0
    sampler.mark()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    stage = stage_pass(sgm, fp, stream, flush, min(args.steps, 200))
    total_s = sum(step_ms) / 1e3
    total_s_max = reduce_max(total_s, world)
    de = w.de_per_frame
    value = whole_job_rate(de * args.steps, world, total_s_max) / 1e6
    ms_per_step = total_s_max / args.steps * 1e3

    # the dominant kernel (the aggregation) against the measured INT32 issue
    # rate, and the whole path against min(integer bound, HBM bound)
    kernels = kernel_rooflines(w, stage, peaks, hbm_gbs)
    dom = "aggregate" if "aggregate" in kernels else "sweep"
    agg = kernels[dom]
    src = {"aggregate": "aggregate.cu", "sweep": "sweep.cu"}[dom]
    digest = kernel_source_digest([f"paper_1807_06271_gb300/csrc/{src}", "paper_1807_06271_gb300/csrc/sgm_internal.cuh"])
    traffic = profiled_traffic(dom, w.name, digest)
    path = path_roofline(w, value / world, peaks, hbm_gbs)
    roofline = {"bound": "alu", "kernel": dom, "achieved": agg["achieved_tops"],
                "peak": peaks["int32_tops"], "unit": "Tops/s", "frac": agg["frac"], "traffic": traffic,
                "ops_per_de": agg["ops_per_de"], "of": "measured", "peak_basis": peaks["basis"],
                "peak_packed": peaks["u16x2_tops"], "frac_packed": agg.get("frac_packed"),
                "path_frac": path["frac"], "path": path, "kernels": kernels,
                "hbm_peak_gbs": hbm_gbs, "hbm_peak_of": hbm_of}

    # Consecutive pairs on two and on four handles and streams, so that one
    # pair's HBM-bound WTA overlaps other pairs' aggregation (how a stream of
    # frames is best run; reported beside the one-pair-per-step value).
    concurrency = None
    if world == 1:
        n2 = max(10, min(args.steps, 200))
        ms2 = stream_rate(torch, sgm, fp, 2, n2, stream)
        ms4 = stream_rate(torch, sgm, fp, 4, n2, stream)
        concurrency = {"streams": 2, "pairs": n2, "ms_per_pair": ms2,
                       "value": de / (ms2 / 1e3) / 1e6, "unit": "MDE/s",
                       "four_streams": {"ms_per_pair": ms4, "value": de / (ms4 / 1e3) / 1e6}}

    e2e = e2e_run(torch, sgm, fp, stream, max(3, min(args.steps, 200)), world)

    # next rows, timed after the headline loop: map post-processing (Sec. 3.2)
    # and the pipeline reading its inputs through identity rectification maps
    # (Sec. 3.1.1)
    extras = {}
    if w.uv:
        uo = torch.empty((w.D, w.W), dtype=torch.uint8, device="cuda")
        vo = torch.empty((w.H, w.D), dtype=torch.uint8, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sgm.uvmap_postprocess(h, umap, vmap, 3, 6, None, None, 1, uo, vo, stream)
        e0.record(stream)
        for _ in range(50):
            sgm.uvmap_postprocess(h, umap, vmap, 3, 6, None, None, 1, uo, vo, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["uv_postprocess_us"] = e0.elapsed_time(e1) / 50 * 1e3
    yy, xx = np.mgrid[0:w.H, 0:w.W]
    mx = torch.from_numpy(xx.astype(np.int16)).cuda()
    my = torch.from_numpy(yy.astype(np.int16)).cuda()
    sgm.sgm_set_rectification(h, mx, my, mx, my)
    for _ in range(3):
        h.compute(left, right, disp, stream)
    sgm.sgm_set_timing(h, True)
    sgm.sgm_get_stage_times(h)
    for _ in range(50):
        h.compute(left, right, disp, stream)
    rect_stage = sgm.sgm_get_stage_times(h)
    sgm.sgm_set_timing(h, False)
    sgm.sgm_set_rectification(h)
    extras["census_rectified_us"] = rect_stage["census"][0] / max(rect_stage["census"][1], 1) * 1e3

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = w.H
        reps = args.cpu_frames
        dt1, de1 = time_oracle(w, scene, rows, reps)
        pool = OraclePool()
        dt, de_cpu = pool.run(w, scene, rows, 1)
        pool.close()
        cpu = {"value": de_cpu / dt / 1e6, "unit": "MDE/s", "cores": pool.procs, "kind": "oracle",
               "sample": (f"{pool.procs} full {w.W}x{w.H} pairs at once, one process per host "
                          f"core, {dt:.1f} s wall; single thread: {de1 / dt1 / 1e6:.2f} MDE/s "
                          f"({reps} pair(s), {dt1:.1f} s)"),
               "single_thread_value": de1 / dt1 / 1e6}

    # every other workload of the metric, timed the same way (rank 0, one GPU)
    per_config = None
    if rank == 0 and world == 1 and not args.no_per_config:
        per_config = {}
        for name, wi in sorted(WORKLOAD_INDEX.items(), key=lambda kv: kv[1]):
            if name == w.name:
                continue
            per_config[name] = per_config_line(torch, sgm, scenes.WORKLOADS[name], wi, min(args.steps, 50),
                                               stream, flush, peaks, hbm_gbs)
        per_config["batch-64-mixed-census9x7-8path"] = batch_summary(torch, sgm, steps=min(args.steps, 10),
                                                                     warmup=3)
        per_config["serve-8cams-30fps-4GB"] = serve_summary(torch, args.line_serve_seconds)

    # planes: census (or SAD cost), cost, aggregate, wta_lr; sweep: census and
    # the sweep; then median (a device copy when off) and U/V
    swept = sgm.sgm_get_schedule(h)[0] == sgm.SGM_SCHEDULE_SWEEP
    launches_per_step = (2 if swept else (3 if w.cost == 1 else 4)) + (1 if w.median_k > 1 else 0) + (1 if w.uv else 0)
    if rank == 0:
        line = {
            "metric": "MDE/s", "value": value, "unit": "MDE/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": dict(workload_config(w), parallelism=f"replicas{world}",
                           agg_blocks_per_sm=bps if bps is not None else "default",
                           schedule=["auto", "planes", "sweep"][sgm.sgm_get_schedule(h)[0]],
                           agg_chunks_per_lane=sgm.sgm_get_aggregation(h)[1],
                           l2="flushed between steps (256 MiB write outside the timed events)"),
            "fps": 1e3 / ms_per_step * world,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
            "concurrency": concurrency,
            "stage_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in stage.items() if v[1]},
            "next_rows": extras,
            "per_config": per_config,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    fp.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# extra modes: batched pairs and continuous serving (not the headline line)
# ---------------------------------------------------------------------------

def batch_specs(n=64, seed=1807 + 3):
    rng = scenes.Rng(seed)
    sizes = [(320, 240), (640, 480), (1242, 375), (1280, 720)]
    si = rng.integers(0, 3, n)
    di = rng.integers(0, 1, n)
    return [(sizes[a][0], sizes[a][1], (64, 128)[b]) for a, b in zip(si, di)]


class BatchSet:
    """The 64 mixed pairs of the batched workload (9x7 census, 8 paths, P1=8,
    P2=96, LR 1, 3x3 median, U/V maps; sizes from {320x240, 640x480,
    1242x375, 1280x720}, D from {64, 128}, per-pair seeds), their handles
    (tuned per shape by sgm_autotune) and device buffers."""

    def __init__(self, torch, sgm):
        self.specs = batch_specs()
        p = sgm.SgmParams(census_w=9, census_h=7, path_mask=0xFF, P1=8, P2=96, lr_tolerance=1, median_k=3)
        self.params = p
        self.hs, self.L, self.R, self.Dd, self.U, self.V, self.pairs = [], [], [], [], [], [], []
        for i, (W, H, D) in enumerate(self.specs):
            sc = scenes.ground_scene(W, H, D, seed=1807 + 3 + i, n_obstacles=3, dlo=D // 6, dhi=(D * 6) // 7,
                                     texture="value", sigma=2.0, occlusion=0.05)
            self.pairs.append((sc.left, sc.right, (D, 9, 7, 0xFF, 8, 96, 1, 3, True, 0)))
            self.hs.append(sgm.Handle(W, H, D, p))
            self.L.append(torch.from_numpy(sc.left).cuda())
            self.R.append(torch.from_numpy(sc.right).cuda())
            self.Dd.append(torch.empty((H, W), dtype=torch.uint8, device="cuda"))
            self.U.append(torch.empty((D, W), dtype=torch.int16, device="cuda"))
            self.V.append(torch.empty((H, D), dtype=torch.int16, device="cuda"))
        self.tuned = {}
        for i, (W, H, D) in enumerate(self.specs):
            if (W, H, D) not in self.tuned:
                self.tuned[(W, H, D)] = sgm.sgm_autotune(self.hs[i], self.L[i], self.R[i], self.Dd[i])
        for i, (W, H, D) in enumerate(self.specs):  # handles made before tuning pick it up here
            self.hs[i].close()
            self.hs[i] = sgm.Handle(W, H, D, p)
        self.de = sum(W * H * D for W, H, D in self.specs)
        self.device_bytes = sum(sum(sgm.sgm_scratch_bytes(W, H, D, p)[:1]) for W, H, D in self.specs)

    def close(self):
        for h in self.hs:
            h.close()


def batch_timings(torch, sgm, bs, steps, warmup):
    """(engine ms, graph-of-handles ms, one-by-one ms, engine tuning) per batch step."""
    st = torch.cuda.current_stream()

    def timed(fn, n):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    graph_ms = timed(lambda: sgm.sgm_batch_compute(bs.hs, bs.L, bs.R, bs.Dd, bs.U, bs.V, st), steps)
    # the batch engine: pooled scratch, one persistent aggregation launch per
    # group of pairs, grouping and blocks per SM chosen by its tuner
    eng = sgm.Batch(bs.specs, bs.params)
    tuning = eng.autotune(bs.L, bs.R, bs.Dd, bs.U, bs.V, st)
    batch_ms = timed(lambda: eng.run(bs.L, bs.R, bs.Dd, bs.U, bs.V, st), steps)
    bs.engine_bytes = eng.device_bytes()
    eng.close()

    def one_by_one():
        for i in range(len(bs.specs)):
            bs.hs[i].compute(bs.L[i], bs.R[i], bs.Dd[i], st)
            bs.hs[i].uvmap(bs.Dd[i], bs.U[i], bs.V[i], st)
    seq_ms = timed(one_by_one, max(1, steps // 4))
    return batch_ms, graph_ms, seq_ms, tuning


def batch_summary(torch, sgm, steps, warmup):
    """The batch engine's value beside the graph of single-pair pipelines and
    the same pairs launched one by one."""
    bs = BatchSet(torch, sgm)
    batch_ms, graph_ms, seq_ms, tuning = batch_timings(torch, sgm, bs, steps, warmup)
    out = {"config": {"workload": "batch-64-mixed-census9x7-8path", "pairs": len(bs.specs), "de_per_step": bs.de,
                      "engine_groups": tuning[0], "engine_blocks_per_sm": tuning[1],
                      "engine_chunks_per_lane": tuning[2]},
           "value": bs.de / (batch_ms / 1e3) / 1e6, "unit": "MDE/s", "ms_per_step": batch_ms, "steps": steps,
           "api": "sgm_batch_run (pooled scratch, one aggregation launch per group)",
           "graph_of_handles": {"ms_per_step": graph_ms, "value": bs.de / (graph_ms / 1e3) / 1e6,
                                "api": "sgm_batch_compute"},
           "one_pair_per_launch": {"ms_per_step": seq_ms, "value": bs.de / (seq_ms / 1e3) / 1e6},
           "device_bytes": bs.engine_bytes, "handles_device_bytes": bs.device_bytes,
           "tuned_blocks_per_sm": {f"{k[0]}x{k[1]}d{k[2]}": v for k, v in bs.tuned.items()}}
    bs.close()
    return out


def run_batch(args):
    """64 pairs of mixed size and disparity range (9x7 census, 8 paths,
    P1=8, P2=96, LR 1, 3x3 median, U/V maps): one graph-replayed batch call per
    step, against the same pairs launched one after another."""
    import torch

    from paper_1807_06271_gb300 import sgm
    torch.cuda.set_device(0)
    bs = BatchSet(torch, sgm)
    batch_ms, graph_ms, seq_ms, tuning = batch_timings(torch, sgm, bs, args.steps, args.warmup)
    line = {"metric": "MDE/s", "value": bs.de / (batch_ms / 1e3) / 1e6, "unit": "MDE/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": "batch-64-mixed-census9x7-8path", "pairs": len(bs.specs),
                       "de_per_step": bs.de, "engine_groups": tuning[0], "engine_blocks_per_sm": tuning[1],
                       "engine_chunks_per_lane": tuning[2],
                       "tuned_blocks_per_sm": {f"{k[0]}x{k[1]}d{k[2]}": v for k, v in bs.tuned.items()}},
            "graph_of_handles": {"ms_per_step": graph_ms, "value": bs.de / (graph_ms / 1e3) / 1e6},
            "one_pair_per_launch": {"ms_per_step": seq_ms, "value": bs.de / (seq_ms / 1e3) / 1e6},
            "device_bytes": bs.engine_bytes, "cpu_baseline": None}
    pairs = bs.pairs
    bs.close()
    if not args.no_cpu_baseline:
        # the oracle over the same 64 pairs, whole pairs spread over one process per host core
        pool = OraclePool()
        dt, de_cpu = pool.run_pairs(pairs)
        pool.close()
        line["cpu_baseline"] = {"value": de_cpu / dt / 1e6, "unit": "MDE/s", "cores": pool.procs, "kind": "oracle",
                                "sample": f"all {len(pairs)} pairs of the batch once, {dt:.1f} s wall"}
    print(json.dumps(line), flush=True)
    return 0


def serve_run(seconds):
    """8 cameras (4 x 640x480 D=64, 4 x 1280x720 D=128) with Poisson arrivals
    at 30 fps each, full path + U/V per frame, 4 GB device-memory budget."""
    from paper_1807_06271_gb300 import serving
    specs = serving.camera_streams()
    frames = serving.stream_frames(specs, per_stream=4)
    ex = serving.CudaExecutor(specs, frames)
    sch = serving.Scheduler(specs, ex, memory_budget=4 << 30)
    # the warm-up run creates the slots the measured run reuses (one pool of
    # slots, all within the budget); its latencies are dropped
    sch.run(serving.poisson_schedule(specs, duration_s=0.5, seed=1), speed=1.0)
    sch.reset_stats()
    st = sch.run(serving.poisson_schedule(specs, duration_s=seconds, seed=1807 + 4))
    ex.close()
    return specs, frames, st.summary()


def serve_summary(torch, seconds):
    _, _, sm = serve_run(seconds)
    return {"config": {"workload": "serve-8cams-30fps-4GB", "seconds": seconds,
                       "note": ("shortened to keep the default line within minutes; the workload's 60 s run is "
                                "`bench.py --mode serve`") if seconds < 60 else "full 60 s run"},
            "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"], "max_ms": sm["max_ms"], "frames": sm["frames"],
            "mde_per_s": sm["mde_per_s"], "slots": sm["slots"], "device_bytes": sm["device_bytes"],
            "max_queue": sm["max_queue"]}


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    specs, frames, sm = serve_run(args.serve_seconds)
    line = {"metric": "p99 latency", "value": sm["p99_ms"], "unit": "ms", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "serve-8cams-30fps-4GB", "seconds": args.serve_seconds},
            "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"], "max_ms": sm["max_ms"],
            "frames": sm["frames"], "mde_per_s": sm["mde_per_s"], "slots": sm["slots"],
            "device_bytes": sm["device_bytes"], "max_queue": sm["max_queue"], "cpu_baseline": None}
    if not args.no_cpu_baseline:
        # the oracle per camera type: one frame each, single thread, and the
        # frame rate with one frame per host core
        import oracle
        per_frame, tasks = {}, []
        for si, spec in enumerate(specs):
            left, right = frames[si][0]
            fields = (spec.D, 9, 7, 0xFF, 8, 96, 1, 3, True, 0)
            key = f"{spec.W}x{spec.H}d{spec.D}"
            if key not in per_frame:
                t0 = time.perf_counter()
                oracle.sgm(left, right, *fields[:8], uv=True)
                per_frame[key] = (time.perf_counter() - t0) * 1e3
            tasks.append((left, right, fields))
        pool = OraclePool()
        tasks = (tasks * ((pool.procs + len(tasks) - 1) // len(tasks)))[:max(pool.procs, len(tasks))]
        dt, _ = pool.run_pairs(tasks)
        pool.close()
        line["cpu_baseline"] = {"per_frame_ms": per_frame, "unit": "ms", "cores": 1, "kind": "oracle",
                                "all_cores_fps": len(tasks) / dt, "all_cores": pool.procs,
                                "sample": "one frame of each camera type on one core; the camera mix, "
                                          "one frame per host core, for all_cores_fps"}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="kitti-1242x375-d128-census9x7-8path",
                    choices=sorted(WORKLOAD_INDEX))
    ap.add_argument("--cpu-frames", type=int, default=1,
                    help="pairs for the single-thread oracle timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default aggregation blocks per SM instead of sgm_autotune's choice")
    ap.add_argument("--mode", choices=["frame", "batch", "serve"], default="frame",
                    help="frame: the headline single-pair line; batch: 64 mixed pairs per step; "
                         "serve: 8 Poisson camera streams")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the --mode serve run (the workload's 60 s)")
    ap.add_argument("--line-serve-seconds", type=float, default=15.0,
                    help="length of the serve run inside the default frame line's per_config")
    ap.add_argument("--no-per-config", action="store_true",
                    help="time only the headline workload (no per_config block)")
    ap.add_argument("--schedule", choices=["auto", "planes", "sweep"], default="auto",
                    help="path schedule of the headline pair (auto: the tuner's choice)")
    ap.add_argument("--sweep-rows", type=int, default=8, help="rows per thread block with --schedule sweep")
    ap.add_argument("--cost-kernel", choices=["auto", "cuda_cores", "tensor_cores"], default="auto",
                    help="Hamming cost kernel of the headline pair")
    ap.add_argument("--reference-seconds", type=float, default=120.0,
                    help="host time the reference arm's warm-up plus timed steps should take")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    w = scenes.WORKLOADS[args.workload]
    windex = WORKLOAD_INDEX[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, windex)
    return run_ours(args, w, windex)


if __name__ == "__main__":
    sys.exit(main())
