"""Continuous serving of stereo frames from several camera streams.

Frames arrive per stream as a Poisson process.  A frame is admitted as soon as
a slot of its stream's shape is free; a new slot (one sgm handle plus pinned
host and device buffers, on its own CUDA stream) is created while the
device-memory budget allows, so frames that arrive while others are on the
GPU start right away and overlap on the device.  Frames that find no slot
wait in arrival order.  Every frame runs the full path (census, cost,
aggregation, WTA + LR, median, U-/V-maps) through the C ABI, and its latency
is measured from arrival to the completion of its device->host copy.

The scheduler is host logic with a pluggable executor: ``CudaExecutor`` runs
frames on the GPU; tests drive the same scheduler with a fake executor.
"""
from __future__ import annotations

import heapq
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class StreamSpec:
    name: str
    W: int
    H: int
    D: int
    fps: float
    census_w: int = 9
    census_h: int = 7
    path_mask: int = 0xFF
    P1: int = 8
    P2: int = 96
    lr_tolerance: int = 1
    median_k: int = 3

    @property
    def shape_key(self):
        return (self.W, self.H, self.D, self.census_w, self.census_h, self.path_mask, self.P1,
                self.P2, self.lr_tolerance, self.median_k)


def slot_device_bytes(spec: StreamSpec) -> int:
    """Device memory of one slot, as the library reports it: the handle's
    scratch (census codes, cost volume, path planes, LR map, work-queue state)
    plus the two staging slots of its pipelined host-buffer entry point."""
    from . import sgm
    p = sgm.SgmParams(census_w=spec.census_w, census_h=spec.census_h, path_mask=spec.path_mask,
                      P1=spec.P1, P2=spec.P2, lr_tolerance=spec.lr_tolerance, median_k=spec.median_k)
    handle, staging, _ = sgm.sgm_scratch_bytes(spec.W, spec.H, spec.D, p)
    return handle + staging


@dataclass
class Frame:
    stream: int
    index: int
    arrival: float
    start: float = 0.0
    done: float = 0.0


@dataclass
class Stats:
    latencies_ms: list = field(default_factory=list)
    frames: int = 0
    de: int = 0
    wall_s: float = 0.0
    max_slots: int = 0
    max_bytes: int = 0
    max_queue: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"frames": self.frames, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                "mde_per_s": self.de / max(self.wall_s, 1e-9) / 1e6, "wall_s": self.wall_s,
                "slots": self.max_slots, "device_bytes": self.max_bytes,
                "max_queue": self.max_queue}


def poisson_schedule(specs, duration_s: float, seed: int):
    """Arrival times per stream: exponential gaps with mean 1/fps (SplitMix64
    uniforms from the scenes module, so every machine draws the same times)."""
    from . import scenes
    rng = scenes.Rng(seed)
    events = []
    for s, spec in enumerate(specs):
        t, i = 0.0, 0
        while True:
            u = float(rng.uniform(1)[0])
            t += -np.log(1.0 - u) / spec.fps
            if t >= duration_s:
                break
            events.append((t, s, i))
            i += 1
    events.sort()
    return events


class Scheduler:
    """Admission and completion bookkeeping, independent of the device."""

    def __init__(self, specs, executor, memory_budget: int):
        self.specs = list(specs)
        self.ex = executor
        self.budget = memory_budget
        self.free = {}        # shape key -> list of idle slot ids
        self.busy = {}        # slot id -> Frame
        self.slot_key = {}    # slot id -> shape key
        self.bytes = 0
        self.queue = deque()
        self.stats = Stats()

    def _slot_for(self, spec):
        key = spec.shape_key
        idle = self.free.setdefault(key, [])
        if idle:
            return idle.pop()
        need = slot_device_bytes(spec)
        if self.bytes + need > self.budget:
            return None
        sid = self.ex.create_slot(spec)
        self.slot_key[sid] = key
        self.bytes += need
        self.stats.max_slots = max(self.stats.max_slots, len(self.slot_key))
        self.stats.max_bytes = max(self.stats.max_bytes, self.bytes)
        return sid

    def arrive(self, frame: Frame):
        self.queue.append(frame)
        self.stats.max_queue = max(self.stats.max_queue, len(self.queue))

    def admit(self, now: float):
        """Start waiting frames in arrival order while slots are available;
        a frame that cannot start does not block other shapes behind it."""
        waiting = deque()
        while self.queue:
            f = self.queue.popleft()
            sid = self._slot_for(self.specs[f.stream])
            if sid is None:
                waiting.append(f)
                continue
            f.start = now
            self.busy[sid] = f
            self.ex.launch(sid, f)
        self.queue = waiting

    def complete(self, now: float):
        for sid in [s for s in self.busy if self.ex.done(s)]:
            f = self.busy.pop(sid)
            f.done = now
            spec = self.specs[f.stream]
            self.stats.latencies_ms.append((f.done - f.arrival) * 1e3)
            self.stats.frames += 1
            self.stats.de += spec.W * spec.H * spec.D
            self.ex.finished(sid, f)
            self.free[self.slot_key[sid]].append(sid)

    def idle(self) -> bool:
        return not self.busy and not self.queue

    def reset_stats(self):
        """New statistics for the next run, keeping the slots (a warm-up run
        creates them; the measured run then reuses them)."""
        self.stats = Stats(max_slots=len(self.slot_key), max_bytes=self.bytes)

    def run(self, schedule, clock=time.perf_counter, speed: float = 1.0):
        """Replays (time, stream, index) arrivals against the wall clock
        (``speed`` > 1 compresses time) until every frame has completed."""
        t0 = clock()
        pending = list(schedule)
        heapq.heapify(pending)
        while pending or not self.idle():
            now = clock()
            sim = (now - t0) * speed
            while pending and pending[0][0] <= sim:
                t, s, i = heapq.heappop(pending)
                self.arrive(Frame(s, i, t0 + t / speed))
            self.admit(now)
            self.complete(clock())
        self.stats.wall_s = clock() - t0
        return self.stats


class CudaExecutor:
    """Runs frames through the CUDA library: one handle, one CUDA stream and
    pinned host + device buffers per slot; inputs come from a fixed set of
    frames per stream."""

    def __init__(self, specs, frames_per_stream, keep_results: bool = False):
        import torch
        from . import sgm
        self.torch, self.sgm = torch, sgm
        self.specs = specs
        self.frames = frames_per_stream  # stream -> list of (left, right) numpy arrays
        self.slots = []
        self.keep = keep_results
        self.results = {}  # (stream, index) -> (disp, U, V)

    def create_slot(self, spec):
        torch, sgm = self.torch, self.sgm
        p = sgm.SgmParams(census_w=spec.census_w, census_h=spec.census_h, path_mask=spec.path_mask,
                          P1=spec.P1, P2=spec.P2, lr_tolerance=spec.lr_tolerance,
                          median_k=spec.median_k)
        slot = {
            "h": sgm.Handle(spec.W, spec.H, spec.D, p),
            "stream": torch.cuda.Stream(),
            "ev": torch.cuda.Event(),
            "hl": torch.empty((spec.H, spec.W), dtype=torch.uint8).pin_memory(),
            "hr": torch.empty((spec.H, spec.W), dtype=torch.uint8).pin_memory(),
            "hd": torch.empty((spec.H, spec.W), dtype=torch.uint8).pin_memory(),
            "hu": torch.empty((spec.D, spec.W), dtype=torch.int16).pin_memory(),
            "hv": torch.empty((spec.H, spec.D), dtype=torch.int16).pin_memory(),
            "dl": torch.empty((spec.H, spec.W), dtype=torch.uint8, device="cuda"),
            "dr": torch.empty((spec.H, spec.W), dtype=torch.uint8, device="cuda"),
            "dd": torch.empty((spec.H, spec.W), dtype=torch.uint8, device="cuda"),
            "du": torch.empty((spec.D, spec.W), dtype=torch.int16, device="cuda"),
            "dv": torch.empty((spec.H, spec.D), dtype=torch.int16, device="cuda"),
        }
        self.slots.append(slot)
        return len(self.slots) - 1

    def launch(self, sid, frame):
        torch, sgm = self.torch, self.sgm
        sl = self.slots[sid]
        left, right = self.frames[frame.stream][frame.index % len(self.frames[frame.stream])]
        sl["hl"].numpy()[...] = left
        sl["hr"].numpy()[...] = right
        st = sl["stream"]
        with torch.cuda.stream(st):
            sl["dl"].copy_(sl["hl"], non_blocking=True)
            sl["dr"].copy_(sl["hr"], non_blocking=True)
            sgm.sgm_compute(sl["h"], sl["dl"], sl["dr"], sl["dd"], st)
            sgm.uvmap_compute(sl["h"], sl["dd"], sl["du"], sl["dv"], st)
            sl["hd"].copy_(sl["dd"], non_blocking=True)
            sl["hu"].copy_(sl["du"], non_blocking=True)
            sl["hv"].copy_(sl["dv"], non_blocking=True)
            sl["ev"].record(st)

    def done(self, sid):
        return self.slots[sid]["ev"].query()

    def finished(self, sid, frame):
        if self.keep:
            sl = self.slots[sid]
            self.results[(frame.stream, frame.index)] = (
                sl["hd"].numpy().copy(), sl["hu"].numpy().view(np.uint16).copy(),
                sl["hv"].numpy().view(np.uint16).copy())

    def close(self):
        for sl in self.slots:
            sl["h"].close()
        self.slots = []


def camera_streams(n_vga: int = 4, n_hd: int = 4, fps: float = 30.0):
    """Eight simulated cameras: 640x480 with D=64 and 1280x720 with D=128,
    8 paths, 9x7 census, P1=8, P2=96, LR tolerance 1, 3x3 median."""
    specs = [StreamSpec(f"vga{i}", 640, 480, 64, fps) for i in range(n_vga)]
    specs += [StreamSpec(f"hd{i}", 1280, 720, 128, fps) for i in range(n_hd)]
    return specs


def stream_frames(specs, per_stream: int = 4, seed: int = 1807 + 4):
    """Seeded synthetic frames per stream (the boxes-scene recipe)."""
    from . import scenes
    out = []
    for s, spec in enumerate(specs):
        frames = []
        for i in range(per_stream):
            sc = scenes.boxes_scene(spec.W, spec.H, spec.D, seed=seed + 100 * s + i, n_boxes=4,
                                    dlo=4, dhi=min(60, spec.D - 1), texture="blur", sigma=1.0)
            frames.append((sc.left, sc.right))
        out.append(frames)
    return out
