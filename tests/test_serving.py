"""Serving scheduler: admission under a device-memory budget, arrival-order
waiting, overlap, latency statistics (CPU, fake executor) and, on the GPU,
every served frame equal to the same frame computed alone."""
import numpy as np
import pytest

from paper_1807_06271_gb300 import serving


class FakeExecutor:
    """Each frame takes `service` seconds of fake device time from its launch."""

    def __init__(self, clock, service):
        self.clock, self.service = clock, service
        self.slots, self.launched, self.running = 0, [], {}

    def create_slot(self, spec):
        self.slots += 1
        return self.slots - 1

    def launch(self, sid, f):
        self.launched.append((sid, f.stream, f.index))
        self.running[sid] = self.clock() + self.service

    def done(self, sid):
        return self.clock() >= self.running[sid]

    def finished(self, sid, f):
        del self.running[sid]


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4  # every reading advances time a little
        return self.t


def test_budget_limits_slots_and_frames_wait_in_order():
    spec = serving.StreamSpec("a", 64, 48, 32, fps=1000.0)
    need = serving.slot_device_bytes(spec)
    clock = FakeClock()
    ex = FakeExecutor(clock, service=0.01)
    sch = serving.Scheduler([spec], ex, memory_budget=2 * need + 1)
    schedule = [(0.0001 * i, 0, i) for i in range(20)]  # a burst of 20 frames
    st = sch.run(schedule, clock=clock)
    assert st.frames == 20 and ex.slots == 2 and st.max_bytes <= 2 * need + 1
    # frames start in arrival order and at most two overlap
    assert [i for _, _, i in ex.launched] == list(range(20))
    assert st.max_queue >= 10
    s = st.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_slot_reuse_per_shape_and_no_head_of_line_blocking():
    a = serving.StreamSpec("a", 64, 48, 32, fps=100.0)
    b = serving.StreamSpec("b", 32, 24, 16, fps=100.0)
    clock = FakeClock()
    ex = FakeExecutor(clock, service=0.05)
    # room for one slot of each shape only
    sch = serving.Scheduler([a, b], ex, serving.slot_device_bytes(a) + serving.slot_device_bytes(b))
    sch.arrive(serving.Frame(0, 0, 0.0))
    sch.arrive(serving.Frame(0, 1, 0.0))   # must wait for a's slot
    sch.arrive(serving.Frame(1, 0, 0.0))   # b is not blocked behind a's second frame
    sch.admit(clock())
    started = [(s, i) for _, s, i in ex.launched]
    assert (0, 0) in started and (1, 0) in started and (0, 1) not in started
    assert len(sch.queue) == 1


def test_warm_up_slots_are_reused_by_the_measured_run():
    """A warm-up run creates the slots; after reset_stats the measured run
    reuses them (no slot created while it is timed), counts only its own
    frames and still reports the slots and bytes held."""
    spec = serving.StreamSpec("a", 64, 48, 32, fps=1000.0)
    need = serving.slot_device_bytes(spec)
    clock = FakeClock()
    ex = FakeExecutor(clock, service=0.01)
    sch = serving.Scheduler([spec], ex, memory_budget=2 * need + 1)
    sch.run([(0.0001 * i, 0, i) for i in range(10)], clock=clock)
    assert ex.slots == 2
    sch.reset_stats()
    st = sch.run([(0.0001 * i, 0, i) for i in range(6)], clock=clock)
    assert ex.slots == 2  # nothing new allocated
    assert st.frames == 6 and len(st.latencies_ms) == 6
    assert st.max_slots == 2 and st.max_bytes == 2 * need


def test_poisson_schedule_rates():
    specs = [serving.StreamSpec("a", 8, 8, 8, fps=30.0), serving.StreamSpec("b", 8, 8, 8, fps=60.0)]
    ev = serving.poisson_schedule(specs, duration_s=100.0, seed=7)
    n = np.bincount([s for _, s, _ in ev])
    assert abs(n[0] - 3000) < 300 and abs(n[1] - 6000) < 450
    assert all(ev[i][0] <= ev[i + 1][0] for i in range(len(ev) - 1))


@pytest.mark.gpu
def test_served_frames_equal_frames_computed_alone():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1807_06271_gb300 import sgm
    specs = [serving.StreamSpec(f"vga{i}", 320, 240, 64, fps=400.0) for i in range(3)]
    specs += [serving.StreamSpec("hd", 640, 360, 128, fps=300.0)]
    frames = serving.stream_frames(specs, per_stream=3)
    ex = serving.CudaExecutor(specs, frames, keep_results=True)
    budget = 2 * serving.slot_device_bytes(specs[0]) + 2 * serving.slot_device_bytes(specs[3])
    sch = serving.Scheduler(specs, ex, budget)
    st = sch.run(serving.poisson_schedule(specs, duration_s=0.1, seed=11))
    assert st.frames == len(ex.results) > 20
    assert st.max_slots >= 2  # frames overlapped on the device
    for (s, i), (disp, U, V) in ex.results.items():
        spec = specs[s]
        left, right = frames[s][i % len(frames[s])]
        p = sgm.SgmParams(census_w=9, census_h=7, path_mask=0xFF, P1=8, P2=96, lr_tolerance=1, median_k=3)
        with sgm.Handle(spec.W, spec.H, spec.D, p) as h:
            d = np.empty((spec.H, spec.W), np.uint8)
            u = np.empty((spec.D, spec.W), np.uint16)
            v = np.empty((spec.H, spec.D), np.uint16)
            sgm.sgm_compute_host(h, left, right, d, u, v)
        assert np.array_equal(disp, d) and np.array_equal(U, u) and np.array_equal(V, v), (s, i)
    ex.close()
