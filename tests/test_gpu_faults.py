"""Fault detection that faults no GPU (GPU tests).

- An injected allocation failure at any step makes the call return
  SGM_ERR_OOM, releases what it had allocated and leaves the library usable.
- Canary bytes around every device buffer of a handle stay intact across all
  entry points (no kernel writes outside its scratch), and the check sees a
  changed guard byte; the caller's output buffers are checked the same way
  from here.
- A bounded device wait that runs out reports SGM_ERR_TIMEOUT
  (test_bounded_wait_reports_timeout_and_handle_recovers in test_gpu_parity.py).
"""
import numpy as np
import pytest

import oracle
from paper_1807_06271_gb300 import scenes, sgm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

PAD = 4096  # guard bytes around the caller's output buffers


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def params(cw, ch, mask, P1, P2, tol=1, k=3, cost=sgm.SGM_COST_CENSUS):
    return sgm.SgmParams(census_w=cw, census_h=ch, path_mask=mask, P1=P1, P2=P2,
                         lr_tolerance=tol, median_k=k, cost=cost)


def padded(shape, dtype):
    """A device view of `shape` inside a buffer with PAD guard elements of 0x5A
    bytes on both sides; returns (view, whole buffer)."""
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * PAD,), 0x5A5A if dtype != torch.uint8 else 0x5A, dtype=dtype, device="cuda")
    return buf[PAD:PAD + n].view(*shape), buf


def guards_intact(buf):
    torch.cuda.synchronize()
    fill = 0x5A5A if buf.dtype != torch.uint8 else 0x5A
    return bool((buf[:PAD] == fill).all()) and bool((buf[-PAD:] == fill).all())


@pytest.fixture(autouse=True)
def hooks_off():
    yield
    sgm.sgm_debug_fail_alloc(0)
    sgm.sgm_debug_canaries(False)


def test_allocation_failure_at_every_step_of_create():
    W, H, D = 301, 37, 60
    s = scenes.boxes_scene(W, H, D, seed=3, n_boxes=3, dlo=2, dhi=D - 2)
    o = oracle.sgm(s.left, s.right, D, 9, 7, 0xFF, 8, 96, 1, 3, uv=False)["disp"]
    L, R = cuda(s.left), cuda(s.right)
    disp = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    before = free_bytes()
    failed = 0
    for n in range(1, 16):
        sgm.sgm_debug_fail_alloc(n)
        try:
            h = sgm.Handle(W, H, D, params(9, 7, 0xFF, 8, 96))
        except sgm.SgmError as e:
            assert e.status == sgm.SGM_ERR_OOM
            assert abs(free_bytes() - before) < (4 << 20), "a failed create kept device memory"
            failed += 1
            continue
        sgm.sgm_debug_fail_alloc(0)  # create needed fewer than n allocations
        h.compute(L, R, disp)
        torch.cuda.synchronize()
        assert np.array_equal(disp.cpu().numpy(), o)
        h.close()
        break
    # codes, cost volume, work-queue state, planes, LR map
    assert failed == 5
    assert abs(free_bytes() - before) < (4 << 20)


def test_allocation_failure_in_host_staging_recovers():
    w = scenes.SMALL_320
    s = scenes.scene_for(w, scenes.workload_seed(0))
    o = oracle.sgm(s.left, s.right, w.D, w.census_w, w.census_h, w.path_mask, w.P1, w.P2,
                   w.lr_tol, w.median_k)
    p = params(w.census_w, w.census_h, w.path_mask, w.P1, w.P2, w.lr_tol, w.median_k)
    with sgm.Handle(w.W, w.H, w.D, p) as h:
        disp = np.empty((w.H, w.W), np.uint8)
        U = np.empty((w.D, w.W), np.uint16)
        V = np.empty((w.H, w.D), np.uint16)
        for n in (1, 3, 5):  # the first, third and last staging buffer of the slot
            sgm.sgm_debug_fail_alloc(n)
            with pytest.raises(sgm.SgmError) as e:
                sgm.sgm_compute_host(h, s.left, s.right, disp, U, V)
            assert e.value.status == sgm.SGM_ERR_OOM
        sgm.sgm_debug_fail_alloc(0)
        sgm.sgm_compute_host(h, s.left, s.right, disp, U, V)
        assert np.array_equal(disp, o["disp"]) and np.array_equal(U, o["U"]) and np.array_equal(V, o["V"])


CANARY_CASES = [
    # W, H, D, cw, ch, mask, P1, P2, cost
    (301, 9, 60, 5, 5, 0xFF, 4, 24, sgm.SGM_COST_CENSUS),
    (129, 40, 128, 9, 7, 0xFF, 8, 96, sgm.SGM_COST_CENSUS),
    (97, 31, 100, 9, 7, 0x55, 7, 50, sgm.SGM_COST_CENSUS),
    (45, 13, 255, 3, 3, 0x0F, 2, 20, sgm.SGM_COST_CENSUS),
    (160, 24, 64, 5, 5, 0x55, 200, 800, sgm.SGM_COST_SAD),
]


@pytest.mark.parametrize("case", CANARY_CASES, ids=lambda c: "x".join(map(str, c[:3])) + ("-sad" if c[8] else ""))
def test_canaries_stay_intact_over_every_entry_point(case):
    W, H, D, cw, ch, mask, P1, P2, cost = case
    s = scenes.boxes_scene(W, H, D, seed=W + H, n_boxes=3, dlo=1, dhi=D - 1)
    L, R = cuda(s.left), cuda(s.right)
    sgm.sgm_debug_canaries(True)
    h = sgm.Handle(W, H, D, params(cw, ch, mask, P1, P2, cost=cost))
    sgm.sgm_debug_canaries(False)
    try:
        disp, dbuf = padded((H, W), torch.uint8)
        U, ubuf = padded((D, W), torch.int16)
        V, vbuf = padded((H, D), torch.int16)
        h.compute(L, R, disp)
        h.uvmap(disp, U, V)
        if cost == sgm.SGM_COST_CENSUS:
            cl, clb = padded((H, W), torch.int64)
            cr, crb = padded((H, W), torch.int64)
            sgm.sgm_debug_census(h, L, R, cl, cr)
            kernels = [sgm.SGM_COST_KERNEL_CUDA_CORES]
            if 16 < D <= 128:
                kernels.append(sgm.SGM_COST_KERNEL_TENSOR_CORES)
            for k in kernels:
                C, cb = padded((H, W, D), torch.int16)
                sgm.sgm_debug_cost(h, L, R, C, k)
                assert guards_intact(cb)
                sgm.sgm_set_cost_kernel(h, k)
                h.compute(L, R, disp)
            sgm.sgm_set_cost_kernel(h, sgm.SGM_COST_KERNEL_AUTO)
            assert guards_intact(clb) and guards_intact(crb)
        for r in range(8):
            if (mask >> r) & 1:
                Lr, lb = padded((H, W, D), torch.int16)
                sgm.sgm_debug_path(h, r, L, R, Lr)
                assert guards_intact(lb)
        S, sb = padded((H, W, D), torch.int16)
        sgm.sgm_debug_sum(h, L, R, S)
        raws = [padded((H, W), torch.uint8) for _ in range(3)]
        sgm.sgm_debug_raw(h, L, R, *(v for v, _ in raws))
        hd = np.empty((H, W), np.uint8)
        hu = np.empty((D, W), np.uint16)
        hv = np.empty((H, D), np.uint16)
        sgm.sgm_compute_host(h, s.left, s.right, hd, hu, hv)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pl, pr = pin(s.left), pin(s.right)
        outs = [(torch.empty((H, W), dtype=torch.uint8).pin_memory(),
                 torch.empty((D, W), dtype=torch.int16).pin_memory(),
                 torch.empty((H, D), dtype=torch.int16).pin_memory()) for _ in range(3)]
        tickets = [sgm.sgm_compute_host_async(h, pl.numpy(), pr.numpy(), d.numpy(), u.numpy().view(np.uint16),
                                              v.numpy().view(np.uint16)) for d, u, v in outs]
        for t in tickets:
            sgm.sgm_host_wait(h, t)
        assert sgm.sgm_debug_check_canaries(h) == sgm.SGM_OK
        for b in [dbuf, ubuf, vbuf, sb] + [b for _, b in raws]:
            assert guards_intact(b)
        # the check itself: a changed guard byte after the first buffer is seen
        sgm.sgm_debug_poke_canary(h, 0)
        assert sgm.sgm_debug_check_canaries(h) == sgm.SGM_ERR_OVERRUN
    finally:
        h.close()


def test_canary_hooks_reject_handles_without_canaries():
    with sgm.Handle(32, 8, 16, params(5, 5, 0x0F, 4, 24)) as h:
        assert sgm.sgm_debug_check_canaries(h) == sgm.SGM_ERR_UNSUPPORTED
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_debug_poke_canary(h, 0)
        assert e.value.status == sgm.SGM_ERR_UNSUPPORTED
