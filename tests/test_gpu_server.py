"""Serving loop (continuous batching): results equal single calls, the memory
budget is respected, poll semantics hold, destroy cancels what is pending."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3829_gb300 import hrm as h
    h.lib()
    return h


def _reqs(n, seed=0):
    from paper_1105_3829_gb300 import inputs
    reqs = inputs.request_stream(n, rate=1000.0, seed=seed, side_lo=16, side_hi=300, r_max=20)
    return reqs, [inputs.request_image(q) for q in reqs]


def test_results_equal_single_calls_host_and_device(hrm):
    reqs, imgs = _reqs(60, seed=1)
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    srv = hrm.Server(arena, max_inflight=16)
    pending = []
    for i, (q, a) in enumerate(zip(reqs, imgs)):
        if i % 2:  # host (pinned) buffers: copied through the arena
            src = torch.from_numpy(a).pin_memory()
            dst = torch.zeros_like(src).pin_memory()
        else:      # device-resident buffers: used in place
            src = torch.from_numpy(a).cuda()
            dst = torch.zeros_like(src)
        t = srv.submit(src, dst, q["r"])
        pending.append((t, src, dst, q))
    for t, src, dst, q in pending:
        assert srv.poll(t, -1) == hrm.HRM_OK
        assert srv.latency_us(t) > 0
        ref = hrm.filter2d(src.cuda(), q["r"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dst.cpu().numpy(), ref.cpu().numpy())
    st = srv.stats()
    assert st.completed == len(reqs) and st.inflight == 0 and st.bytes_resident == 0
    assert st.bytes_high_water <= st.arena_bytes
    assert st.waves >= 1
    srv.close()


def test_budget_limits_admission(hrm):
    # arena holds one 256x256 uint16 request (in + out = 256 KiB) at a time
    arena = torch.empty(300 * 1024, dtype=torch.uint8, device="cuda")
    srv = hrm.Server(arena, max_inflight=64)
    tickets = []
    for k in range(6):
        a = np.full((256, 256), k, np.uint16)
        src = torch.from_numpy(a).pin_memory()
        dst = torch.zeros_like(src).pin_memory()
        tickets.append((srv.submit(src, dst, 3), src, dst, k))
    for t, src, dst, k in tickets:
        assert srv.poll(t, 10_000_000) == hrm.HRM_OK
        assert np.all(dst.numpy() == k)
    st = srv.stats()
    assert st.bytes_high_water <= 300 * 1024
    with pytest.raises(hrm.HRMError) as e:  # can never fit
        big = torch.zeros((1024, 1024), dtype=torch.uint16).pin_memory()
        srv.submit(big, big.clone(), 3)
    assert e.value.code == hrm.HRM_EINVAL
    srv.close()


def test_poll_semantics_and_cancel(hrm):
    arena = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    srv = hrm.Server(arena, max_inflight=4, max_queue=2)
    a = torch.zeros((512, 512), dtype=torch.uint16, device="cuda")
    outs = [torch.empty_like(a) for _ in range(8)]
    got_eagain = False
    ts = []
    for o in outs:
        try:
            ts.append(srv.submit(a, o, 50))
        except hrm.HRMError as e:
            assert e.code == hrm.HRM_EAGAIN
            got_eagain = True
    assert got_eagain or len(ts) == 8
    rc = srv.poll(ts[-1], 0)
    assert rc in (hrm.HRM_OK, hrm.HRM_EAGAIN)
    if rc == hrm.HRM_EAGAIN:
        assert srv.poll(ts[-1], 1) in (hrm.HRM_OK, hrm.HRM_ETIMEDOUT)
    for t in ts:
        srv.poll(t, -1)
    assert srv.poll(ts[0], 0) == hrm.HRM_EINVAL  # retired
    srv.close()


def test_destroy_with_pending_requests_returns(hrm):
    arena = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    srv = hrm.Server(arena, max_inflight=2)
    a = torch.zeros((1024, 1024), dtype=torch.uint16, device="cuda")
    outs = [torch.empty_like(a) for _ in range(6)]
    for o in outs:
        srv.submit(a, o, 40)
    t0 = time.time()
    srv.close()  # cancels queued requests, waits for launched waves
    assert time.time() - t0 < 60
