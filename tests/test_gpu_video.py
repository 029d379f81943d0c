"""Frame streams (hrm_filter2d_video): every frame's median equals the oracle
and the single-image call, whatever topology the previous frame left."""
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


@pytest.mark.parametrize("r", [3, 9, 20])
def test_frames_match_oracle_and_single_calls(hrm, oracle, r):
    from paper_1105_3829_gb300 import inputs
    topo = hrm.Topology()
    for f, frame in enumerate(inputs.video_frames(4, 150, 270, drift=6, seed=100 + r)):
        src = torch.from_numpy(frame).cuda()
        got = hrm.filter2d_video(src, r, topo)
        single = hrm.filter2d(src, r)
        hrm.device_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), single.cpu().numpy())
        if f in (0, 3):
            np.testing.assert_array_equal(got.cpu().numpy(), oracle.median2d(frame, r))
    topo.close()


def test_dtype_change_and_unrelated_frames(hrm, oracle):
    """A u8 frame after u16 frames, then a u16 frame unlike the previous ones:
    the stale estimate only costs speed."""
    from paper_1105_3829_gb300 import inputs
    topo = hrm.Topology()
    frames = [next(inputs.video_frames(1, 120, 200, seed=5)),
              np.random.default_rng(1).integers(0, 256, size=(90, 130)).astype(np.uint8),
              inputs.xray12_u16(120, 200, seed=9),
              np.full((64, 64), 65535, np.uint16)]
    for frame in frames:
        src = torch.from_numpy(frame).cuda()
        got = hrm.filter2d_video(src, 12, topo)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.median2d(frame, 12))
    topo.close()


def _u8_frames(n, h, w, seed):
    """A u8 stream: a slowly shifting ramp plus noise."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w]
    for f in range(n):
        base = 90 + 60 * np.sin((xx + 5 * f) / 23.0) + 25 * rng.standard_normal((h, w))
        yield np.clip(np.rint(base), 0, 255).astype(np.uint8)


def _same_top_level(a, b):
    ia, ib = a.info(), b.info()
    assert ia == ib, (ia, ib)
    return ia


@pytest.mark.parametrize("r16,r8", [(12, 9), (4, 30)])
def test_batch_frames_follow_the_video_path(hrm, oracle, r16, r8):
    """Two frame streams (u16 and u8) inside batches with a plain job: every
    output is the exact median, and each topology ends every step holding the
    same top level as the same stream run through hrm_filter2d_video."""
    from paper_1105_3829_gb300 import inputs
    ta, tb, va, vb = hrm.Topology(), hrm.Topology(), hrm.Topology(), hrm.Topology()
    plain = torch.from_numpy(inputs.xray12_u16(100, 140, seed=3)).cuda()
    fa_all = list(inputs.video_frames(4, 130, 210, drift=5, seed=41))
    fb_all = list(_u8_frames(4, 90, 170, seed=42))
    for f in range(4):
        fa, fb = torch.from_numpy(fa_all[f]).cuda(), torch.from_numpy(fb_all[f]).cuda()
        oa, ob, op = torch.empty_like(fa), torch.empty_like(fb), torch.empty_like(plain)
        hrm.filter_batch([hrm.make_job(fa, oa, r16, topo=ta), hrm.make_job(plain, op, 7),
                          hrm.make_job(fb, ob, r8, topo=tb)])
        ra = hrm.filter2d_video(fa, r16, va)
        rb = hrm.filter2d_video(fb, r8, vb)
        hrm.device_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(oa.cpu().numpy(), ra.cpu().numpy())
        np.testing.assert_array_equal(ob.cpu().numpy(), rb.cpu().numpy())
        np.testing.assert_array_equal(op.cpu().numpy(), hrm.filter2d(plain, 7).cpu().numpy())
        if f in (0, 3):
            np.testing.assert_array_equal(oa.cpu().numpy(), oracle.median2d(fa_all[f], r16))
            np.testing.assert_array_equal(ob.cpu().numpy(), oracle.median2d(fb_all[f], r8))
        assert _same_top_level(ta, va)["dtype"] == hrm.HRM_U16
        assert _same_top_level(tb, vb)["dtype"] == hrm.HRM_U8
    for t in (ta, tb, va, vb):
        t.close()


def test_noalloc_batch_and_graph_frames(hrm, oracle):
    """The no-allocation batch and a replayed graph carry the stream too."""
    from paper_1105_3829_gb300 import inputs
    frames = list(inputs.video_frames(5, 120, 180, drift=6, seed=77))
    t, v = hrm.Topology(), hrm.Topology()
    src = torch.from_numpy(frames[0]).cuda()
    out = torch.empty_like(src)
    # a graph needs a topology that already holds a top level of the job's dtype
    with pytest.raises(hrm.HRMError) as e:
        hrm.BatchGraph([hrm.make_job(src, out, 10, topo=t)])
    assert e.value.code == hrm.HRM_EINVAL
    hrm.filter_batch_noalloc([hrm.make_job(src, out, 10, topo=t)])
    ref = hrm.filter2d_video(src, 10, v)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    _same_top_level(t, v)
    g = hrm.BatchGraph([hrm.make_job(src, out, 10, topo=t)])
    for f in range(1, 5):
        src.copy_(torch.from_numpy(frames[f]).cuda())
        g.launch()
        ref = hrm.filter2d_video(src, 10, v)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
        _same_top_level(t, v)
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.median2d(frames[4], 10))
    g.close()
    t.close()
    v.close()


def test_frame_job_argument_errors(hrm):
    t = hrm.Topology()
    a = torch.zeros((32, 32), dtype=torch.uint16, device="cuda")
    b, c = torch.empty_like(a), torch.empty_like(a)
    vol = torch.zeros((4, 16, 16), dtype=torch.uint16, device="cuda")
    bad = [[hrm.make_job(a, b, 3, topo=t), hrm.make_job(a, c, 3, topo=t)],   # one topology twice
           [hrm.make_job(a, b, 3, adaptive=True, topo=t)],                    # flags
           [hrm.make_job(a, b, 3, rank=0, topo=t)],                           # not the median
           [hrm.make_job(vol, torch.empty_like(vol), 1, topo=t)]]             # 3D
    for jobs in bad:
        with pytest.raises(hrm.HRMError) as e:
            hrm.filter_batch(jobs)
        assert e.value.code == hrm.HRM_EINVAL
    assert t.info()["dtype"] == 0   # rejected calls leave the topology untouched
    t.close()


def test_server_frame_streams_keep_order(hrm, oracle):
    """Frames of two streams submitted all at once (with plain requests in
    between) come out as the video path gives them, in submission order, and
    leave the same top levels; no wave holds two frames of one stream."""
    from paper_1105_3829_gb300 import inputs
    n = 6
    fa = [torch.from_numpy(x).cuda() for x in inputs.video_frames(n, 110, 150, drift=4, seed=5)]
    fb = [torch.from_numpy(x) for x in _u8_frames(n, 80, 120, seed=6)]   # host frames
    plain = torch.from_numpy(inputs.xray12_u16(70, 90, seed=8)).cuda()
    arena = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    srv = hrm.Server(arena)
    ta, tb = hrm.Topology(), hrm.Topology()
    try:
        with pytest.raises(hrm.HRMError):
            srv.submit(fa[0], torch.empty_like(fa[0]), 5, adaptive=True, topo=ta)
        tickets = []
        for f in range(n):
            oa, ob, op = torch.empty_like(fa[f]), torch.empty_like(fb[f]), torch.empty_like(plain)
            tickets.append((srv.submit(fa[f], oa, 11, topo=ta), oa, "a", f))
            tickets.append((srv.submit(plain, op, 6), op, "p", f))
            tickets.append((srv.submit(fb[f], ob, 8, topo=tb), ob, "b", f))
        for t, _, _, _ in tickets:
            assert srv.poll(t, -1) == hrm.HRM_OK
        assert srv.stats().waves >= n
    finally:
        srv.close()
    va, vb = hrm.Topology(), hrm.Topology()
    want = {}
    for f in range(n):
        want["a", f] = hrm.filter2d_video(fa[f], 11, va).cpu().numpy()
        want["b", f] = hrm.filter2d_video(fb[f].cuda(), 8, vb).cpu().numpy()
    want_p = hrm.filter2d(plain, 6).cpu().numpy()
    torch.cuda.synchronize()
    for _, out, kind, f in tickets:
        np.testing.assert_array_equal(out.cpu().numpy(), want_p if kind == "p" else want[kind, f])
    np.testing.assert_array_equal(tickets[-1][1].numpy(), oracle.median2d(fb[-1].numpy(), 8))
    _same_top_level(ta, va)
    _same_top_level(tb, vb)
    for t in (ta, tb, va, vb):
        t.close()


def test_server_large_frames_first_waves(hrm):
    """A fresh server whose first wave runs long (whole 2048^2 low-key
    frames) while its next wave starts on the other, still unused compute
    stream: the new stream's buffers must be cleared in that stream's order,
    not on the legacy default stream behind the running kernel."""
    from paper_1105_3829_gb300 import inputs
    fr = [torch.from_numpy(x).cuda() for x in inputs.video_frames(4, 2048, 2048, drift=4, seed=91)]
    arena = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    for with_topo in (False, True):
        srv = hrm.Server(arena, max_inflight=4096, max_queue=16384)
        topos = [hrm.Topology() if with_topo else None for _ in range(4)]
        outs = [[torch.empty_like(fr[0]) for _ in range(2)] for _ in range(4)]
        try:
            tickets = [srv.submit(fr[(k + f) % 4], outs[k][f], 15, topo=topos[k]) for f in range(2) for k in range(4)]
            assert [srv.poll(t, 60_000_000) for t in tickets] == [hrm.HRM_OK] * len(tickets)
        finally:
            srv.close()
        for k in range(4):
            for f in range(2):
                want = hrm.filter2d(fr[(k + f) % 4], 15)
                torch.cuda.synchronize()
                assert torch.equal(outs[k][f].view(torch.int16), want.view(torch.int16)), (with_topo, k, f)
        for t in topos:
            if t is not None:
                t.close()
