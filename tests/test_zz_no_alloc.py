"""The no-allocation batch entry point (hrm_filter_batch_noalloc).

It serves callers that cannot allocate device memory: frame loops with a hard
latency budget (cudaMalloc may synchronise the device) and programs whose
device memory belongs to their own pooling allocator.  Its scratch is a fixed
device array rather than cudaMalloc'ed buffers.  This test calls it through
the C ABI twice in a row on a mixed batch (2D and 3D, both dtypes, small and
large radii, a radius-0 copy and one frame-stream job) and compares every
output with the allocating entry point, hrm_filter_batch, and with the CPU
oracle, bit for bit.  It also checks that a kernel error word planted in the
array is reported by hrm_device_status and cleared.  It lives in its own file,
collected last, and passes alone or after the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1105_3829_gb300 import hrm as h
    h.lib()
    return h


def _batch(seed):
    from paper_1105_3829_gb300 import inputs
    rng = np.random.default_rng(seed)
    return [
        (inputs.xray12_u16(200, 333, seed=seed), 5, False),
        (rng.integers(0, 256, size=(150, 260)).astype(np.uint8), 3, False),
        (inputs.xray12_u16(96, 140, seed=seed + 1), 1, False),
        (inputs.lowkey16_u16(120, 180, seed=seed + 2), 15, True),
        (inputs.xray12_volume(12, 20, 70, seed=seed + 3), 2, False),
        (rng.integers(0, 4096, size=(33, 47)).astype(np.uint16), 0, False),
    ]


def _expected(oracle, a, r):
    if r == 0:
        return a
    return oracle.median3d(a, r) if a.ndim == 3 else oracle.median2d(a, r)


def test_noalloc_matches_allocating_batch_and_oracle_twice(hrm, oracle):
    from paper_1105_3829_gb300 import inputs
    topo_ref, topo_got = hrm.Topology(), hrm.Topology()
    try:
        for call, seed in enumerate((5, 6)):  # two calls in a row on fresh data
            data = _batch(seed)
            frame = inputs.lowkey16_u16(130, 210, seed=seed + 9)  # one frame of a stream per call
            srcs = [torch.from_numpy(a).cuda() for a, _, _ in data]
            fsrc = torch.from_numpy(frame).cuda()
            ref = [torch.zeros_like(s) for s in srcs] + [torch.zeros_like(fsrc)]
            got = [torch.full_like(s, 7) for s in srcs] + [torch.full_like(fsrc, 7)]
            jobs_ref = [hrm.make_job(s, o, r, adaptive=ad) for s, o, (_, r, ad) in zip(srcs, ref, data)]
            jobs_got = [hrm.make_job(s, o, r, adaptive=ad) for s, o, (_, r, ad) in zip(srcs, got, data)]
            jobs_ref.append(hrm.make_job(fsrc, ref[-1], 12, topo=topo_ref))
            jobs_got.append(hrm.make_job(fsrc, got[-1], 12, topo=topo_got))
            hrm.filter_batch(jobs_ref)
            hrm.filter_batch_noalloc(jobs_got)
            assert hrm.device_status() == hrm.HRM_OK
            torch.cuda.synchronize()
            arrays = [a for a, _, _ in data] + [frame]
            radii = [r for _, r, _ in data] + [12]
            for o, e, a, r in zip(got, ref, arrays, radii):
                g = o.cpu().numpy()
                np.testing.assert_array_equal(g, e.cpu().numpy())
                np.testing.assert_array_equal(g, _expected(oracle, a, r))
            # both frame streams now hold the same top level for the next frame
            assert topo_got.info() == topo_ref.info()
    finally:
        topo_ref.close()
        topo_got.close()


def test_noalloc_error_word_is_reported_and_cleared(hrm):
    a = torch.zeros((40, 50), dtype=torch.uint16, device="cuda")
    o = torch.empty_like(a)
    hrm.filter_batch_noalloc([hrm.make_job(a, o, 7)])
    assert hrm.device_status() == hrm.HRM_OK
    # plant an error code from the host (no kernel is made to fail)
    assert hrm.lib().hrm_debug_set_error_word(0, None, 5) == hrm.HRM_OK
    with pytest.raises(hrm.HRMError) as e:
        hrm.device_status()
    assert e.value.code == hrm.HRM_EDEVICE
    assert "noalloc" in str(e.value)
    assert hrm.device_status() == hrm.HRM_OK  # read once, then cleared


def test_noalloc_rejects_more_than_its_limit(hrm):
    a = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    outs = [torch.empty_like(a) for _ in range(65)]
    with pytest.raises(hrm.HRMError) as e:
        hrm.filter_batch_noalloc([hrm.make_job(a, o, 1) for o in outs])
    assert e.value.code == hrm.HRM_EINVAL
    assert "64" in str(e.value)
