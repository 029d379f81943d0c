"""The no-allocation batch entry point (hrm_filter_batch_noalloc).

It serves callers that cannot allocate device memory (for example while a
stream is being captured, or inside a pooled-memory application), so its
scratch is a fixed device array rather than cudaMalloc'ed buffers.  This test
calls it through the C ABI twice in a row on a mixed batch and compares every
output with the allocating entry point, hrm_filter_batch, bit for bit.  It
lives in its own file, collected last, and passes alone or after the others.
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


def test_noalloc_matches_allocating_batch_twice(hrm):
    for call, seed in enumerate((5, 6)):  # two calls in a row on fresh data
        data = _batch(seed)
        srcs = [torch.from_numpy(a).cuda() for a, _, _ in data]
        ref = [torch.zeros_like(s) for s in srcs]
        got = [torch.full_like(s, 7) for s in srcs]
        hrm.filter_batch([hrm.make_job(s, o, r, adaptive=ad) for s, o, (_, r, ad) in zip(srcs, ref, data)])
        hrm.filter_batch_noalloc([hrm.make_job(s, o, r, adaptive=ad) for s, o, (_, r, ad) in zip(srcs, got, data)])
        torch.cuda.synchronize()
        for o, e in zip(got, ref):
            np.testing.assert_array_equal(o.cpu().numpy(), e.cpu().numpy())


def test_noalloc_rejects_more_than_its_limit(hrm):
    a = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    outs = [torch.empty_like(a) for _ in range(65)]
    with pytest.raises(hrm.HRMError) as e:
        hrm.filter_batch_noalloc([hrm.make_job(a, o, 1) for o in outs])
    assert e.value.code == hrm.HRM_EINVAL
    assert "64" in str(e.value)
