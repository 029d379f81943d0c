"""Seeded synthetic workloads: determinism, dtype, value ranges and shape of
the distributions (no filter arithmetic here)."""
import numpy as np
import pytest

from paper_1105_3829_gb300 import inputs


def test_deterministic_and_typed():
    a = inputs.uniform_u8(64, 48)
    b = inputs.uniform_u8(64, 48)
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.uint8 and a.shape == (64, 48)
    x = inputs.xray12_u16(256, 200)
    assert x.dtype == np.uint16 and x.max() <= 4095
    np.testing.assert_array_equal(x, inputs.xray12_u16(256, 200))


def test_xray_mixture_statistics():
    x = inputs.xray12_u16(512, 512).astype(np.int64)
    frac_salt = np.mean((x == 0) | (x == 4095))
    assert 0.007 < frac_salt < 0.013
    low = np.mean(x < 1900)
    assert 0.55 < low < 0.65


def test_lowkey_compact_mode():
    x = inputs.lowkey16_u16(512, 512).astype(np.int64)
    near = np.mean(np.abs(x - 2000) < 800)
    assert 0.85 < near < 0.95
    assert x.max() > 60000


def test_volume_and_octants():
    v = inputs.xray12_volume(32, 32, 32)
    assert v.shape == (32, 32, 32) and v.max() <= 4095
    oc = inputs.octants(v)
    assert len(oc) == 8 and all(o.shape == (16, 16, 16) for o in oc)
    np.testing.assert_array_equal(oc[7], v[16:, 16:, 16:])


def test_request_stream():
    reqs = inputs.request_stream(500, rate=300.0)
    ts = np.array([q["t"] for q in reqs])
    assert np.all(np.diff(ts) >= 0)
    assert all(64 <= q["w"] <= 4096 and 64 <= q["h"] <= 4096 for q in reqs)
    assert all(1 <= q["r"] <= 50 for q in reqs)
    frac16 = np.mean([q["dtype"] == "u16" for q in reqs])
    assert 0.4 < frac16 < 0.6
    img = inputs.request_image(reqs[0])
    assert img.shape == (reqs[0]["h"], reqs[0]["w"])


@pytest.mark.parametrize("bits", [8, 16])
def test_paper_normal_three_sigma_is_half_range(bits):
    """Tables I/II's random normal images: mean at mid-range, 3 sigma = half
    the range (128 for 8-bit), rounded and clamped."""
    x = inputs.paper_normal(512, 512, bits, seed=3).astype(np.float64)
    mid = float(1 << (bits - 1))
    assert abs(x.mean() - mid) < 0.01 * mid
    assert abs(x.std() - mid / 3.0) < 0.01 * mid / 3.0
    assert x.min() >= 0 and x.max() <= (1 << bits) - 1


@pytest.mark.parametrize("period,bits", [(100, 8), (25, 8), (100, 16)])
def test_paper_sine_is_diagonal_and_periodic(period, bits):
    """Diagonal sines: the value depends on x + y only and repeats every
    `period` pixels; it spans the full range."""
    x = inputs.paper_sine(300, 400, period, bits).astype(np.int64)
    assert np.array_equal(x[1:, :-1], x[:-1, 1:])            # constant along anti-diagonals
    shifted = np.abs(x[:, period:] - x[:, :-period])
    # one period along x: equal up to the rounding of exact halves (sin = 0 gives k + 0.5)
    assert shifted.max() <= 1 and (shifted == 0).mean() > 0.98
    assert x.min() == 0 and x.max() == (1 << bits) - 1


def test_video_frames_drift():
    """Frame streams: deterministic per seed, fresh pixel noise every frame,
    and a blob field that moves `drift` px right and down per frame (block
    medians of frame f+1, shifted back by the drift, match frame f's)."""
    a = list(inputs.video_frames(3, 256, 256, drift=8, seed=5))
    b = list(inputs.video_frames(3, 256, 256, drift=8, seed=5))
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert all(f.dtype == np.uint16 and f.shape == (256, 256) for f in a)
    assert not np.array_equal(a[0], a[1])

    def block_medians(img, y0, x0, n=8, s=24):
        return np.array([[np.median(img[y0 + i * s:y0 + (i + 1) * s, x0 + j * s:x0 + (j + 1) * s])
                          for j in range(n)] for i in range(n)])

    for f in range(2):
        ref = block_medians(a[f], 16, 16)
        moved = block_medians(a[f + 1], 24, 24)   # the same content, 8 px right and down
        still = block_medians(a[f + 1], 16, 16)
        assert np.abs(moved - ref).mean() < 0.5 * np.abs(still - ref).mean()
