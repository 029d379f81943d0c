"""Seeded synthetic workloads: determinism, dtype, value ranges and shape of
the distributions (no filter arithmetic here)."""
import numpy as np

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
