"""Seeded synthetic inputs for the running-median workloads.

This module holds random-data recipes only (no filter arithmetic) and is the
one piece of code that both the CUDA path's tests/bench and the CPU oracle's
tests use.  Every generator is deterministic in its seed (numpy PCG64).

Workloads (sizes are parameters so the same distribution can be drawn at a
small parity size and at the full bench size):

* ``uniform_u8``        -- i.i.d. uniform integers 0..255 (512x512, r=3).
* ``xray12_u16``        -- 12-bit X-ray-like content in uint16: per pixel a
  two-Gaussian mixture (weight 0.6: mean 800, sd 150; weight 0.4: mean 3000,
  sd 400), rounded half-to-even, clamped to 0..4095, then 1% salt-and-pepper
  at 0 / 4095 (4096x4096; radii 1, 5, 15, 50).  Stands in for the paper's
  16-bit X-ray weld image (Table II), which is not available.
* ``lowkey16_u16``      -- full 16-bit low-key compact-mode image: 90% of
  pixels N(2000, 120), 10% uniform 0..65535, plus a smooth blob field
  (a seeded uniform grid in [-300, 300] at 64-pixel spacing, bilinearly
  upsampled), clamped to 0..65535 (8192x8192; radii 15, 50).  Stands in for
  the paper's compact-histogram image (Table I, "Venice at night").
* ``xray12_volume``     -- the x-ray mixture in a volume plus 3D-correlated
  low-frequency noise (seeded grid at 16-voxel spacing, trilinear, amplitude
  +-200), clamped to 0..4095 (256^3 or 8 x 128^3; radii 1, 3, 7).
* ``paper_normal``      -- the paper's "random uncorrelated normally
  distributed values" (mean 2^(b-1), 3 sigma = 2^(b-1)) for b = 8 or 16.
* ``paper_sine``        -- the paper's diagonal sine pattern with a given
  period in pixels.
* ``request_stream``    -- a seeded serving workload: Poisson arrivals, image
  side log-uniform in [64, 4096] per axis, half uint8-uniform / half uint16
  x-ray mixture, radius uniform 1..50.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 110538290


def seed_for(config: int, sub: int = 0) -> int:
    """Seed of sub-stream ``sub`` of workload ``config`` (1..5)."""
    return SEED_BASE + 100 * config + sub


def _rng(seed):
    return np.random.default_rng(seed)


def _round_clamp(x: np.ndarray, hi: int, dtype) -> np.ndarray:
    return np.clip(np.rint(x), 0, hi).astype(dtype)


def uniform_u8(h: int = 512, w: int = 512, seed: int | None = None) -> np.ndarray:
    rng = _rng(seed_for(1) if seed is None else seed)
    return rng.integers(0, 256, size=(h, w), dtype=np.uint8)


def _xray_mixture(rng, shape) -> np.ndarray:
    pick = rng.random(shape, dtype=np.float32) < 0.6
    a = rng.standard_normal(shape, dtype=np.float32)
    val = np.where(pick, 800.0 + 150.0 * a, 3000.0 + 400.0 * a)
    return val


def xray12_u16(h: int = 4096, w: int = 4096, seed: int | None = None) -> np.ndarray:
    rng = _rng(seed_for(2) if seed is None else seed)
    img = _round_clamp(_xray_mixture(rng, (h, w)), 4095, np.uint16)
    salt = rng.random((h, w), dtype=np.float32) < 0.01
    hi = rng.random((h, w), dtype=np.float32) < 0.5
    img[salt & hi] = 4095
    img[salt & ~hi] = 0
    return img


def _upsample_axis(grid: np.ndarray, axis: int, length: int, spacing: int) -> np.ndarray:
    pos = np.arange(length, dtype=np.float32) / spacing
    i0 = np.floor(pos).astype(np.int64)
    t = (pos - i0).astype(np.float32)
    a = np.take(grid, i0, axis=axis)
    b = np.take(grid, i0 + 1, axis=axis)
    shape = [1] * grid.ndim
    shape[axis] = length
    t = t.reshape(shape)
    return a * (1.0 - t) + b * t


def smooth_field(rng, shape, spacing: int, amp: float) -> np.ndarray:
    """Seeded uniform grid in [-amp, amp] at ``spacing`` px, multilinearly
    upsampled to ``shape`` (2D bilinear or 3D trilinear)."""
    gshape = tuple(s // spacing + 2 for s in shape)
    f = rng.uniform(-amp, amp, size=gshape).astype(np.float32)
    for ax, n in enumerate(shape):
        f = _upsample_axis(f, ax, n, spacing)
    return f


def lowkey16_u16(h: int = 8192, w: int = 8192, seed: int | None = None) -> np.ndarray:
    rng = _rng(seed_for(3) if seed is None else seed)
    base = 2000.0 + 120.0 * rng.standard_normal((h, w), dtype=np.float32)
    outl = rng.random((h, w), dtype=np.float32) < 0.10
    uni = rng.integers(0, 65536, size=(h, w)).astype(np.float32)
    val = np.where(outl, uni, base)
    val += smooth_field(rng, (h, w), 64, 300.0)
    return _round_clamp(val, 65535, np.uint16)


def xray12_volume(d: int = 256, h: int = 256, w: int = 256, seed: int | None = None) -> np.ndarray:
    rng = _rng(seed_for(4) if seed is None else seed)
    val = _xray_mixture(rng, (d, h, w))
    val += smooth_field(rng, (d, h, w), 16, 200.0)
    return _round_clamp(val, 4095, np.uint16)


def octants(vol: np.ndarray) -> list[np.ndarray]:
    """Split a (2a, 2b, 2c) volume into its 8 independent (a, b, c) octants."""
    d, h, w = (s // 2 for s in vol.shape)
    return [np.ascontiguousarray(vol[z * d:(z + 1) * d, y * h:(y + 1) * h, x * w:(x + 1) * w])
            for z in range(2) for y in range(2) for x in range(2)]


def paper_normal(h: int, w: int, bits: int = 8, seed: int = 0) -> np.ndarray:
    rng = _rng(seed)
    mid = float(1 << (bits - 1))
    val = mid + (mid / 3.0) * rng.standard_normal((h, w))
    dt = np.uint8 if bits == 8 else np.uint16
    return _round_clamp(val, (1 << bits) - 1, dt)


def paper_sine(h: int, w: int, period: float, bits: int = 8) -> np.ndarray:
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    hi = (1 << bits) - 1
    val = 0.5 * hi * (1.0 + np.sin(2.0 * np.pi * (xx + yy) / period))
    dt = np.uint8 if bits == 8 else np.uint16
    return _round_clamp(val, hi, dt)


def request_stream(n: int = 10000, rate: float = 1000.0, seed: int | None = None,
                   side_lo: int = 64, side_hi: int = 4096, r_max: int = 50) -> list[dict]:
    """Serving workload: per request its arrival time (s), width, height,
    dtype ('u8' or 'u16'), radius and a per-request image seed."""
    rng = _rng(seed_for(5) if seed is None else seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps) - gaps[0]
    lo, hi = np.log(side_lo), np.log(side_hi)
    ws = np.floor(np.exp(rng.uniform(lo, hi, size=n))).astype(int)
    hs = np.floor(np.exp(rng.uniform(lo, hi, size=n))).astype(int)
    u16 = rng.random(n) < 0.5
    rs = rng.integers(1, r_max + 1, size=n)
    seeds = rng.integers(0, 2 ** 31 - 1, size=n)
    return [dict(t=float(t[i]), w=int(ws[i]), h=int(hs[i]), dtype="u16" if u16[i] else "u8",
                 r=int(rs[i]), seed=int(seeds[i])) for i in range(n)]


def request_image(req: dict) -> np.ndarray:
    if req["dtype"] == "u8":
        return uniform_u8(req["h"], req["w"], seed=req["seed"])
    return xray12_u16(req["h"], req["w"], seed=req["seed"])


def video_frames(nframes: int = 8, h: int = 4096, w: int = 4096, drift: int = 4, seed: int | None = None):
    """A frame stream with the low-key recipe: each frame has fresh pixel noise
    (90 % N(2000,120), 10 % uniform 0..65535) over a smooth blob field (grid
    in [-300, 300] at 64 px, bilinear) that drifts by ``drift`` px right and
    down per frame.  Yields uint16 (h, w) arrays."""
    rng = _rng(seed_for(6) if seed is None else seed)
    pad = drift * nframes
    field = smooth_field(rng, (h + pad, w + pad), 64, 300.0)
    for f in range(nframes):
        base = 2000.0 + 120.0 * rng.standard_normal((h, w), dtype=np.float32)
        outl = rng.random((h, w), dtype=np.float32) < 0.10
        uni = rng.integers(0, 65536, size=(h, w)).astype(np.float32)
        o = pad - drift * f
        val = np.where(outl, uni, base) + field[o:o + h, o:o + w]
        yield _round_clamp(val, 65535, np.uint16)
