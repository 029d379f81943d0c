"""Edge cases at the limits of the method's counters, against the oracle.

* 2D radius 127 (n = 255, the largest window): a column of 255 equal values
  fills one 8-bit column counter exactly, and a window holds 65,025 values,
  just below the 16-bit window-count range; random and constant images, both
  dtypes, and the minimum and maximum order statistics at that radius.
* 3D radius 19 (n = 39): window counts reach n^3 = 59,319 (16-bit column
  counters in 3D), random and constant volumes.
* Degenerate shapes at large radii: a single row (the 1D running median),
  a single column, a 1 x 1 image, images smaller than the window.
* Two-value images (only 0 and the top value) at the largest radius.
* Empty extents (width, height or depth 0) are no-ops.
"""
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


def _run2d(hrm, img, r):
    out = hrm.filter2d(torch.from_numpy(np.ascontiguousarray(img)).cuda(), r)
    hrm.device_status()
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_max_radius_2d_random(hrm, oracle, dt):
    rng = np.random.default_rng(127 + np.dtype(dt).itemsize)
    top = 256 if dt == np.uint8 else 4096
    img = rng.integers(0, top, size=(260, 300)).astype(dt)
    np.testing.assert_array_equal(_run2d(hrm, img, 127), oracle.median2d(img, 127))


def test_max_radius_2d_constant_fills_the_counters(hrm):
    for dt, v in ((np.uint8, 200), (np.uint16, 65535), (np.uint16, 0)):
        img = np.full((300, 280), v, dt)
        np.testing.assert_array_equal(_run2d(hrm, img, 127), img)


def test_max_radius_2d_min_and_max_rank(hrm, oracle):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 65536, size=(90, 270)).astype(np.uint16)
    N = 255 * 255
    src = torch.from_numpy(img).cuda()
    for rank in (0, N - 1):
        out = hrm.rank_filter2d(src, 127, rank)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.median2d(img, 127, rank=rank))


def test_max_radius_2d_two_values(hrm, oracle):
    rng = np.random.default_rng(9)
    img = np.where(rng.random((180, 330)) < 0.5, 0, 65535).astype(np.uint16)
    np.testing.assert_array_equal(_run2d(hrm, img, 127), oracle.median2d(img, 127))


@pytest.mark.parametrize("shape", [(1, 700), (700, 1), (1, 1), (3, 5), (20, 9)])
def test_degenerate_shapes_large_radius(hrm, oracle, shape):
    rng = np.random.default_rng(sum(shape))
    img = rng.integers(0, 4096, size=shape).astype(np.uint16)
    for r in (60, 127):
        np.testing.assert_array_equal(_run2d(hrm, img, r), oracle.median2d(img, r))


def test_max_radius_3d(hrm, oracle):
    rng = np.random.default_rng(19)
    vol = rng.integers(0, 4096, size=(40, 45, 50)).astype(np.uint16)
    out = hrm.filter3d(torch.from_numpy(vol).cuda(), 19)
    hrm.device_status()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.median3d(vol, 19))
    const = np.full((30, 20, 45), 777, np.uint16)
    out = hrm.filter3d(torch.from_numpy(const).cuda(), 19)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), const)


def test_empty_extents_are_noops(hrm):
    for shape in [(0, 10), (10, 0)]:
        img = torch.zeros(shape, dtype=torch.uint16, device="cuda")
        out = hrm.filter2d(img, 5)
        assert tuple(out.shape) == shape
    for shape in [(0, 4, 4), (4, 0, 4), (4, 4, 0)]:
        vol = torch.zeros(shape, dtype=torch.uint16, device="cuda")
        out = hrm.filter3d(vol, 2)
        assert tuple(out.shape) == shape
    hrm.device_status()
