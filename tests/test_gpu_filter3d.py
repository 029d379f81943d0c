"""GPU parity of the 3D (cubic window) filters against the CPU oracle."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rand(shape, dt, seed, hi=None):
    rng = np.random.default_rng(seed)
    top = (256 if dt == np.uint8 else 65536) if hi is None else hi
    return rng.integers(0, top, size=shape).astype(dt)


def run3d(hrm, vol, r, adaptive=False, rank=None):
    out = hrm.filter3d(_dev(vol), r, adaptive=adaptive, rank=rank)
    hrm.device_status()
    return _host(out)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("r", [1, 2, 3, 5])
def test_random_volumes(hrm, oracle, dt, r):
    vol = _rand((19, 23, 70), dt, 300 + r)
    np.testing.assert_array_equal(run3d(hrm, vol, r), oracle.median3d(vol, r))


@pytest.mark.parametrize("r", [8, 10])
def test_sixteen_bit_counters(hrm, oracle, r):
    # n*n > 255: slab counters switch to 16 bits
    vol = _rand((9, 13, 40), np.uint16, 77 + r, hi=4096)
    np.testing.assert_array_equal(run3d(hrm, vol, r), oracle.median3d(vol, r))


@pytest.mark.parametrize("r", [1, 3, 7])
def test_xray_volume_distribution(hrm, oracle, r):
    from paper_1105_3829_gb300 import inputs
    vol = inputs.xray12_volume(24, 30, 150, seed=5 + r)
    exp = oracle.median3d(vol, r)
    np.testing.assert_array_equal(run3d(hrm, vol, r), exp)
    np.testing.assert_array_equal(run3d(hrm, vol, r, adaptive=True), exp)


def test_depth_one_equals_2d(hrm, oracle):
    img = _rand((33, 90), np.uint16, 9, hi=4096)
    for r in (1, 4):
        np.testing.assert_array_equal(run3d(hrm, img[None], r)[0], oracle.median2d(img, r))


def test_rank_3d(hrm, oracle):
    vol = _rand((10, 12, 50), np.uint16, 21, hi=3000)
    for rank in (0, 26, 13, 5):
        np.testing.assert_array_equal(run3d(hrm, vol, 1, rank=rank), oracle.median3d(vol, 1, rank=rank))


def test_tiny_and_thin(hrm, oracle):
    for shape in [(1, 1, 1), (3, 1, 5), (1, 7, 1), (6, 2, 3)]:
        vol = _rand(shape, np.uint8, sum(shape))
        for r in (1, 3):
            np.testing.assert_array_equal(run3d(hrm, vol, r), oracle.median3d(vol, r))


def test_full_size_volume_sampled(hrm, oracle):
    """256^3 uint16 volume at r = 3, checked on seeded sample points."""
    from paper_1105_3829_gb300 import inputs
    vol = inputs.xray12_volume()
    out = run3d(hrm, vol, 3)
    rng = np.random.default_rng(3)
    zs, ys, xs = (np.concatenate([rng.integers(0, 256, 200), [0, 255]]) for _ in range(3))
    np.testing.assert_array_equal(out[zs, ys, xs], oracle.points(vol, 3, ys, xs, zs=zs))


def test_edge_slabs_along_z(hrm, oracle):
    """A volume deep enough that the slices within r of both z ends are cut
    into short edge strips ahead of the interior ones."""
    vol = _rand((64, 11, 30), np.uint16, 5, hi=4096)
    np.testing.assert_array_equal(run3d(hrm, vol, 8), oracle.median3d(vol, 8))
