"""Seeded random sweep over shapes, radii, dtypes, value distributions and
entry points, each compared bit for bit with the oracle.  The distributions
are chosen to stress the node cache: narrow and wide value ranges, bands
whose medians jump across the tile, ramps, and heavy ties."""
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


def _image(rng, shape, dt):
    top = 255 if dt == np.uint8 else 65535
    kind = rng.integers(0, 5)
    h, w = shape
    if kind == 0:
        a = rng.integers(0, top + 1, size=shape)
    elif kind == 1:  # narrow range around a random level
        c = int(rng.integers(0, top + 1))
        a = np.clip(c + rng.integers(-20, 21, size=shape), 0, top)
    elif kind == 2:  # bands of two populations with a drifting phase
        yy, xx = np.mgrid[0:h, 0:w]
        p = int(rng.integers(8, 60))
        band = ((xx + int(rng.integers(0, 5)) * yy) // p) % 2
        a = np.where(band, rng.integers(0, top // 3, size=shape), rng.integers(2 * top // 3, top + 1, size=shape))
    elif kind == 3:  # steep ramp
        yy, xx = np.mgrid[0:h, 0:w]
        a = (xx * int(rng.integers(1, 400)) + yy * int(rng.integers(0, 50))) % (top + 1)
    else:  # heavy ties
        a = rng.choice(np.array([0, 1, top // 2, top - 1, top]), size=shape)
    return np.asarray(a).astype(dt)


def test_random_sweep(hrm, oracle):
    rng = np.random.default_rng(20261204)
    for case in range(150):
        dt = np.uint8 if rng.integers(0, 2) else np.uint16
        shape = (int(rng.integers(1, 140)), int(rng.integers(1, 330)))
        r = int(rng.choice([1, 2, 3, 4, 5, 6, 8, 11, 16, 23, 31, 45, 60]))
        img = _image(rng, shape, dt)
        src = torch.from_numpy(img).cuda()
        mode = int(rng.integers(0, 4))
        if mode == 0:
            got, exp = hrm.filter2d(src, r), oracle.median2d(img, r)
        elif mode == 1:
            got, exp = hrm.filter2d(src, r, adaptive=True), oracle.median2d(img, r)
        elif mode == 2:
            k = int(rng.integers(0, (2 * r + 1) ** 2))
            got, exp = hrm.rank_filter2d(src, r, k), oracle.median2d(img, r, rank=k)
        else:
            topo = hrm.Topology()
            hrm.filter2d_video(src, r, topo)
            got, exp = hrm.filter2d_video(src, r, topo), oracle.median2d(img, r)
            torch.cuda.synchronize()
            topo.close()
        hrm.device_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), exp, err_msg="case %d: %s %s r=%d mode %d" % (
            case, shape, dt.__name__, r, mode))


def test_random_volumes(hrm, oracle):
    rng = np.random.default_rng(4051)
    for case in range(30):
        dt = np.uint8 if rng.integers(0, 2) else np.uint16
        shape = (int(rng.integers(1, 24)), int(rng.integers(1, 30)), int(rng.integers(1, 70)))
        r = int(rng.choice([1, 2, 3, 5, 8]))
        vol = np.stack([_image(rng, shape[1:], dt) for _ in range(shape[0])])
        got = hrm.filter3d(torch.from_numpy(vol).cuda(), r)
        hrm.device_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.median3d(vol, r),
                                      err_msg="case %d: %s %s r=%d" % (case, shape, dt.__name__, r))
