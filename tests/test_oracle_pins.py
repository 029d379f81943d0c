"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check is chosen so that a plausible slip in the oracle (a dropped or
extra window row/column, a wrong clamp, an off-by-one rank, a transposed
window, a wrong dtype path) fails at least one of them:

* hand-worked windows (tests/golden/hand_worked.json, derived from the
  definition in Section II);
* closed forms and special cases: r = 0 is the identity, a constant image is
  unchanged, a one-row image gives the 1D running median, a depth-1 volume
  gives the 2D result, a binary image gives the majority vote computed from
  box sums;
* threshold decomposition: out >= t  <=>  #{v >= t in window} >= (N+1)/2,
  evaluated for every t with integral images (an independent exact
  reference);
* invariants: min <= out <= max of the window (scipy min/max filters),
  commutation with strictly increasing gray maps, transpose/flip symmetry;
* a library special case: scipy.ndimage.median_filter / rank_filter with
  mode='nearest' (replicate border);
* self-consistency of the C oracle's two selection methods, its points()
  entry and the numpy restatement.
"""
import json
import os

import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")


def _rand(shape, dtype, seed, hi=None):
    rng = np.random.default_rng(seed)
    top = (256 if dtype == np.uint8 else 65536) if hi is None else hi
    return rng.integers(0, top, size=shape).astype(dtype)


# ---- hand-worked windows -------------------------------------------------

@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_worked(oracle, case):
    dt = np.uint8 if case["dtype"] == "u8" else np.uint16
    img = np.array(case["image"], dtype=dt)
    exp = np.array(case["expected"], dtype=dt)
    for method in ("sort", "select"):
        np.testing.assert_array_equal(oracle.median2d(img, case["radius"], method=method), exp)
    np.testing.assert_array_equal(oracle.median2d_numpy(img, case["radius"]), exp)


# ---- closed forms / special cases ----------------------------------------

@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_radius_zero_is_identity(oracle, dt):
    img = _rand((17, 23), dt, 1)
    np.testing.assert_array_equal(oracle.median2d(img, 0), img)
    vol = _rand((5, 6, 7), dt, 2)
    np.testing.assert_array_equal(oracle.median3d(vol, 0), vol)


@pytest.mark.parametrize("r", [1, 4, 9])
def test_constant_image_unchanged(oracle, r):
    img = np.full((13, 9), 4095, np.uint16)
    np.testing.assert_array_equal(oracle.median2d(img, r), img)


@pytest.mark.parametrize("r", [1, 3, 6])
def test_one_row_is_1d_running_median(oracle, r):
    row = _rand((1, 40), np.uint16, 3 + r)
    n = 2 * r + 1
    exp = np.empty_like(row)
    for x in range(row.shape[1]):
        idx = np.clip(np.arange(x - r, x + r + 1), 0, row.shape[1] - 1)
        exp[0, x] = sorted(row[0, idx])[n // 2]
    np.testing.assert_array_equal(oracle.median2d(row, r), exp)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_depth_one_volume_equals_2d(oracle, r):
    img = _rand((11, 14), np.uint16, 5 + r, hi=4096)
    np.testing.assert_array_equal(oracle.median3d(img[None], r)[0], oracle.median2d(img, r))


def _box_count(mask, r):
    """Window counts of a boolean image with replicate border, via an
    integral image of the edge-padded mask."""
    p = np.pad(mask.astype(np.int64), r, mode="edge")
    s = np.zeros((p.shape[0] + 1, p.shape[1] + 1), np.int64)
    s[1:, 1:] = p.cumsum(0).cumsum(1)
    n = 2 * r + 1
    H, W = mask.shape
    return s[n:n + H, n:n + W] - s[0:H, n:n + W] - s[n:n + H, 0:W] + s[0:H, 0:W]


@pytest.mark.parametrize("r", [1, 2, 5])
def test_binary_image_is_majority_vote(oracle, r):
    img = _rand((21, 30), np.uint8, 7 + r, hi=2)
    n = 2 * r + 1
    exp = (_box_count(img == 1, r) >= (n * n + 1) // 2).astype(np.uint8)
    np.testing.assert_array_equal(oracle.median2d(img, r), exp)


@pytest.mark.parametrize("r,seed", [(1, 11), (3, 12), (7, 13)])
def test_threshold_decomposition_u8(oracle, r, seed):
    img = _rand((33, 41), np.uint8, seed)
    n = 2 * r + 1
    need = (n * n + 1) // 2
    exp = np.zeros(img.shape, np.int64)
    for t in range(1, 256):
        exp += _box_count(img >= t, r) >= need
    np.testing.assert_array_equal(oracle.median2d(img, r), exp.astype(np.uint8))


def test_threshold_decomposition_u16_sparse_levels(oracle):
    # 16-bit values drawn from a small level set: only thresholds at the
    # levels change the count, so summing level gaps reconstructs the median.
    rng = np.random.default_rng(21)
    levels = np.array([0, 3, 700, 701, 4095, 40000, 65535])
    img = levels[rng.integers(0, len(levels), size=(29, 31))].astype(np.uint16)
    r = 4
    n = 2 * r + 1
    need = (n * n + 1) // 2
    exp = np.zeros(img.shape, np.int64)
    for lo, hi in zip(levels[:-1], levels[1:]):
        exp += (hi - lo) * (_box_count(img >= hi, r) >= need)
    np.testing.assert_array_equal(oracle.median2d(img, r), exp.astype(np.uint16))


# ---- invariants -----------------------------------------------------------

@pytest.mark.parametrize("r", [1, 4])
def test_output_within_window_min_max(oracle, r):
    img = _rand((25, 19), np.uint16, 31 + r)
    out = oracle.median2d(img, r)
    n = 2 * r + 1
    lo = scipy_ndimage.minimum_filter(img, size=n, mode="nearest")
    hi = scipy_ndimage.maximum_filter(img, size=n, mode="nearest")
    assert np.all(lo <= out) and np.all(out <= hi)


def test_commutes_with_increasing_map(oracle):
    img = _rand((24, 27), np.uint8, 41)
    rng = np.random.default_rng(42)
    lut = np.sort(rng.choice(65536, size=256, replace=False)).astype(np.uint16)
    for r in (1, 3):
        np.testing.assert_array_equal(oracle.median2d(lut[img], r), lut[oracle.median2d(img, r)])


def test_transpose_and_flips(oracle):
    img = _rand((19, 26), np.uint16, 51)
    r = 3
    out = oracle.median2d(img, r)
    np.testing.assert_array_equal(oracle.median2d(np.ascontiguousarray(img.T), r), out.T)
    np.testing.assert_array_equal(oracle.median2d(np.ascontiguousarray(img[::-1]), r), out[::-1])
    np.testing.assert_array_equal(oracle.median2d(np.ascontiguousarray(img[:, ::-1]), r), out[:, ::-1])


# ---- library special case ---------------------------------------------------

@pytest.mark.parametrize("shape,r,dt,seed", [((31, 37), 1, np.uint8, 61), ((40, 23), 5, np.uint16, 62),
                                             ((9, 50), 12, np.uint16, 63), ((5, 4), 6, np.uint8, 64)])
def test_matches_scipy_median_filter(oracle, shape, r, dt, seed):
    img = _rand(shape, dt, seed)
    exp = scipy_ndimage.median_filter(img, size=2 * r + 1, mode="nearest")
    np.testing.assert_array_equal(oracle.median2d(img, r), exp)


def test_matches_scipy_median_filter_3d(oracle):
    vol = _rand((9, 11, 13), np.uint16, 71, hi=4096)
    for r in (1, 2):
        exp = scipy_ndimage.median_filter(vol, size=2 * r + 1, mode="nearest")
        np.testing.assert_array_equal(oracle.median3d(vol, r), exp)


@pytest.mark.parametrize("rank", [0, 7, 24])
def test_rank_matches_scipy_rank_filter(oracle, rank):
    img = _rand((22, 18), np.uint16, 81)
    exp = scipy_ndimage.rank_filter(img, rank, size=5, mode="nearest")
    np.testing.assert_array_equal(oracle.median2d(img, 2, rank=rank), exp)


@pytest.mark.parametrize("rank", [0, 13, 26])
def test_rank_3d_matches_scipy_rank_filter(oracle, rank):
    """Order statistics over the cubic 3x3x3 window (minimum, median, maximum)
    against the library routine, replicate border."""
    vol = _rand((7, 9, 10), np.uint8, 83, hi=256)
    exp = scipy_ndimage.rank_filter(vol, rank, size=3, mode="nearest")
    np.testing.assert_array_equal(oracle.median3d(vol, 1, rank=rank), exp)


# ---- internal consistency ---------------------------------------------------

def test_sort_select_numpy_and_points_agree(oracle):
    img = _rand((37, 29), np.uint16, 91)
    for r in (0, 2, 6):
        a = oracle.median2d(img, r, method="sort")
        b = oracle.median2d(img, r, method="select", threads=3)
        c = oracle.median2d_numpy(img, r)
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)
        rng = np.random.default_rng(r)
        ys = rng.integers(0, img.shape[0], 50)
        xs = rng.integers(0, img.shape[1], 50)
        np.testing.assert_array_equal(oracle.points(img, r, ys, xs), a[ys, xs])
    vol = _rand((6, 7, 8), np.uint8, 92)
    a = oracle.median3d(vol, 2)
    np.testing.assert_array_equal(a, oracle.median3d_numpy(vol, 2))
    zs, ys, xs = np.nonzero(np.ones(vol.shape, bool))
    np.testing.assert_array_equal(oracle.points(vol, 2, ys, xs, zs=zs), a[zs, ys, xs])


def test_strided_and_tiny_inputs(oracle):
    big = _rand((20, 30), np.uint16, 93)
    view = big[3:15, 5:22]  # non-contiguous view: oracle copies to contiguous
    np.testing.assert_array_equal(oracle.median2d(view, 2), oracle.median2d_numpy(view, 2))
    one = np.array([[77]], np.uint8)
    for r in (0, 1, 10):
        np.testing.assert_array_equal(oracle.median2d(one, r), one)


def test_rejects_bad_arguments(oracle):
    with pytest.raises(TypeError):
        oracle.median2d(np.zeros((3, 3), np.int32), 1)
    with pytest.raises(ValueError):
        oracle.median2d(np.zeros((3, 3), np.uint8), 1, rank=9)


# ---- the pins catch plausible mistakes (mistakes planted in numpy copies) --

def _mutants():
    def off_by_one_rank(img, r):
        n = 2 * r + 1
        p = np.pad(img, r, mode="edge")
        w = np.lib.stride_tricks.sliding_window_view(p, (n, n)).reshape(img.shape + (n * n,))
        return np.sort(w, -1)[..., (n * n - 1) // 2 + 1]

    def wrap_border(img, r):
        n = 2 * r + 1
        p = np.pad(img, r, mode="wrap")
        w = np.lib.stride_tricks.sliding_window_view(p, (n, n)).reshape(img.shape + (n * n,))
        return np.sort(w, -1)[..., (n * n - 1) // 2]

    def narrow_rows(img, r):  # window one row short (dropped term)
        n = 2 * r + 1
        p = np.pad(img, r, mode="edge")
        w = np.lib.stride_tricks.sliding_window_view(p, (n, n))[:, :, 1:, :]
        w = w.reshape(img.shape + (n * (n - 1),))
        return np.sort(w, -1)[..., (n * n - 1) // 2]

    def shifted_window(img, r):  # window anchored at x-r+1 instead of x-r
        n = 2 * r + 1
        p = np.pad(img, ((r, r), (r - 1, r + 1)), mode="edge")
        w = np.lib.stride_tricks.sliding_window_view(p, (n, n)).reshape(img.shape + (n * n,))
        return np.sort(w, -1)[..., (n * n - 1) // 2]

    return [off_by_one_rank, wrap_border, narrow_rows, shifted_window]


@pytest.mark.parametrize("mutant", _mutants(), ids=lambda f: f.__name__)
def test_pins_detect_planted_mistakes(mutant):
    cases = json.load(open(GOLDEN))["cases"]
    caught = False
    for c in cases:
        dt = np.uint8 if c["dtype"] == "u8" else np.uint16
        img = np.array(c["image"], dtype=dt)
        if not np.array_equal(mutant(img, c["radius"]), np.array(c["expected"], dt)):
            caught = True
    img = _rand((31, 37), np.uint8, 61)
    if not np.array_equal(mutant(img, 2), scipy_ndimage.median_filter(img, size=5, mode="nearest")):
        caught = True
    assert caught, "pins failed to catch %s" % mutant.__name__
