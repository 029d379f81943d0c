"""GPU parity of the 2D filters against the CPU oracle (bit-exact).

Every call goes through the C ABI (libhrm.so via the ctypes binding); the
expected values come only from oracle/.  Sizes span several warp tiles
(128-column tiles, strips of rows) with ragged right and bottom edges.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rand(shape, dt, seed, hi=None):
    rng = np.random.default_rng(seed)
    top = (256 if dt == np.uint8 else 65536) if hi is None else hi
    return rng.integers(0, top, size=shape).astype(dt)


def run2d(hrm, img, r, adaptive=False):
    out = hrm.filter2d(_dev(img), r, adaptive=adaptive)
    hrm.device_status()
    return _host(out)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("r", [1, 2, 3, 4, 7, 12])
def test_random_small(hrm, oracle, dt, r):
    img = _rand((97, 301), dt, 1000 + r)
    np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (45, 1), (3, 5), (17, 129), (130, 257), (64, 64)])
@pytest.mark.parametrize("r", [1, 2, 5, 20])
def test_shapes_and_big_radius(hrm, oracle, shape, r):
    img = _rand(shape, np.uint16, sum(shape) + r, hi=4096)
    np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))


@pytest.mark.parametrize("r", [5, 15, 50])
def test_xray_distribution(hrm, oracle, r):
    from paper_1105_3829_gb300 import inputs
    img = inputs.xray12_u16(203, 389, seed=7 + r)
    np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))


@pytest.mark.parametrize("r", [15, 50])
def test_lowkey_adaptive_equals_uniform(hrm, oracle, r):
    from paper_1105_3829_gb300 import inputs
    img = inputs.lowkey16_u16(150, 333, seed=11 + r)
    exp = oracle.median2d(img, r)
    np.testing.assert_array_equal(run2d(hrm, img, r, adaptive=False), exp)
    np.testing.assert_array_equal(run2d(hrm, img, r, adaptive=True), exp)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_value_extremes(hrm, oracle, dt):
    top = 255 if dt == np.uint8 else 65535
    rng = np.random.default_rng(3)
    img = rng.choice(np.array([0, 1, top - 1, top]), size=(70, 140)).astype(dt)
    for r in (1, 2, 3, 9):
        np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
    const = np.full((40, 40), top, dt)
    for r in (1, 4):
        np.testing.assert_array_equal(run2d(hrm, const, r), const)
    spike = np.zeros((50, 60), dt)
    spike[25, 30] = top
    for r in (1, 3):
        np.testing.assert_array_equal(run2d(hrm, spike, r), oracle.median2d(spike, r))


def test_effective_bit_depths(hrm, oracle):
    for bits in (1, 3, 8, 12, 16):
        img = _rand((61, 150), np.uint16, bits, hi=1 << bits)
        for r in (3, 10):
            np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))


def test_many_nodes_per_row(hrm, oracle):
    # a steep diagonal ramp: every output of a row sits in a different leaf
    yy, xx = np.mgrid[0:120, 0:300]
    img = ((xx * 211 + yy * 17) % 65536).astype(np.uint16)
    for r in (3, 6, 30):
        np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
    from paper_1105_3829_gb300 import inputs
    sine = inputs.paper_sine(90, 260, period=25, bits=16)
    np.testing.assert_array_equal(run2d(hrm, sine, 12), oracle.median2d(sine, 12))


def test_pitched_views(hrm, oracle):
    big = _rand((80, 300), np.uint16, 5, hi=4096)
    src = _dev(big)[:, 7:250]          # row pitch 600 B, width 243, offset start
    out_full = torch.zeros((80, 256), dtype=torch.uint16, device="cuda")
    out = out_full[:, :243]
    hrm.filter2d(src, 6, out=out)
    res = _host(out_full)
    np.testing.assert_array_equal(res[:, :243], oracle.median2d(big[:, 7:250], 6))
    assert np.all(res[:, 243:] == 0), "padding of dst must stay untouched"


@pytest.mark.parametrize("r", [1, 2, 4])
def test_rank_filters(hrm, oracle, r):
    img = _rand((77, 140), np.uint16, 40 + r, hi=5000)
    n = 2 * r + 1
    for rank in (0, n * n - 1, (n * n) // 3, (n * n - 1) // 2):
        out = _host(hrm.rank_filter2d(_dev(img), r, rank))
        np.testing.assert_array_equal(out, oracle.median2d(img, r, rank=rank))


@pytest.mark.parametrize("s", [1, 4, 6])
def test_lowprec_is_truncated_median(hrm, oracle, s):
    img = _rand((90, 200), np.uint16, 50 + s, hi=4096)
    exact = oracle.median2d(img, 7)
    out = _host(hrm.filter2d_lowprec(_dev(img), 7, s))
    np.testing.assert_array_equal(out, exact & np.uint16(~((1 << s) - 1) & 0xFFFF))


def test_radius_zero_and_errors(hrm):
    img = _rand((10, 12), np.uint8, 9)
    np.testing.assert_array_equal(run2d(hrm, img, 0), img)
    t = _dev(img)
    with pytest.raises(hrm.HRMError) as e:
        hrm.filter2d(t, 128)
    assert e.value.code == hrm.HRM_EINVAL
    with pytest.raises(hrm.HRMError):
        hrm.filter2d(t, 3, out=t)  # in-place (overlap) is rejected
    rc = hrm.hrm_filter2d(1, t.data_ptr(), 12, t.data_ptr() + 4096, 12, 12, 10, 1, 1, 0, None)
    assert rc == hrm.HRM_EINVAL  # unknown border mode
    rc = hrm.hrm_filter2d(1, t.data_ptr(), 12, t.data_ptr() + 4096, 12, 12, 10, 1, 0, 8, None)
    assert rc == hrm.HRM_EINVAL  # unknown flag bits
    assert hrm.hrm_filter2d(1, 0, 0, 0, 0, 0, 0, 3, 0, 0, None) == hrm.HRM_OK  # empty image


@pytest.mark.parametrize("r", [5, 50])
def test_full_size_xray_sampled(hrm, oracle, r):
    """4096x4096 uint16 x-ray workload in the bench's launch configuration,
    checked on a seeded sample of output points (plus all four corners)."""
    from paper_1105_3829_gb300 import inputs
    img = inputs.xray12_u16()
    out = run2d(hrm, img, r)
    rng = np.random.default_rng(r)
    ys = np.concatenate([rng.integers(0, 4096, 300), [0, 0, 4095, 4095]])
    xs = np.concatenate([rng.integers(0, 4096, 300), [0, 4095, 0, 4095]])
    np.testing.assert_array_equal(out[ys, xs], oracle.points(img, r, ys, xs))


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("r", [3, 4, 5])
def test_wide_networks_shapes_and_offsets(hrm, oracle, dt, r):
    """Radius 3..5 medians take the k x k pruned networks: warp tiles of
    52-56 columns, ragged edges, images narrower than one tile, and row starts
    that break the paired loads' alignment."""
    for shape in [(1, 1), (1, 37), (45, 1), (3, 5), (17, 129), (130, 257), (66, 113)]:
        img = _rand(shape, dt, 7 * r + sum(shape))
        np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
    big = _rand((70, 240), dt, 99 + r)
    for off in (1, 3):
        sub = big[:, off:off + 201]
        out = _host(hrm.filter2d(_dev(big)[:, off:off + 201], r))
        np.testing.assert_array_equal(out, oracle.median2d(sub, r))


@pytest.mark.parametrize("r", [3, 4, 5])
def test_histogram_path_at_small_radius(hrm, oracle, r):
    """The histogram kernel still serves radius 3..5 when a plan asks for it."""
    img = _rand((111, 263), np.uint16, 300 + r, hi=4096)
    plan = hrm.hrm_plan(128, 0, 0, 2)
    hrm.set_plan(2, 2, 263, 111, 1, r, plan)
    try:
        np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
        assert hrm.get_plan(2, 2, 263, 111, 1, r).path == 2
    finally:
        hrm.set_plan(2, 2, 263, 111, 1, r, hrm.hrm_plan(0, 0, 0, 1))


@pytest.mark.parametrize("r,H", [(8, 120), (21, 200), (40, 420)])
def test_edge_strips(hrm, oracle, r, H):
    """Images tall enough that the rows within r of the top and bottom edges
    are cut into short edge strips ahead of the interior strips."""
    from paper_1105_3829_gb300 import inputs
    img = inputs.xray12_u16(H, 300, seed=60 + r)
    np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
    for sh in (24, 40):  # other interior strip lengths (edge strips of 8 rows)
        hrm.set_plan(2, 2, 300, H, 1, r, hrm.hrm_plan(128, sh, 0, 2))
        try:
            np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
        finally:
            hrm.set_plan(2, 2, 300, H, 1, r, hrm.hrm_plan(0, 0, 0, 0))


@pytest.mark.parametrize("r", [6, 9, 14])
def test_node_spans_widen_across_gaps(hrm, oracle, r):
    """Alternating 40-px bands of two value populations whose phase drifts
    down the image: a node first built for outputs at one side of a tile is
    later wanted by outputs far away, so its column span widens across a gap."""
    rng = np.random.default_rng(70 + r)
    yy, xx = np.mgrid[0:160, 0:300]
    band = ((xx + 3 * yy) // 40) % 2
    img = np.where(band, rng.integers(1800, 2600, size=xx.shape), rng.integers(300, 900, size=xx.shape))
    img = img.astype(np.uint16)
    np.testing.assert_array_equal(run2d(hrm, img, r), oracle.median2d(img, r))
    rank = (2 * r + 1) ** 2 // 3
    out = _host(hrm.rank_filter2d(_dev(img), r, rank))
    np.testing.assert_array_equal(out, oracle.median2d(img, r, rank=rank))


def test_autotune_plans_keep_parity(hrm, oracle):
    """hrm_autotune times candidate plans on the image and caches the fastest;
    whatever it picks, the output stays the exact median."""
    from paper_1105_3829_gb300 import inputs
    img = inputs.lowkey16_u16(180, 420, seed=31)
    src = _dev(img)
    for r, adaptive in ((3, False), (9, False), (9, True), (24, False)):
        plan = hrm.autotune(src, r, adaptive=adaptive)
        assert plan.path in (1, 2)
        assert plan.tile_width in ((0, 128, 256) if plan.path == 1 else (128, 256))  # networks have no tiles
        assert plan.tree in ((0,) if plan.path == 1 else (1, 2))
        got = hrm.get_plan(2, 2, 420, 180, 1, r, adaptive=adaptive)
        assert (got.tile_width, got.strip_height, got.slot_kbytes, got.path, got.tree) == \
            (plan.tile_width, plan.strip_height, plan.slot_kbytes, plan.path, plan.tree)
        out = _host(hrm.filter2d(src, r, adaptive=adaptive))
        np.testing.assert_array_equal(out, oracle.median2d(img, r))
    vol = inputs.xray12_volume(20, 24, 70, seed=3)
    vsrc = _dev(vol)
    hrm.autotune(vsrc, 3)
    out = _host(hrm.filter3d(vsrc, 3))
    np.testing.assert_array_equal(out, oracle.median3d(vol, 3))


def test_very_large_image_sampled(hrm, oracle):
    """A 12288 x 16384 uint16 image (384 MiB in, 384 MiB out): index
    arithmetic beyond 2^31 bytes of addressed data, sampled against the oracle."""
    rng = np.random.default_rng(77)
    H, W = 12288, 16384
    img = rng.integers(0, 4096, size=(H, W), dtype=np.uint16)
    src = _dev(img)
    for r in (2, 7, 40):
        out = hrm.filter2d(src, r)
        hrm.device_status()
        ys = np.concatenate([rng.integers(0, H, 200), [0, H - 1, 0, H - 1]])
        xs = np.concatenate([rng.integers(0, W, 200), [0, 0, W - 1, W - 1]])
        got = out.view(torch.int16)[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()]
        got = got.cpu().numpy().view(np.uint16)  # (CUDA indexing has no uint16 kernel)
        np.testing.assert_array_equal(got, oracle.points(img, r, ys, xs))
        del out


def test_node_cache_feedback(hrm, oracle):
    """A noisy 16-bit image with a compact mode (a few dozen distinct nodes
    per tile row) moves its class to the large node cache: the first call
    reports many node installs, the second (the large-cache trial) far fewer.
    An x-ray image keeps the default plan.  Every call is exact."""
    from paper_1105_3829_gb300 import inputs
    cases = [("lowkey", inputs.lowkey16_u16(301, 517, seed=61), True),
             ("xray", inputs.xray12_u16(299, 515, seed=62), False)]
    for name, img, deep in cases:
        h, w = img.shape
        src = torch.from_numpy(img).cuda()
        before = hrm.get_plan(hrm.HRM_U16, 2, w, h, 1, 15)
        want = oracle.median2d(img, 15)
        for call in range(3):
            got = hrm.filter2d(src, 15)
            hrm.device_status()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), want, err_msg="%s call %d" % (name, call))
        after = hrm.get_plan(hrm.HRM_U16, 2, w, h, 1, 15)
        for call in range(2):  # settled from the third call on: later calls keep the plan
            hrm.filter2d(src, 15)
        torch.cuda.synchronize()
        later = hrm.get_plan(hrm.HRM_U16, 2, w, h, 1, 15)
        assert (later.tile_width, later.strip_height, later.slot_kbytes) == \
            (after.tile_width, after.strip_height, after.slot_kbytes), name
        assert before.slot_kbytes < 100, (name, before.slot_kbytes)
        if deep:
            # as many node slots as fit in up to 200 KB (the slot count caps it): one or two tiles per SM
            assert after.slot_kbytes >= before.slot_kbytes + 30 and after.strip_height == before.strip_height, \
                (name, before.slot_kbytes, after.slot_kbytes)
        else:
            assert after.slot_kbytes == before.slot_kbytes, (name, after.slot_kbytes)


def test_tree_plans_keep_parity(hrm, oracle):
    """A plan's top-level choice (1 = uniform, 2 = the adaptive power-of-16
    split) overrides the call's adaptive flag, in single calls and in
    batches; the output stays the exact median either way (Section III-C:
    the topology changes the speed only)."""
    from paper_1105_3829_gb300 import inputs
    img16 = inputs.lowkey16_u16(150, 333, seed=44)
    img8 = (inputs.lowkey16_u16(97, 301, seed=45) >> 4).astype(np.uint8)
    for img, code in ((img16, hrm.HRM_U16), (img8, hrm.HRM_U8)):
        H, W = img.shape
        src = _dev(img)
        for r in (7, 23):
            exp = oracle.median2d(img, r)
            for adaptive in (False, True):
                for tree in (1, 2):
                    hrm.set_plan(code, 2, W, H, 1, r, hrm.hrm_plan(0, 0, 0, 2, tree), adaptive=adaptive)
                    try:
                        assert hrm.get_plan(code, 2, W, H, 1, r, adaptive=adaptive).tree == tree
                        np.testing.assert_array_equal(_host(hrm.filter2d(src, r, adaptive=adaptive)), exp)
                        dst = torch.empty_like(src)
                        hrm.filter_batch([hrm.make_job(src, dst, r, adaptive=adaptive)])
                        hrm.device_status()
                        np.testing.assert_array_equal(_host(dst), exp)
                    finally:
                        hrm.set_plan(code, 2, W, H, 1, r, hrm.hrm_plan(0, 0, 0, 0, 0), adaptive=adaptive)


@pytest.mark.parametrize("r", [6, 17, 31, 32])
def test_small_node_caches_many_rounds(hrm, oracle, r):
    """Full-range 16-bit noise: a 16-value node holds one or two window
    values, so a tile row visits far more nodes than a small node cache
    holds and levels take several rounds of node builds (slots reassigned
    between rounds of one level).  Small caches without the shared-memory row
    ring (builds read global memory) and larger ones with it; the median,
    extreme and interior ranks, and the truncated median all match the
    oracle."""
    rng = np.random.default_rng(900 + r)
    H, W = 70 + r, 260
    img = rng.integers(0, 65536, size=(H, W)).astype(np.uint16)
    src = _dev(img)
    n = 2 * r + 1
    exp = oracle.median2d(img, r)
    for kb in (32, 96):
        hrm.set_plan(hrm.HRM_U16, 2, W, H, 1, r, hrm.hrm_plan(128, 0, kb, 2, 1))
        try:
            np.testing.assert_array_equal(_host(hrm.filter2d(src, r)), exp)
            for rank in (0, n * n - 1, (n * n) // 5):
                np.testing.assert_array_equal(_host(hrm.rank_filter2d(src, r, rank)),
                                              oracle.median2d(img, r, rank=rank))
            np.testing.assert_array_equal(_host(hrm.filter2d_lowprec(src, r, 5)), exp & np.uint16(0xFFE0))
            hrm.device_status()
        finally:
            hrm.set_plan(hrm.HRM_U16, 2, W, H, 1, r, hrm.hrm_plan(0, 0, 0, 0, 0))
