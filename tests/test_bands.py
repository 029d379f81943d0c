"""Row-band split of one image across ranks (host logic, CPU): the band and
halo arithmetic, the halo exchange over gloo with world sizes 2 and 3
(including bands shorter than the radius, whose halo comes from several
ranks), and least-loaded request placement.  Each rank filters its band with
the CPU oracle; the stitched bands must equal the oracle on the whole image
bit for bit (the per-window definition of Section II makes bands
independent once their halos are present)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_band_rows_cover_the_image_with_clamped_halos():
    from paper_1105_3829_gb300.bands import band_rows
    for H, G, r in [(100, 2, 5), (101, 3, 7), (7, 4, 3), (3, 5, 1), (64, 1, 50), (0, 2, 3)]:
        bands = band_rows(H, G, r)
        assert len(bands) == G
        assert bands[0].y0 == 0 and bands[-1].y1 == H
        for a, b in zip(bands, bands[1:]):
            assert a.y1 == b.y0
        sizes = [b.y1 - b.y0 for b in bands]
        assert max(sizes) - min(sizes) <= 1
        for b in bands:
            assert b.in0 == max(0, b.y0 - r) and b.in1 == min(H, b.y1 + r)
            assert b.top_halo + b.bottom_halo + (b.y1 - b.y0) == b.in1 - b.in0
    with pytest.raises(ValueError):
        band_rows(10, 0, 1)


def test_band_with_halo_equals_whole_image_rows(oracle):
    """The arithmetic alone, without communication: filtering each band with
    its halo and keeping the band's rows reproduces the whole image."""
    from paper_1105_3829_gb300 import inputs
    from paper_1105_3829_gb300.bands import band_rows
    img = inputs.xray12_u16(53, 71, seed=5)
    for G, r in [(2, 3), (3, 9), (5, 12)]:
        whole = oracle.median2d(img, r)
        parts = []
        for b in band_rows(img.shape[0], G, r):
            out = oracle.median2d(np.ascontiguousarray(img[b.in0:b.in1]), r)
            parts.append(out[b.y0 - b.in0:b.y1 - b.in0])
        np.testing.assert_array_equal(np.concatenate(parts, axis=0), whole)
        # a band without its halo is wrong somewhere (the halo matters)
        b = band_rows(img.shape[0], G, r)[0]
        bare = oracle.median2d(np.ascontiguousarray(img[b.y0:b.y1]), r)
        assert not np.array_equal(bare, whole[b.y0:b.y1])


def _oracle_filter(band, r):
    import oracle
    out = oracle.median2d(band.numpy(), r, threads=1)
    return torch.from_numpy(out)


def _rank_main(rank, ws, port, H, W, r, q):
    sys.path.insert(0, ROOT)
    from paper_1105_3829_gb300 import inputs
    from paper_1105_3829_gb300.bands import band_rows, filter2d_bands
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        img = inputs.xray12_u16(H, W, seed=77)  # every rank builds the same image, keeps its band
        b = band_rows(H, ws, r)[rank]
        local = torch.from_numpy(np.ascontiguousarray(img[b.y0:b.y1]))
        out = filter2d_bands(local, r, _oracle_filter)
        parts = [None] * ws
        dist.all_gather_object(parts, out.numpy())
        if rank == 0:
            q.put(np.concatenate(parts, axis=0))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,H,W,r", [(2, 60, 47, 6), (3, 20, 33, 9)])
def test_gloo_bands_stitch_to_the_whole_image(oracle, ws, H, W, r):
    """World size 2 (halo inside each neighbour) and 3 with 20 rows and r = 9
    (bands of 7 rows: a halo spans two other ranks)."""
    from paper_1105_3829_gb300 import inputs
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_rank_main, args=(ws, port, H, W, r, q), nprocs=ws, join=True, start_method="spawn")
    got = q.get(timeout=120)
    np.testing.assert_array_equal(got, oracle.median2d(inputs.xray12_u16(H, W, seed=77), r))


def test_least_loaded_placement():
    from paper_1105_3829_gb300 import inputs
    from paper_1105_3829_gb300.bands import place_requests, request_cost
    reqs = inputs.request_stream(400, rate=1000.0, seed=3)
    for G in (1, 2, 4, 8):
        dev = place_requests(reqs, G)
        assert len(dev) == len(reqs) and set(dev) <= set(range(G))
        load = np.zeros(G)
        for q, d in zip(reqs, dev):
            load[d] += request_cost(q["w"], q["h"], q["r"])
        biggest = max(request_cost(q["w"], q["h"], q["r"]) for q in reqs)
        assert load.max() - load.min() <= biggest  # greedy bound: within one request of balance
    # a busy device gets the next request only once the others caught up
    assert place_requests([{"w": 10, "h": 10, "r": 3}], 3, load=[5.0, 0.0, 1.0]) == [1]
    with pytest.raises(ValueError):
        place_requests(reqs, 0)
