"""Row-band split of one 2D image across ranks, and request placement across
devices.

Every output pixel depends only on the n x n window around it (Section II
definition; the method is a per-window order statistic), so an image can be
cut into horizontal bands, one per rank.  A band of output rows [y0, y1)
needs input rows [y0 - r, y1 + r) clamped to the image: its own rows plus an
r-row halo from each neighbour.  Filtering the band together with its halo
(replicate border) gives exactly the whole-image result on rows [y0, y1):
inside the image the halo supplies the real neighbour rows, and at the image
edges the band's own clamping is the image's clamping.

The exchange is the only communication: each rank sends its first and last r
rows to its neighbours (point-to-point send/receive of torch.distributed:
NCCL between GPUs, gloo on the CPU) before filtering, then filters its band
on its own device.  Nothing here computes a median: ``filter_fn`` does
(``hrm.filter2d`` in the product; the tests pass the CPU oracle).

``place_requests`` assigns serving requests to devices, least-loaded first,
by an estimate of each request's work (output pixels times a per-radius
cost), so that each device's own server (continuous batching, one per GPU)
receives a balanced share.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Band:
    rank: int
    y0: int   # first output row of the band
    y1: int   # one past its last output row
    in0: int  # first input row the band needs (halo included, clamped to the image)
    in1: int  # one past the last input row it needs

    @property
    def top_halo(self) -> int:
        return self.y0 - self.in0

    @property
    def bottom_halo(self) -> int:
        return self.in1 - self.y1


def band_rows(height: int, nranks: int, radius: int) -> list[Band]:
    """Split rows 0..height-1 into nranks contiguous bands of near-equal size
    (the first height % nranks bands get one extra row); each band's input
    range adds the r-row halo on both sides, clamped to the image."""
    if nranks <= 0 or height < 0 or radius < 0:
        raise ValueError("need nranks > 0, height >= 0, radius >= 0")
    base, extra = divmod(height, nranks)
    out, y = [], 0
    for k in range(nranks):
        h = base + (1 if k < extra else 0)
        y0, y1 = y, y + h
        out.append(Band(k, y0, y1, max(0, y0 - radius), min(height, y1 + radius)))
        y = y1
    return out


def filter2d_bands(local, radius: int, filter_fn, group=None, height: int | None = None):
    """Filter this rank's rows of a row-sharded image.

    ``local`` holds this rank's output rows [y0, y1) of the input image, as
    ``band_rows`` assigns them (a (rows, width) torch tensor on this rank's
    device, CPU for gloo).  The r halo rows above and below are received from
    the neighbouring ranks (which hold them) while this rank sends its own
    first and last rows; ranks whose band is shorter than r forward only what
    they hold, so each band's halo may come from several ranks.  Returns
    filter_fn(band with halo, radius) restricted to the rows [y0, y1)."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group) if group is not None else dist.get_rank()
    nranks = dist.get_world_size(group) if group is not None else dist.get_world_size()
    sizes = torch.tensor([local.shape[0]], dtype=torch.int64)
    all_sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(nranks)]
    dist.all_gather(all_sizes, sizes, group=group)  # band heights (host-side bookkeeping only)
    heights = [int(s.item()) for s in all_sizes]
    total = sum(heights) if height is None else height
    starts = [sum(heights[:k]) for k in range(nranks)]
    y0, y1 = starts[rank], starts[rank] + heights[rank]
    in0, in1 = max(0, y0 - radius), min(total, y1 + radius)

    # which rows each rank must send where: every rank k holding rows that
    # another rank j's halo needs sends them, and j receives them
    def need(j):
        a0, a1 = max(0, starts[j] - radius), min(total, starts[j] + heights[j] + radius)
        return [(a0, starts[j]), (starts[j] + heights[j], a1)]

    ops, recv = [], []
    for j in range(nranks):
        if j == rank:
            continue
        for lo, hi in need(j):  # rows of j's halo that this rank holds
            s0, s1 = max(lo, y0), min(hi, y1)
            if s0 < s1:
                ops.append(dist.P2POp(dist.isend, local[s0 - y0:s1 - y0].contiguous(), j, group=group))
    for lo, hi in need(rank):  # this rank's halo rows, by the rank that holds them
        for k in range(nranks):
            if k == rank:
                continue
            s0, s1 = max(lo, starts[k]), min(hi, starts[k] + heights[k])
            if s0 < s1:
                buf = torch.empty((s1 - s0,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
                ops.append(dist.P2POp(dist.irecv, buf, k, group=group))
                recv.append((s0, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    pieces = sorted(recv + [(y0, local)], key=lambda p: p[0])
    band = torch.cat([p[1] for p in pieces], dim=0)
    assert band.shape[0] == in1 - in0, (band.shape, in0, in1)
    out = filter_fn(band, radius)
    return out[y0 - in0:y1 - in0]


def request_cost(width: int, height: int, radius: int) -> float:
    """Relative work of one request: output pixels times a per-radius factor
    (selection networks up to radius 5 cost about as much as the histogram
    path at radius 15; beyond that the histogram path grows slowly)."""
    px = float(width) * float(height)
    if radius <= 1:
        return px * 0.02
    if radius <= 5:
        return px * 0.4
    return px * (0.8 + radius / 60.0)


def place_requests(requests, ndevices: int, load=None) -> list[int]:
    """Least-loaded placement: each request (dicts with w, h, r) goes to the
    device whose assigned work is smallest at that moment (ties to the lower
    index).  ``load`` gives the devices' outstanding work to start from.
    Returns one device index per request, in order."""
    if ndevices <= 0:
        raise ValueError("ndevices must be > 0")
    cur = list(load) if load is not None else [0.0] * ndevices
    out = []
    for q in requests:
        d = min(range(ndevices), key=lambda k: (cur[k], k))
        cur[d] += request_cost(q["w"], q["h"], q["r"])
        out.append(d)
    return out
