"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
filters its own image (weak scaling, no collective on the data path), the
timing is the max over ranks, the whole-job value counts every rank's outputs,
and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
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


def _rank_main(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1105_3829_gb300 import inputs
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        # each rank its own image; the filter needs nothing from the other rank
        img = inputs.xray12_u16(40, 24, seed=bench.rank_seed(rank))
        out = oracle.median2d(img, 2, threads=1)
        seeds = [None] * ws
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        # per-rank step time: rank 1 is slower; both ranks must see its time
        local = [1.5 + rank, 10.0 * (ws - rank)]
        got = bench.max_over_ranks(dist, local, torch.device("cpu"))
        q.put((rank, seeds, got, int(out.sum()), int(img.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_max():
    import oracle
    oracle.build()
    ws, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_rank_main, args=(ws, port, q), nprocs=ws, join=True, start_method="spawn")
    res = sorted(q.get(timeout=60) for _ in range(ws))
    (r0, seeds0, got0, o0, i0), (r1, seeds1, got1, o1, i1) = res
    assert (r0, r1) == (0, 1)
    assert seeds0 == seeds1 and len(set(seeds0)) == ws          # distinct images per rank
    assert i0 != i1 and o0 != o1
    assert got0 == got1 == [2.5, 20.0]                            # max over ranks, everywhere


def test_job_value_counts_all_ranks():
    import bench
    one = bench.job_value(1, 4, 4096 * 4096, 10.0)
    two = bench.job_value(2, 4, 4096 * 4096, 10.0)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(4 * 4096 * 4096 / 0.010 / 1e6)


def test_reference_arm_runs_on_rank0_only():
    import oracle
    oracle.build()
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-step-seconds", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=240, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert np.isfinite(line["ms_per_step"])
