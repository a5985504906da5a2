"""The bench's multi-process path on CPU: world size 2 over gloo (127.0.0.1).  Each rank runs its
own replica; the job time is the slowest rank's, the value sums the ranks' units (weak
scaling), and the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        local_ms = [4.0, 5.5][rank]                      # the ranks finish at different times
        t = bench.max_over_ranks(dist, local_ms, "cpu")
        dist.barrier()
        out.put((rank, t, bench.whole_job_rate(1000.0, world, t * 1e-3)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.5, 5.5]              # both ranks see the slowest time
    assert all(abs(r[2] - 2 * 1000.0 / 5.5e-3) < 1e-6 for r in res)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    import argparse
    import bench
    args = argparse.Namespace(config="large", warmup=3, steps=1, gpus=2)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=1)              # other ranks exit without work
    assert buf.getvalue() == ""
