"""The N > 1 path of bench.py on the host (replicas, no data-path
collective): two gloo ranks on the CPU.  The timing reduction returns the
slowest rank's time on every rank, and the reference arm does its work on
rank 0 only (the other ranks return at once)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import time
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank reports a different time; all must see the largest
    got = bench.max_over_ranks(1.5 + rank, world, "cpu")
    t0 = time.perf_counter()

    class Args:
        workload = "small"
        steps = 1
        warmup = 0
        seed = 20241122
        mesh = (200, 200, 4)

    rc = 0
    if rank != 0:
        rc = bench.run_reference(Args, rank, world)
    took = time.perf_counter() - t0
    with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{got} {rc} {took}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for got, rc, took in vals:
        assert float(got) == 2.5
        assert int(rc) == 0
    # rank 1 returned from the reference arm without running the oracle
    assert float(vals[1][2]) < 5.0
