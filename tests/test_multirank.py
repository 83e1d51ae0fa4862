"""The N>1 bench path (independent replicas, one process per GPU) aggregates whole-job
numbers: max of the ranks' device times, sum of their boxes.  Checked with two gloo ranks
on CPU (no GPU involved)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as td
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    t, b = bench.reduce_over_ranks(1.5 + rank, 1000 * (rank + 1), device="cpu")
    q.put((rank, t, b))
    td.barrier()
    td.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, b in out:
        assert t == 2.5 and b == 3000.0


def test_oracle_all_cores_baseline_counts_boxes():
    """The all-cores oracle baseline runs independent spawned processes over the top-level
    sub-boxes and counts what they processed."""
    import bench
    from paper_1802_00330_gb300 import synth
    s = synth.config_n2()
    boxes, secs, cores = bench.oracle_all_cores(s, 2000, cores=2)
    assert cores == 2 and secs > 0 and 0 < boxes <= 2 * 2000
