"""The multi-rank (torchrun, N > 1) logic of bench.py on CPU: two gloo ranks.

On GPUs every rank transforms its own batch with no data-path collective
(weak scaling); the only cross-rank steps are the barriers around the timed
region and the max over ranks of the elapsed time.  Here those run over gloo
on 127.0.0.1, and the reference arm's rule that only rank 0 works and prints
is checked on a small band limit.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    try:
        bench.rank_barrier()
        t = bench.rank_max(1.5 + rank)  # rank 1 is the slower one
        v = bench.whole_job_value(world, 16, 3, t)
        args = argparse.Namespace(L=16, steps=1, warmup=0)
        ref = bench.run_reference(args, rank, world)
        q.put((rank, t, v, None if ref is None else (ref["impl"], ref["n_gpus"], ref["value"] > 0)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, t, v, ref in res:
        assert t == 2.5                       # max over ranks, seen by every rank
        assert v == pytest.approx(2 * 2 * 16 * 3 / 2.5)
        if rank == 0:
            assert ref == ("reference", 2, True)
        else:
            assert ref is None                # only rank 0 runs the reference arm


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.0) == 3.0         # no process group: identity
    assert bench.whole_job_value(1, 16, 5, 2.0) == pytest.approx(80.0)
