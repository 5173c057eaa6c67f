"""Multi-process path of bench.py on CPU (gloo, world size 2): the replicas'
timing is reduced to the slowest rank and turned into whole-job rates."""
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


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        # rank r took 1000 (r + 1) ms for its 4 iterations; 100 key switches and
        # 3000 limb transforms per iteration on every rank
        ms_max, sec_iter, rates = bench.replica_rates(1000.0 * (rank + 1), 4, world, {"ks": 100, "limbs": 3000})
        bench.barrier(world)
        q.put((rank, ms_max, sec_iter, rates))
    finally:
        dist.destroy_process_group()


def test_replica_rates_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, sec_iter, rates in out:
        assert ms_max == 2000.0                       # the slowest rank bounds the job
        assert sec_iter == pytest.approx(2.0 / (4 * 2))  # 8 iterations in 2 s
        assert rates["ks"] == pytest.approx(100 / 0.25)
        assert rates["limbs"] == pytest.approx(3000 / 0.25)


def test_replica_rates_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, sec_iter, rates = bench.replica_rates(500.0, 5, 1, {"ks": 10})
    assert (ms_max, sec_iter) == (500.0, 0.1)
    assert rates["ks"] == pytest.approx(100.0)
