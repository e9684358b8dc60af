"""The multi-GPU launch path of bench.py on CPU: two gloo ranks (one process
each, 127.0.0.1 rendezvous) check that ranks fit disjoint instances, that
the slowest rank's time is what every rank reports, and that the job rate
counts every rank's solves over that time.  (Each rank fits its own
instances; there is no collective on the data path, only this reduction of
the timings.)"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 5)
        my_ms = 10.0 + 7.0 * rank                   # rank 1 is the slow one
        worst = bench.max_over_ranks(my_ms)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (seeds, worst, bench.job_rate(5, world, worst), gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    (s0, w0, r0, g0), (s1, w1, r1, g1) = res[0], res[1]
    assert not set(s0) & set(s1)                    # disjoint instances
    assert g0 == g1 == [s0, s1]
    assert w0 == w1 == 17.0                         # the slowest rank's time everywhere
    assert r0 == r1 == pytest.approx(2 * 5 / 0.017)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(10, 1, 20.0) == pytest.approx(500.0)
