"""The multi-GPU path of the benchmark is replicas only: one independent
problem per rank, timings combined as the maximum over ranks, whole-job
value = ranks x cells x stages / slowest time.  Checked with two gloo ranks
on the CPU (rendezvous on 127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2608_00746_b300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 5.0 - rank, 7.5]
        q.put((rank, replicas.max_over_ranks(times)))
    finally:
        tdist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [11.0, 5.0, 7.5]


def test_single_rank_is_identity_and_weak_value():
    assert replicas.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    # 2 ranks x 524,288 cells x 3 stages in 10 ms = 314.5728 Mcell-stage/s
    assert replicas.weak_value(2, 524288, 3, 10.0) == pytest.approx(314.5728)
