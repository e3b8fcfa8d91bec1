"""The multi-GPU path is replicas only: each rank runs its own system and
the whole-job rate is (sum of units) / (slowest rank's time).  Checked here
with two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_2112_12271_gb300 import replicas
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                            rank=rank, world_size=world)
    ms = [400.0, 1000.0][rank]                   # rank 1 is the slow one
    units = [3.0e6, 5.0e6][rank]
    value, tmax = replicas.aggregate(units, ms, device="cpu")
    out.put((rank, value, tmax, replicas.replica_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_to_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, seed in res:
        assert tmax == 1000.0
        assert value == pytest.approx(8.0e6 / 1.0)
    assert [r[3] for r in res] == [0, 1]


def test_single_process_is_its_own_aggregate():
    from paper_2112_12271_gb300 import replicas
    assert replicas.aggregate(2.0e6, 500.0) == (4.0e6, 500.0)
