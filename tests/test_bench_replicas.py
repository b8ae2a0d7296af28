"""The bench's multi-rank aggregation (independent replicas per GPU) on two gloo ranks on the CPU:
the job time is the slowest rank's and the job rate sums the ranks' DoFs."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = [2.0, 5.0][rank]
    dofs = [1_000_000, 3_000_000][rank]
    q.put((rank, bench.aggregate_replicas(step_ms, dofs, "cpu")))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, dofs, rate = res[r]
        assert ms == 5.0 and dofs == 4_000_000
        assert rate == pytest.approx(4_000_000 / 5e-3 / 1e6)


def test_single_process_is_identity():
    import bench
    ms, dofs, rate = bench.aggregate_replicas(4.0, 2_000_000)
    assert (ms, dofs) == (4.0, 2_000_000.0) and rate == pytest.approx(500.0)
