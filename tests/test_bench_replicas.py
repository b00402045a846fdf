"""The multi-GPU form of the benchmark is independent replicas: each rank
decodes its own copy of the workload and the job's throughput is the sum
over ranks timed by the slowest one.  The aggregation is checked here with
two gloo ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = [1.5, 2.25][rank]
        ms_max = bench.max_over_ranks(ms)
        q.put((r, w, local, ms_max, bench.replica_value(ms_max, 1 << 30, w)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_summed_bytes():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, local, ms_max, value) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert ms_max == 2.25
        assert value == pytest.approx(2 * (1 << 30) / 2.25e-3 / 1e9)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(1.0, 10 ** 9, 1) == pytest.approx(1000.0)
