"""The N > 1 path of the benchmark on CPU: two gloo ranks, independent replicas (no collective
on the data path); only the timing is combined, as the max over ranks, and the rate is the
work of all ranks over that time (weak scaling)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its K rounds took 100 + 50 r ms and its e2e loop 1 + r s
    t = bench.max_over_ranks([100.0 + 50.0 * rank, 1.0 + rank])
    rate = bench.whole_job_rate(5.12e6 * 10, world, t[0])
    q.put((rank, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in out:
        assert t == [150.0, 2.0]  # both ranks see the slowest rank's times
        assert rate == pytest.approx(5.12e7 * 2 / 0.150)
