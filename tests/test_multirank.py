"""The N > 1 path of bench.py on the CPU: world-size-2 process groups over
gloo (no GPU).  The benchmark runs independent replicas, one workload per rank
(no data-path collective); these tests cover what the ranks share: the
max-over-ranks time, the summed launch count, the whole-job throughput, and
that each rank builds a different problem of the same shape."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, launches = bench.reduce_over_ranks(100.0 + 50.0 * rank, 10 + rank, torch.device("cpu"))
        qp = bench.host_workload(bench.WORKLOADS["small-fp64"], rank)[0]
        out.put((rank, ms, launches, qp.A.shape, float(qp.A[0, 0]),
                 bench.job_throughput(3, 1, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_time_launches_and_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    res = sorted(out.get(timeout=5) for _ in range(world))
    for rank, ms, launches, shape, a00, value in res:
        assert ms == 150.0                      # the slowest rank's time
        assert launches == 21                   # launches of both ranks
        assert shape == (200, 500)
        assert value == pytest.approx(3 * 1 * world / 0.150)
    assert res[0][4] != res[1][4]               # each rank solves its own problem
