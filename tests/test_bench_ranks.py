"""Host logic of the multi-rank benchmark on CPU: two gloo ranks, each timing
its own replica, agree on the slowest rank's time and report the whole-job
weak-scaling throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [100.0 + 50.0 * rank, 2.0 + rank]        # this rank's ms and e2e seconds
    t_max, e2e = bench.reduce_max_over_ranks(local)
    v = bench.weak_scaling_mlups(1000, 10, world, t_max)
    q.put((rank, t_max, e2e, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    assert [o[2] for o in out] == [3.0, 3.0]
    # 2 ranks x 1000 cells x 100 steps x 10 bench steps in 0.15 s
    assert out[0][3] == pytest.approx(2 * 1000 * 100 * 10 / 0.15 / 1e6)
