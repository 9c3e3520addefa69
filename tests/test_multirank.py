"""World-size-2 gloo test of the multi-rank bench path (replicas only: barrier + max of times)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" (r + 1) * 100 ms for 5 solves: the job time is the slowest rank's
    m = bench.reduce_max((rank + 1) * 100.0)
    v = bench.aggregate(5, (rank + 1) * 100.0)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 200.0
        assert v == pytest.approx(2 * 5 / 0.2)


def test_single_process_reduction_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.aggregate(4, 2000.0) == pytest.approx(2.0)


def test_gpus_flag_relaunches_as_replica_ranks():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    cmd = bench.relaunch_cmd(["--gpus", "2", "--steps", "3"], 2, 29511)
    assert cmd[1:4] == ["-m", "torch.distributed.run", "--nnodes=1"]
    assert "--nproc-per-node=2" in cmd and cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29511"
    assert cmd[-4:] == ["--gpus", "2", "--steps", "3"] and cmd[-5].endswith("bench.py")
