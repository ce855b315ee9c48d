"""The multi-GPU form is replicas only: each rank contracts its own copy of the workload
and the process group carries only the timing reduction. This runs that host logic with
two gloo ranks on the CPU: whole-job throughput = units of all ranks / slowest rank."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 250.0][rank]       # the second rank is the slow one
    units = [10.0, 30.0][rank]
    value, ms_max = bench.replica_throughput(ms, units, dist, device="cpu")
    q.put((rank, value, ms_max, bench.dist_env()))
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max, env in out:
        assert ms_max == 250.0
        assert abs(value - 40.0 / 0.25) < 1e-9    # (10 + 30) units / 0.25 s
        assert env == (2, rank, 0)


def test_replica_throughput_single_process():
    import bench
    value, ms = bench.replica_throughput(200.0, 5.0, None)
    assert value == 25.0 and ms == 200.0
