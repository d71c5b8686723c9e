"""Replica path of the benchmark (N > 1 ranks, one per GPU, no data-path collective) on the CPU:
two gloo ranks set up the process group from the launcher's environment, meet at the barrier,
agree on the slowest rank's time and on the whole-job rate; every rank draws its own inputs."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import workloads as W
    r, w, _ = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 * (r + 1), w)
    field = W.mppi_batch_inputs(r, K=1, H=1, n=50)[1]
    q.put((r, w, t, bench.job_throughput(100.0, w, t), float(field[:, 0].sum())))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 20.0 for o in out)                  # the slowest rank's time
    assert all(o[3] == 100.0 * 2 / 20.0 for o in out)      # whole-job rate
    assert out[0][4] != out[1][4]                          # each replica its own field
