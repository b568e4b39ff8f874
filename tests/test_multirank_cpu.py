"""The multi-process (replica) path of the benchmark on CPU: two gloo ranks
draw different states from the same workload recipe, agree on the slowest
rank's time (the job value is the units of all ranks over that time), and
combine their DOS into the mean over all ranks' states."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    args = argparse.Namespace(workload="disordered", L=16, time_steps=8)
    w, theta = bench.workload_inputs(args, rank)
    ms = bench.reduce_max_time(100.0 + 50.0 * rank, world)
    mean = bench.combine_mean(np.array([[rank + 1.0, 2.0 * rank, 5.0]]), world)
    dist.barrier()
    out.put((rank, float(theta[0, :4].sum()), w.sample.n_orb, ms, mean.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, th0, n0, ms0, m0), (r1, th1, n1, ms1, m1) = res
    assert n0 == n1                      # same lattice on every rank
    assert th0 != th1                    # independent states per rank (weak scaling)
    assert ms0 == ms1 == 150.0           # both see the slowest rank's time
    assert m0 == m1 == [[1.5, 1.0, 5.0]]  # the DOS mean over both ranks' states
