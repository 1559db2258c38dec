"""The multi-GPU path of bench.py on CPU: two gloo ranks (one process each).
Circuits are independent, so each rank takes its own disjoint slice of the
workload (weak scaling, no data-path collective); the timed step is reduced
to the slowest rank, and the reported value is the units all ranks processed
over that time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        circs = bench.rank_circuits(rank, 3)
        keys = [np.asarray(c.V).tobytes() for c in circs]
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        q.put((rank, keys, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_circuits_and_take_the_slowest_time():
    import multiprocessing as mp
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            rank, keys, slowest = q.get(timeout=120)
            got[rank] = (keys, slowest)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    k0, s0 = got[0]
    k1, s1 = got[1]
    # disjoint slices whose union is the first 6 circuits of the workload
    assert not set(k0) & set(k1)
    whole = [np.asarray(c.V).tobytes() for c in bench.rank_circuits(0, 6)]
    assert k0 + k1 == whole
    # both ranks see the slowest rank's time
    assert s0 == s1 == 15.0
    # whole-job rate: all ranks' units over the slowest time
    assert bench.job_rate(2, 3, 100, s0) == pytest.approx(2 * 3 * 100 / 15e-3)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.job_rate(1, 16, 10, 2.0) == pytest.approx(16 * 10 / 2e-3)
