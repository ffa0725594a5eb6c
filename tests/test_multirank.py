"""The multi-rank path on CPU: two gloo ranks run the bench's host logic (disjoint per-rank disorder
samples, MAX-over-ranks timing, whole-job rate) and each simulates its own shard with the FP64 oracle;
the shards are independent problems, so no collective touches the data path."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2511_13508_gb300 import workload
    seeds = bench.rank_seeds([1, 2], rank)
    # every rank its own samples (N = 4, tiny), simulated without any exchange
    Js = [workload.couplings(4, len(oracle.enumerate_quads(4)), s) for s in seeds]
    pt = oracle.OraclePT([4, 4], Js, workload.geometric_ladder(0.5, 1.5, 2), 2, 100 + rank, swap_every=4,
                         measure_every=2, resync_every=4)
    pt.sweep(8)
    E = pt.state()[1]
    ms = 10.0 * (rank + 1)
    mx = bench.max_over_ranks(ms, dist)
    rate = bench.whole_job_rate(1000, world, mx)
    gathered = [None] * world
    dist.all_gather_object(gathered, (seeds, E.tolist(), mx, rate))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples_and_time_by_the_slowest():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [set(r[0]) for r in res]
    assert not (seeds[0] & seeds[1]) and len(seeds[0] | seeds[1]) == 4
    assert all(r[2] == 20.0 for r in res)                 # MAX over ranks
    assert all(abs(r[3] - 1000 * 2 / 0.020) < 1e-6 for r in res)
    assert not np.allclose(res[0][1], res[1][1])          # independent shards
