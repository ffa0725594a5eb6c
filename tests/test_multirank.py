"""The multi-rank path on CPU: `bench.spawn_ranks` (the launcher `bench.py --gpus N` uses when no torchrun is
around) starts two gloo ranks with RANK/WORLD_SIZE/MASTER_* set; each runs the bench's host logic (disjoint
per-rank disorder samples, MAX-over-ranks timing, whole-job rate) and simulates its own shard with the FP64
oracle.  The shards are independent problems, so no collective touches the data path."""
import multiprocessing as mp
import os

import numpy as np

import bench


def _cpu_rank(rank, world, dist, out):
    import oracle
    from paper_2511_13508_gb300 import workload
    assert os.environ["RANK"] == str(rank) and os.environ["WORLD_SIZE"] == str(world)
    assert os.environ["MASTER_ADDR"] == "127.0.0.1"
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
    return 0


def _failing_rank(rank, world, dist):
    dist.barrier()
    return 3 if rank == 1 else 0


def test_two_gloo_ranks_shard_samples_and_time_by_the_slowest():
    q = mp.get_context("spawn").Queue()
    codes = bench.spawn_ranks(2, _cpu_rank, (q,), init_group=True, backend="gloo", timeout=300)
    assert codes == [0, 0]
    res = q.get(timeout=30)
    seeds = [set(r[0]) for r in res]
    assert not (seeds[0] & seeds[1]) and len(seeds[0] | seeds[1]) == 4
    assert all(r[2] == 20.0 for r in res)                 # MAX over ranks
    assert all(abs(r[3] - 1000 * 2 / 0.020) < 1e-6 for r in res)
    assert not np.allclose(res[0][1], res[1][1])          # independent shards


def test_spawned_rank_failure_is_reported():
    assert bench.spawn_ranks(2, _failing_rank, (), init_group=True, backend="gloo", timeout=300) == [0, 3]


def test_bench_refuses_more_ranks_than_devices():
    import torch
    n = torch.cuda.device_count()
    assert bench.main(["--gpus", str(max(2, n + 1)), "--steps", "1", "--warmup", "3"]) == 2
