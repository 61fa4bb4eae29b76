"""The N > 1 path of bench.py on the CPU: two gloo ranks on 127.0.0.1.  Each
rank indexes its own map (weak scaling: independent, seeded shards and no
data-path collective); the job's time is the slowest rank's, taken by a MAX
all-reduce; the whole-job rate counts every rank's patterns; the reference arm
runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, dist, torch.device("cpu"))
        # the shard every rank draws: the map of its own seed
        truth = synth.smooth_orientation_map(4, 4, seed=rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, truth.tobytes())
        dist.barrier()
        out[rank] = (ms, bench.whole_job_rate(16, 3, world, ms), [g == truth.tobytes() for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_shards():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, rate, same = res[rank]
        assert ms == 150.0                                   # the slowest rank's time on every rank
        assert rate == 16 * 3 * world / 0.150                # all ranks' patterns over that time
        assert same == [r == rank for r in range(world)]     # each rank's shard is its own


def test_single_rank_helpers_pass_through():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert np.isclose(bench.whole_job_rate(10000, 10, 1, 9321.0), 10728.5)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
