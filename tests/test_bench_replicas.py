"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): a MAORY frame does not
shard, so N GPUs run N independent replicas; the job's time is the slowest rank's and its
throughput counts every rank's frames.  No GPU, no data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed (r + 1) * 100 ms of FP32 frames and 50 / (r + 1) ms of something else
        totals = bench.max_over_ranks([(rank + 1) * 100.0, 50.0 / (rank + 1)], world, "cpu")
        out[rank] = (totals, bench.replica_throughput(world, 40, totals[0]))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_frames():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        totals, value = res[r]
        assert totals == [200.0, 50.0]
        # 2 ranks x 40 frames in 0.2 s
        assert value == pytest.approx(400.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.replica_throughput(1, 10, 100.0) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host cores) runs and prints on
    rank 0 alone; every other rank returns at once without work."""
    import types
    import bench
    args = types.SimpleNamespace(gpus=2, steps=3, warmup=3)
    assert bench.run_reference(args, 2, 1) is None
