"""The bench's N-GPU path on CPU: world_size-2 gloo ranks.  Sessions are independent problems
(one per rank, seeded by rank) with no data-path collective; the job's time is the slowest rank's
and its pairs the sum of the ranks'."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = [3.0, 5.0][rank]
    pairs = [100.0, 250.0][rank]
    got = bench.combine_ranks(ms, pairs, ws, "cpu")
    env = bench.dist_env()
    p0, _, _ = bench.make_workload(0)
    p1, _, _ = bench.make_workload(1)
    out[rank] = (got, env, bool((p0 != p1).any()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_by_max_and_pairs_by_sum():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    for r in range(ws):
        (ms, pairs), env, diff_p = out[r]
        assert ms == 5.0 and pairs == 350.0
        assert env == (2, r, r)
        assert diff_p  # each rank's session is its own seeded problem


def test_single_rank_is_unchanged():
    import bench
    assert bench.combine_ranks(2.5, 7.0, 1, "cpu") == (2.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the oracle's line comes from rank 0; the other ranks exit without work."""
    import argparse
    import bench

    def no_work(*a, **k):
        raise AssertionError("a rank other than 0 ran the oracle")

    monkeypatch.setattr(bench, "cpu_baseline_run", no_work)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=3, warmup=3, gpus=2)) is None


def test_all_cores_oracle_baseline_runs_its_steps_together():
    """The host-cores baseline: one oracle step per process of a spawn pool, started at a common
    barrier; the figure is all their pairs over the span from the first start to the last end."""
    import bench
    val, procs, span, pairs = bench.cpu_baseline_all_cores(2)
    assert procs == 2 and span > 0 and pairs > 0
    assert val == pytest.approx(2 * pairs / span, rel=1e-6)
