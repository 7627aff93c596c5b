"""The multi-GPU path of bench.py (replicas: one process per GPU, no
collective on the data path) on CPU with world_size-2 gloo process groups:
the job time is the slowest rank's (all-reduce MAX), the job throughput
counts every rank's positions, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 40.0][rank]
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.job_rate(512 * 10, world, ms / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate))


def test_two_rank_timing_is_max_over_ranks_and_rate_counts_all_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 40.0                       # the slower rank's time
        assert rate == pytest.approx(2 * 512 * 10 / 0.040)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_rate(100, 1, 2.0) == 50.0


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2505_14372_b300 import synth
    # a non-zero rank returns at once, without touching the oracle or a GPU
    assert bench.run_reference(None, synth.WORKLOADS[1], rank=1) is None
