"""The bench's multi-rank path (independent replicas, one per GPU) on CPU:
two gloo ranks take the maximum of their timings and compute the whole-job
throughput; the reference arm does its work on rank 0 only."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + r ms for 3 steps and 2.5 - r s end to end
        total_ms, e2e_s = bench.max_over_ranks([10.0 + rank, 2.5 - rank])
        out[rank] = (total_ms, e2e_s, bench.job_gbps(world, 1 << 30, 3, total_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        total_ms, e2e_s, gbps = res[rank]
        assert total_ms == 11.0 and e2e_s == 2.5  # every rank sees the maximum
        assert gbps == pytest.approx(2 * (1 << 30) * 3 / 11e-3 / 1e9)


def test_single_process_is_unchanged():
    assert not dist.is_initialized()
    assert bench.max_over_ranks([4.0, 7.5]) == [4.0, 7.5]
    assert bench.job_gbps(1, 1 << 30, 400, 300.0) == pytest.approx((1 << 30) * 400 / 0.3 / 1e9)


def test_reference_arm_works_on_rank_zero_only():
    # other ranks return at once, without building or running the oracle
    assert bench.run_reference(None, rank=1, world=2) == 0
