"""The benchmark's N > 1 path on CPU: two gloo ranks, one process each.

ApplyFilter shards as replicas (every rank filters its own volume, no exchange on the data
path), so the only collective the benchmark makes is the max over ranks of the timed
region, from which the whole-job throughput is computed.  These tests run that reduction
over a world of two gloo ranks, check the weak-scaling throughput formula, and check that
the reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        mine = 1.0 + 2.5 * rank                  # rank 1 is the slow replica
        dist.barrier()
        got = bench.max_over_ranks(mine, "cpu", world)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr(got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    got = [float(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    assert got == [3.5, 3.5]                     # every rank sees the slowest replica's time


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(0.4375, "cpu", 1) == 0.4375


def test_replica_throughput_is_weak_scaling():
    # 2 x 512^3 output voxels per replica step in 0.5 ms
    one = bench.replica_gvoxel_s(2 * 512 ** 3, 1, 0.5)
    assert one == pytest.approx(2 * 512 ** 3 / 0.5e-3 / 1e9)
    # N replicas over the same slowest-rank step time do N times the voxels
    for n in (2, 4, 8):
        assert bench.replica_gvoxel_s(2 * 512 ** 3, n, 0.5) == pytest.approx(n * one)


def test_reference_arm_does_no_work_off_rank_zero(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    def no_oracle(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "workload_host", no_oracle)
    monkeypatch.setattr(bench, "oracle_sample_rate", no_oracle)

    class Args:
        steps, warmup = 3, 3

    assert bench.run_reference(Args()) is None
