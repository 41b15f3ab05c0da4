"""The multi-rank timing logic of bench.py on CPU: two gloo ranks, each with
its own grid; the job's throughput uses the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank], dist, device="cpu")
    out[rank] = bench.aggregate_mlups(world, 256 ** 3, 300, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_use_the_slowest_time():
    world, port = 2, _free_port()
    times = [0.30, 0.45]
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
    expected = world * 256 ** 3 * 300 / 0.45 / 1e6
    assert out[0] == pytest.approx(expected) and out[1] == pytest.approx(expected)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(0.5, None) == 0.5
    assert bench.aggregate_mlups(1, 1000, 10, 0.01) == pytest.approx(1.0)


def test_kernel_source_hash_covers_existing_files():
    """The sources bench.py hashes to key its measured traffic all exist, and
    the hash is a stable 16-digit hex string."""
    import os
    import bench
    for rel in bench.KERNEL_SOURCES:
        root = bench.ROOT if rel.startswith("include/") else os.path.join(bench.ROOT, "paper_2101_04550_gb300")
        assert os.path.isfile(os.path.join(root, rel)), rel
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0 and h == bench.kernel_source_hash()
