"""The multi-rank logic of bench.py on CPU: world size 2 over gloo (127.0.0.1).

The ranks split one frame (strong scaling): every rank holds the same frame, the step
time is the slowest rank's and the value counts the frame's units once."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.env_rank()
    t = bench.max_over_ranks(10.0 * (r + 1), dist, "cpu")
    out[rank] = (r, w, t, bench.frame_seed(r), bench.strong_value(1000, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_units():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, t, seed, value) in res.items():
        assert r == rank and w == world
        assert t == 20.0                       # max over ranks
        assert value == pytest.approx(1000 / 0.020)
    assert res[0][3] == res[1][3]              # one frame shared by the ranks


def test_single_rank_defaults():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_value(10, 1, 1000.0) == pytest.approx(10.0)
    assert bench.strong_value(10, 1000.0) == pytest.approx(10.0)
