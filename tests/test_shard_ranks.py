"""The sharded single-frame path's partition and merge logic on two CPU ranks (gloo).

One frame is split by z slabs of query cells.  Each rank builds its pieces with the
oracle: partial neighbor counts in which every unordered pair is counted once, by the
rank that owns its lower-indexed point, and added to both points; the full rows of its
own queries, packed in query order; the RDF histogram of its own queries.  The ranks sum
the counts and histograms with a gloo all-reduce, and rank 0 places every rank's rows at
the global row starts.  The result must equal the single-rank oracle NeighborList, order
included, and its RDF counts, bit for bit; the global Q6 (a sum over ranks of their own
particles' q6) must equal the single-rank mean.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from paper_1906_06317_gb300 import shard  # noqa: E402

R_MAX, BINS, RDF_R = 1.6, 40, 3.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def frame():
    box = W.Box(11.0, 10.0, 12.0, 0.1, -0.05, 0.08)
    return box, W.small_random(31, 1500, box)


def owner(box, x, world, nz=7):
    """Rank of each point: its z slab of nz cell layers, split by shard.cell_ranges."""
    M = np.array([[box.Lx, box.xy * box.Ly, box.xz * box.Lz], [0.0, box.Ly, box.yz * box.Lz], [0.0, 0.0, box.Lz]])
    s = x.astype(np.float64) @ np.linalg.inv(M).T + 0.5
    cz = np.minimum((np.mod(s[:, 2], 1.0) * nz).astype(np.int64), nz - 1)
    ranges = shard.cell_ranges(0, nz, world)
    rank = np.zeros(len(x), np.int64)
    for r, (lo, hi) in enumerate(ranges):
        rank[(cz >= lo) & (cz < hi)] = r
    return rank


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    box, x = frame()
    n = len(x)
    own = owner(box, x, world) == rank
    _, off, pj, d = oracle.ball_query(box, x, R_MAX, threads=2)
    # partial counts: each unordered pair once, by the owner of its lower-indexed point
    qi = np.repeat(np.arange(n), np.diff(off))
    first = qi < pj
    mine = first & own[qi]
    part = np.zeros(n, np.int64)
    np.add.at(part, qi[mine], 1)
    np.add.at(part, pj[mine], 1)
    counts = torch.from_numpy(part)
    dist.all_reduce(counts)                      # the one exchange of the list
    counts = counts.numpy()
    global_seg = np.concatenate([[0], np.cumsum(counts)])
    local_seg = np.concatenate([[0], np.cumsum(np.where(own, counts, 0))])
    rows = np.concatenate([np.arange(off[i], off[i + 1]) for i in np.flatnonzero(own)] or [np.zeros(0, np.int64)])
    piece = (local_seg, qi[rows].astype(np.int32), pj[rows].astype(np.int32), d[rows].astype(np.float32))
    # RDF of the rank's own queries: the owned points first, then the rest
    perm = np.concatenate([np.flatnonzero(own), np.flatnonzero(~own)])
    h = oracle.rdf_counts(box, x[perm], BINS, RDF_R, queries=(0, int(own.sum())), threads=2).astype(np.int64)
    hist = torch.from_numpy(h)
    dist.all_reduce(hist)
    # global Q6: the sum of the rank's own particles' q6, summed over ranks
    q_own = oracle.steinhardt(box, x, off, pj, 6, which=np.flatnonzero(own), threads=2)
    qsum = torch.tensor([q_own.sum()], dtype=torch.float64)
    dist.all_reduce(qsum)
    pieces = [None] * world
    dist.all_gather_object(pieces, piece)
    if rank == 0:
        out["merged"] = shard.merge_rows(global_seg, pieces)
        out["global_seg"] = global_seg
        out["counts"] = counts
        out["hist"] = hist.numpy()
        out["q6"] = float(qsum.item()) / n
        out["sizes"] = [int(p[0][-1]) for p in pieces]
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_the_single_rank_list_and_rdf():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    box, x = frame()
    counts, off, pj, d = oracle.ball_query(box, x, R_MAX, threads=2)
    qi_m, pj_m, d_m = out["merged"]
    assert np.array_equal(out["counts"], counts)
    assert np.array_equal(out["global_seg"], off)
    assert np.array_equal(qi_m, np.repeat(np.arange(len(x)), np.diff(off)))
    assert np.array_equal(pj_m, pj)
    assert np.array_equal(d_m, d.astype(np.float32))
    assert min(out["sizes"]) > 0 and sum(out["sizes"]) == len(pj)    # both ranks own rows
    assert np.array_equal(out["hist"], oracle.rdf_counts(box, x, BINS, RDF_R, threads=2).astype(np.int64))
    q = oracle.steinhardt(box, x, off, pj, 6, threads=2)
    assert out["q6"] == pytest.approx(q.mean(), rel=1e-12, abs=0)


def test_cell_ranges_partition_the_cells():
    for lo, hi, world in ((0, 10, 3), (5, 5, 2), (100, 1000, 8), (0, 7, 7)):
        rg = shard.cell_ranges(lo, hi, world)
        assert len(rg) == world and rg[0][0] == lo and rg[-1][1] == hi
        assert all(a[1] == b[0] for a, b in zip(rg, rg[1:]))
        assert all(r[1] >= r[0] for r in rg)
        sizes = [r[1] - r[0] for r in rg]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.cell_ranges(0, 5, 0)


def test_merge_rows_places_interleaved_rows():
    # three queries owned alternately by two ranks; rows land at the global starts
    g = np.array([0, 2, 3, 6])
    a = (np.array([0, 2, 2, 5]), np.array([0, 0, 2, 2, 2], np.int32), np.array([4, 7, 1, 5, 9], np.int32),
         np.arange(5, dtype=np.float32))
    b = (np.array([0, 0, 1, 1]), np.array([1], np.int32), np.array([3], np.int32), np.array([9.0], np.float32))
    qi, pj, d = shard.merge_rows(g, [a, b])
    assert qi.tolist() == [0, 0, 1, 2, 2, 2]
    assert pj.tolist() == [4, 7, 3, 1, 5, 9]
    assert d.tolist() == [0.0, 1.0, 9.0, 2.0, 3.0, 4.0]
