"""One frame split across ranks by contiguous ranges of query cells.

The paper's parallel wrappers split the per-particle work of a compute across worker
threads (Section "Implementation").  Here a worker is one GPU that holds every point of
the frame (positions are replicated, so no halo is exchanged) and walks a contiguous
range of the cell list's query cells, i.e. a stack of z slabs:

* counts: each rank counts the pairs whose half-stencil cell lies in its range (every
  unordered pair once, added to both points); the sum over ranks of these partial counts
  is every point's neighbor count, and its exclusive scan the row starts of the frame's
  NeighborList;
* rows: each rank writes the rows of its own query points, sorted by point index, packed
  in query order (``local_segments``); placing every rank's rows at the global row starts
  gives the single-rank NeighborList, order included;
* RDF: each rank histograms the pairs of its half stencils; the ranks' histograms sum to
  the frame's.

The only exchange is the sum of the counts and of the histogram.  The library does no
communication: ``all_reduce`` is any in-place sum over ranks (``torch.distributed``'s
NCCL or gloo ``all_reduce``); ``None`` means one rank.  Every computing step runs in
libfgb (``fgb_nq_count_cells``, ``fgb_nq_shard_segments``, ``fgb_nq_write_cells``,
``fgb_rdf_compute_cells``).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import NeighborQuery, RDF, _I64, _check, _stream, lib


def walked_cells(nq: NeighborQuery) -> tuple[int, int]:
    """The query cells [lo, hi) of the grid: all of them, or a 2D box's point layer."""
    nx, ny, nz = nq.cell_dims()
    if nq.box.is2D:
        return nx * ny, 2 * nx * ny
    return 0, nx * ny * nz


def cell_ranges(lo: int, hi: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, nearly equal ranges of [lo, hi), one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    span = hi - lo
    return [(lo + span * r // world, lo + span * (r + 1) // world) for r in range(world)]


def rank_range(nq: NeighborQuery, rank: int, world: int) -> tuple[int, int]:
    return cell_ranges(*walked_cells(nq), world)[rank]


@dataclass
class ShardedList:
    """One rank's rows of a sharded ball query."""
    cell_range: tuple[int, int]
    counts: torch.Tensor            # summed neighbor counts of every point (int32, n)
    local_segments: torch.Tensor    # row starts of this rank's rows in its arrays (int64, n + 1)
    global_segments: torch.Tensor   # row starts in the frame's NeighborList (int64, n + 1)
    query_point_indices: torch.Tensor
    point_indices: torch.Tensor
    distances: torch.Tensor

    @property
    def n_pairs(self) -> int:
        return int(self.point_indices.numel())


def shard_count(nq: NeighborQuery, r_max: float, cell_range, exclude_ii: bool = True) -> torch.Tensor:
    """This range's partial neighbor counts of every point (int32, n)."""
    n = nq.n_points
    c = torch.empty(max(n, 1), dtype=torch.int32, device=nq.points.device)
    lo, hi = cell_range
    _check(lib().fgb_nq_count_cells(nq._h, float(r_max), int(bool(exclude_ii)), int(lo), int(hi), c.data_ptr(),
                                    _stream()))
    return c[:n]


def shard_write(nq: NeighborQuery, r_max: float, cell_range, counts: torch.Tensor,
                exclude_ii: bool = True) -> ShardedList:
    """This range's rows, given the summed counts of every point."""
    n = nq.n_points
    dev = nq.points.device
    counts = counts.to(torch.int32).contiguous()
    lo, hi = cell_range
    local_seg = torch.empty(n + 1, dtype=torch.int64, device=dev)
    global_seg = torch.empty(n + 1, dtype=torch.int64, device=dev)
    m, mx = _I64(), ctypes.c_uint32()
    _check(lib().fgb_nq_shard_segments(nq._h, int(lo), int(hi), counts.data_ptr(), local_seg.data_ptr(),
                                       global_seg.data_ptr(), ctypes.byref(m), ctypes.byref(mx), _stream()))
    m = m.value
    qi = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    pj = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    d = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    if m > 0:
        _check(lib().fgb_nq_write_cells(nq._h, float(r_max), int(bool(exclude_ii)), int(lo), int(hi),
                                        local_seg.data_ptr(), counts.data_ptr(), mx.value, qi.data_ptr(),
                                        pj.data_ptr(), d.data_ptr(), _stream()))
    return ShardedList((int(lo), int(hi)), counts, local_seg, global_seg, qi[:m], pj[:m], d[:m])


def sharded_ball_query(nq: NeighborQuery, r_max: float, rank: int, world: int, all_reduce=None,
                       exclude_ii: bool = True) -> ShardedList:
    """Rank `rank`'s rows of the frame's ball query (counts summed by `all_reduce`)."""
    rng = rank_range(nq, rank, world)
    c = shard_count(nq, r_max, rng, exclude_ii)
    if all_reduce is not None:
        all_reduce(c)
    return shard_write(nq, r_max, rng, c, exclude_ii)


def shard_rdf(rdf: RDF, nq: NeighborQuery, cell_range, reset: bool = True):
    """Adds this range's pairs to the RDF accumulator."""
    lo, hi = cell_range
    _check(lib().fgb_rdf_compute_cells(rdf._h, nq._h, int(lo), int(hi), int(bool(reset)), _stream()))


def sharded_rdf(rdf: RDF, nq: NeighborQuery, rank: int, world: int, all_reduce=None, reset: bool = True):
    """The frame's RDF on every rank: this rank's pairs, then the sum over ranks."""
    shard_rdf(rdf, nq, rank_range(nq, rank, world), reset)
    if all_reduce is not None:
        all_reduce(rdf.counts_device().view(torch.int64))


def merge_rows(global_segments, pieces) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The frame's NeighborList arrays (query index, point index, distance) from every
    rank's rows: each rank's row i moves from its local start to global_segments[i].
    pieces: (local_segments, qi, pj, dist) per rank, as numpy arrays."""
    g = np.asarray(global_segments, dtype=np.int64)
    total = int(g[-1])
    qi = np.full(total, -1, np.int32)
    pj = np.full(total, -1, np.int32)
    dist = np.zeros(total, np.float32)
    for local, q, p, d in pieces:
        local = np.asarray(local, dtype=np.int64)
        cnt = np.diff(local)
        m = int(local[-1])
        if m == 0:
            continue
        # destination of every local entry: its row's global start + its place in the row
        shift = np.repeat(g[:-1] - local[:-1], cnt)
        dst = np.arange(m, dtype=np.int64) + shift
        qi[dst], pj[dst], dist[dst] = q[:m], p[:m], d[:m]
    return qi, pj, dist
