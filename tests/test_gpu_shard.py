"""GPU parity of the sharded single-frame path: ranks emulated one after another on one
GPU (no kernel waits on another), through the C ABI's cell-range calls.

Every range's partial counts are summed, every range writes its own rows at the summed
counts, and the rows are placed at the global row starts: the merged NeighborList must
equal the single-rank list and the oracle's (segments, query and point indices, order
included) and its distances the single-rank ones bit for bit; the ranges' RDF
histograms must sum to the single-rank histogram and the oracle's.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_06317_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def run_shards(fgb, nq, r, world, bins, rdf_r):
    from paper_1906_06317_gb300 import shard
    ranges = shard.cell_ranges(*shard.walked_cells(nq), world)
    counts = sum(shard.shard_count(nq, r, rg).to(torch.int64) for rg in ranges)
    pieces = [shard.shard_write(nq, r, rg, counts) for rg in ranges]
    g = pieces[0].global_segments.cpu().numpy()
    host = [(p.local_segments.cpu().numpy(), p.query_point_indices.cpu().numpy(), p.point_indices.cpu().numpy(),
             p.distances.cpu().numpy()) for p in pieces]
    merged = shard.merge_rows(g, host)
    total = np.zeros(bins, np.uint64)
    rdf = fgb.RDF(bins, rdf_r)
    for rg in ranges:
        shard.shard_rdf(rdf, nq, rg, reset=True)
        total += rdf.bin_counts
    return counts.cpu().numpy(), g, merged, total, [p.n_pairs for p in pieces]


@pytest.mark.parametrize("case", ["triclinic", "cubic", "2d"])
def test_sharded_frame_equals_single_rank(fgb, case):
    if case == "triclinic":
        b, n, r, rc, bins, rdf_r = W.Box(24.0, 22.0, 26.0, 0.1, -0.05, 0.15), 12000, 1.6, 1.6, 60, 3.2
    elif case == "cubic":
        b, n, r, rc, bins, rdf_r = W.Box.cube(30.0), 20000, 2.0, 2.0, 80, 4.0
    else:
        b, n, r, rc, bins, rdf_r = W.Box.square(60.0), 9000, 1.5, 1.5, 50, 3.0
    x = W.small_random(700 + len(case), n, b)
    pts = dev(x)
    nq = fgb.NeighborQuery(b, pts, r_cell=rc)
    single = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    s_seg = single.segments.cpu().numpy()
    s_pj = single.point_indices.cpu().numpy()
    s_d = single.distances.cpu().numpy()
    ref_counts, ref_off, ref_pj, _ = oracle.ball_query(b, x, r)
    assert np.array_equal(s_seg, ref_off) and np.array_equal(s_pj, ref_pj)
    rdf1 = fgb.RDF(bins, rdf_r)
    rdf1.compute(nq, reset=True)
    ref_h = oracle.rdf_counts(b, x, bins, rdf_r)
    assert np.array_equal(rdf1.bin_counts, ref_h)
    for world in (1, 2, 3, 5):
        counts, g, (qi, pj, d), hist, sizes = run_shards(fgb, nq, r, world, bins, rdf_r)
        assert np.array_equal(counts, ref_counts), world
        assert np.array_equal(g, ref_off), world
        assert np.array_equal(qi, np.repeat(np.arange(n), np.diff(ref_off))), world
        assert np.array_equal(pj, ref_pj), world
        assert np.array_equal(d, s_d), world
        assert sum(sizes) == len(ref_pj) and min(sizes) > 0, world
        assert np.array_equal(hist, ref_h), world


def test_sharded_empty_range_and_bad_ranges(fgb):
    from paper_1906_06317_gb300 import shard
    b = W.Box.cube(20.0)
    x = W.small_random(731, 4000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.5)
    lo, hi = shard.walked_cells(nq)
    c = shard.shard_count(nq, 1.5, (lo, lo))
    assert int(c.abs().sum()) == 0                        # no cell walked, no pair counted
    full = shard.shard_count(nq, 1.5, (lo, hi)).to(torch.int64)
    p = shard.shard_write(nq, 1.5, (lo, lo), full)
    assert p.n_pairs == 0
    with pytest.raises(fgb.FGBError):
        shard.shard_count(nq, 1.5, (0, hi + 1))           # beyond the grid
    with pytest.raises(fgb.FGBError):
        shard.shard_count(nq, 1.5, (5, 4))                # reversed
