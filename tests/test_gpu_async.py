"""GPU parity of the self ball query without host synchronisation (fgb_nq_query_async).

The pending list, once completed, must equal the oracle's list and the synchronous
query's bit for bit (segments, query and point indices in order, distances), whatever
route completion took: the queued passes alone, or the rewrite when the capacity was too
small or a cell beyond the write kernel's stage held a row longer than the asynchronous
fallback takes.  Analyses given a pending list wait for it and agree with the completed
list's results; queries without the cell-tile route return a complete list.
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


def host(nl):
    return (nl.segments.cpu().numpy(), nl.query_point_indices.cpu().numpy(), nl.point_indices.cpu().numpy(),
            nl.distances.cpu().numpy())


def assert_same(a, b):
    for u, v, what in zip(host(a), host(b), ("segments", "query indices", "point indices", "distances")):
        assert np.array_equal(u, v), what


def assert_oracle(nl, ref, r_max):
    _, off, pj, dist = ref
    seg, qi, p, d = host(nl)
    assert np.array_equal(seg, off)
    assert np.array_equal(p, pj)
    assert np.array_equal(qi, np.repeat(np.arange(len(off) - 1), np.diff(off)))
    assert np.all(np.abs(d - dist) <= 2e-6 * r_max + 1e-7)


CASES = {
    "cubic": (W.Box.cube(30.0), 22000, 2.0),
    "triclinic": (W.Box(26.0, 24.0, 28.0, 0.1, -0.05, 0.15), 15000, 1.7),
    "2d": (W.Box.square(80.0), 12000, 1.5),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_async_query_equals_oracle_and_sync(fgb, case):
    b, n, r = CASES[case]
    x = W.small_random(900 + n % 97, n, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=r)
    pending = nq.query_async(r, exclude_ii=True)
    assert pending.__dict__["_pending"]                 # queued, not completed
    sync = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    pending.wait()
    assert not pending.rewritten
    assert_same(pending, sync)
    assert pending.escalations == sync.escalations
    assert_oracle(pending, oracle.ball_query(b, x, r), r)
    # the next query reuses the size of this one as its capacity
    again = nq.query_async(r, exclude_ii=True)
    assert len(again) == len(sync) and not again.rewritten
    assert_same(again, sync)


def test_async_query_keeps_self_pairs_when_asked(fgb):
    b = W.Box.cube(24.0)
    x = W.small_random(911, 9000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.8)
    a = nq.query_async(1.8, exclude_ii=False)
    s = nq.query(None, dict(r_max=1.8, exclude_ii=False)).toNeighborList()
    assert_same(a, s)
    assert len(a) == len(nq.query(None, dict(r_max=1.8, exclude_ii=True)).toNeighborList()) + len(x)


@pytest.mark.parametrize("capacity", [1, 1000])
def test_async_query_too_small_capacity_is_rewritten(fgb, capacity):
    b = W.Box.cube(28.0)
    x = W.small_random(913, 18000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.0)
    a = nq.query_async(2.0, exclude_ii=True, capacity=capacity)
    a.wait()
    assert a.rewritten
    s = nq.query(None, dict(r_max=2.0, exclude_ii=True)).toNeighborList()
    assert_same(a, s)
    assert_oracle(a, oracle.ball_query(b, x, 2.0), 2.0)


def test_async_query_long_rows_beyond_the_stage(fgb):
    # blob cells exceed the write kernel's stage and hold rows of hundreds to about
    # 2,000 neighbors: the asynchronous fallback flags them and completion rewrites
    b = W.Box.cube(40.0)
    rng = np.random.default_rng(77)
    bg = W.uniform_points(rng, b, 10000)
    centres = rng.uniform(-15, 15, size=(4, 3))
    blobs = (np.repeat(centres, 2500, axis=0) + rng.normal(0.0, 0.45, size=(10000, 3))).astype(np.float32)
    x = np.concatenate([bg, blobs]).astype(np.float32)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.0)
    a = nq.query_async(1.0, exclude_ii=True, capacity=10 ** 8)
    a.wait()
    assert a.rewritten
    ref = oracle.ball_query(b, x, 1.0)
    assert np.diff(ref[1]).max() > 128
    assert_oracle(a, ref, 1.0)


def test_async_query_consumers_wait(fgb):
    # an analysis handed a pending list waits for it and matches the completed list's
    b = W.Box.cube(26.0)
    x = W.small_random(917, 14000, b)
    pts = dev(x)
    nq = fgb.NeighborQuery(b, pts, r_cell=1.6)
    ref_nl = nq.query(None, dict(r_max=1.6, exclude_ii=True)).toNeighborList()
    st_ref = fgb.Steinhardt(6)
    st_ref.compute(nq, neighbors=ref_nl)
    rdf_ref = fgb.RDF(40, 1.6)
    rdf_ref.compute(nq, neighbors=ref_nl)

    st = fgb.Steinhardt(6)
    st.compute(nq, neighbors=nq.query_async(1.6))
    assert torch.equal(st.particle_order, st_ref.particle_order)
    rdf = fgb.RDF(40, 1.6)
    rdf.compute(nq, neighbors=nq.query_async(1.6))
    assert np.array_equal(rdf.bin_counts, rdf_ref.bin_counts)
    cl = fgb.Cluster()
    cl.compute(nq, neighbors=nq.query_async(1.6))
    cl_ref = fgb.Cluster()
    cl_ref.compute(nq, neighbors=ref_nl)
    assert np.array_equal(cl.cluster_idx.cpu().numpy(), cl_ref.cluster_idx.cpu().numpy())


def test_async_query_dropped_before_completion(fgb):
    # lists destroyed while pending release their arrays in stream order; later queries
    # and completions are unaffected
    b = W.Box.cube(30.0)
    x = W.small_random(919, 20000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.0)
    for _ in range(8):
        nq.query_async(2.0)
    s = nq.query(None, dict(r_max=2.0, exclude_ii=True)).toNeighborList()
    lists = [nq.query_async(2.0) for _ in range(4)]
    for a in lists:
        assert_same(a, s)


def test_async_query_on_a_side_stream(fgb):
    b = W.Box.cube(30.0)
    x = W.small_random(921, 20000, b)
    pts = dev(x)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        nq = fgb.NeighborQuery(b, pts, r_cell=2.0)
        a = nq.query_async(2.0)
        a.wait()
    torch.cuda.synchronize()
    assert_oracle(a, oracle.ball_query(b, x, 2.0), 2.0)


def test_async_query_without_the_tile_route(fgb):
    # a tree NeighborQuery and a grid too small for the cell tiles answer synchronously
    b = W.Box.cube(12.0)
    x = W.small_random(923, 3000, b)
    ref = oracle.ball_query(b, x, 1.5)
    tq = fgb.AABBQuery(b, dev(x))
    a = tq.query_async(1.5)
    assert not a.__dict__.get("_pending") or a.wait() is a
    assert_oracle(a, ref, 1.5)
    small = fgb.NeighborQuery(b, dev(x), r_cell=1.5)
    assert_oracle(small.query_async(1.5), ref, 1.5)


def test_async_query_rejects_bad_arguments(fgb):
    b = W.Box.cube(20.0)
    nq = fgb.NeighborQuery(b, dev(W.small_random(925, 2000, b)), r_cell=1.5)
    with pytest.raises(fgb.FGBError):
        nq.query_async(1.5, capacity=-1)
    with pytest.raises(fgb.FGBError):
        nq.query_async(0.0)
    with pytest.raises(fgb.FGBError):
        nq.query_async(10.5)                                # beyond half the box
