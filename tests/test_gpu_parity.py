"""GPU parity: every kernel of the hot path against the FP64 oracle, through the C ABI.

Neighbor sets, their order and RDF counts must match bit for bit; stored float32
distances within 2e-6 relative (FP32 rounding of r); q_l within
1e-5 * max(q_ref, 1e-2); gradients within 1e-4 relative (L2) and 1e-4 * max|g_ref| per
component.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q_TOL = 1e-5
G_TOL = 1e-4


@pytest.fixture(scope="module")
def fgb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_06317_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def nl_host(nl):
    return (nl.segments.cpu().numpy(), nl.point_indices.cpu().numpy(), nl.distances.cpu().numpy(),
            nl.query_point_indices.cpu().numpy())


def assert_ball_equal(nl, ref, r_max):
    _, off, pj, dist = ref
    seg, p, d, qi = nl_host(nl)
    assert np.array_equal(seg, off), "segments differ"
    assert np.array_equal(p, pj), "point indices differ"
    assert np.array_equal(qi, np.repeat(np.arange(len(off) - 1), np.diff(off))), "query indices differ"
    assert np.all(np.abs(d - dist) <= 2e-6 * r_max + 1e-7), "distances differ"


BOXES = [
    W.Box.cube(12.0),
    W.Box(11.0, 9.5, 10.5, 0.1, 0.05, 0.0),
    W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15),
    W.Box(10.0, 10.0, 10.0, 0.2, -0.2, -0.2),
]


# ------------------------------------------------------------------ cell list


def test_cell_list_is_a_stable_sort(fgb):
    b = BOXES[2]
    x = W.small_random(1, 20000, b)
    x[:50] += 25.0                                   # points far outside the box
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.1)
    srt, cell, start = (t.cpu().numpy() for t in nq.cells())
    idx = srt[:, 3].view(np.int32)
    assert np.array_equal(np.sort(idx), np.arange(len(x)))
    cell = cell.view(np.uint32).astype(np.int64)
    assert np.all(np.diff(cell) >= 0)
    same = np.diff(cell) == 0
    assert np.all(np.diff(idx)[same] > 0), "not stable within a cell"
    start = start.view(np.uint32).astype(np.int64)
    assert start[0] == 0 and start[-1] == len(x)
    assert np.array_equal(np.searchsorted(cell, np.arange(len(start) - 1)), start[:-1])
    # local coordinate + cell origin reproduces the point up to a box vector
    nc = np.array(nq.cell_dims())
    cz, cy, cx = cell // (nc[0] * nc[1]), (cell // nc[0]) % nc[1], cell % nc[0]
    M = b.matrix()
    g = np.stack([cx / nc[0], cy / nc[1], cz / nc[2]], 1) - 0.5
    pos = srt[:, :3].astype(np.float64) + g @ M.T
    diff = x[idx].astype(np.float64) - pos
    s = diff @ np.linalg.inv(M).T
    assert np.allclose(s, np.round(s), atol=1e-6)


# ------------------------------------------------------------------ ball query


@pytest.mark.parametrize("bi", range(len(BOXES)))
@pytest.mark.parametrize("r_max,r_cell", [(1.3, 1.3), (2.2, 1.0), (4.4, 4.4)])
def test_ball_query_matches_oracle(fgb, bi, r_max, r_cell):
    b = BOXES[bi]
    x = W.small_random(10 + bi, 6000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=r_cell)
    nl = nq.query(None, dict(r_max=r_max, exclude_ii=True)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, x, r_max), r_max)


def test_ball_query_c1_full(fgb):
    w = W.c1()
    r = w.params["r_max"]
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=r)
    nl = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(w.box, w.points, r), r)


def test_ball_query_outside_points_and_include_self(fgb):
    b = BOXES[1]
    rng = np.random.default_rng(3)
    x = W.small_random(3, 3000, b)
    x[::7] += (rng.integers(-3, 4, size=(len(x[::7]), 3)) @ b.matrix().T).astype(np.float32)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.7)
    nl = nq.query(None, dict(r_max=1.7, exclude_ii=False)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, x, 1.7, exclude_ii=False), 1.7)


def test_ball_query_separate_query_points(fgb):
    b = BOXES[3]
    x = W.small_random(4, 5000, b)
    y = W.small_random(5, 777, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.0)
    for excl in (False, True):
        nl = nq.query(dev(y), dict(r_max=2.0, exclude_ii=excl)).toNeighborList()
        assert_ball_equal(nl, oracle.ball_query(b, x, 2.0, exclude_ii=excl, query_points=y), 2.0)


def test_ball_query_small_box_general_route(fgb):
    b = W.Box(5.0, 5.5, 6.0, 0.15, -0.1, 0.2)          # fewer than 3 cells per axis
    x = W.small_random(6, 400, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.2)
    assert min(nq.cell_dims()) < 3
    nl = nq.query(None, dict(r_max=2.2, exclude_ii=True)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, x, 2.2), 2.2)


def test_ball_query_exact_edges(fgb):
    # integer lattice: many pairs at exactly r_max = 2 and sqrt(5), decided by the strict rule
    b = W.Box.cube(16.0)
    g = np.stack(np.meshgrid(*[np.arange(-8, 8)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    for r in (2.0, float(np.sqrt(np.float64(5.0)))):
        nq = fgb.NeighborQuery(b, dev(g), r_cell=r)
        nl = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
        assert_ball_equal(nl, oracle.ball_query(b, g, r), r)
        assert nl.escalations > 0
    # a half-spaced lattice on the cell tiles with r_max one ulp above 1: every pair at
    # exactly 1 is a neighbor that only the FP64 decision finds
    h = g * np.float32(0.5)
    r = float(np.nextafter(1.0, 2.0))
    nl = fgb.NeighborQuery(b, dev(h), r_cell=r).query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    ref = oracle.ball_query(b, h, r)
    assert_ball_equal(nl, ref, r)
    assert nl.escalations > 0 and np.diff(ref[1]).max() >= 18


def test_ball_query_degenerate(fgb):
    b = W.Box.cube(10.0)
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    nq = fgb.NeighborQuery(b, empty, r_cell=1.0)
    nl = nq.query(None, dict(r_max=1.0)).toNeighborList()
    assert nl.n_pairs == 0 and nl.segments.cpu().tolist() == [0]
    one = dev(np.zeros((1, 3)))
    nl = fgb.NeighborQuery(b, one, 1.0).query(None, dict(r_max=1.0)).toNeighborList()
    assert nl.n_pairs == 0 and nl.segments.cpu().tolist() == [0, 0]
    with pytest.raises(fgb.FGBError) as e:
        fgb.NeighborQuery(b, one, 1.0).query(None, dict(r_max=5.0)).toNeighborList()
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL
    with pytest.raises(fgb.FGBError) as e:
        fgb.NeighborQuery(b, one, 1.0).query(None, dict(r_max=1.0, num_neighbors=3)).toNeighborList()
    assert e.value.code == fgb.ERR_INVALID_ARG
    with pytest.raises(fgb.FGBError):
        fgb.NeighborQuery([10.0, 0.0, 10.0], one, 1.0)


# ------------------------------------------------------------------------ kNN


def assert_knn_equal(nl, ref, k):
    n, j, r = ref
    seg, p, d, qi = nl_host(nl)
    m = int(n[0])
    assert np.all(n == m)
    assert np.array_equal(seg, np.arange(len(n) + 1) * m)
    assert np.array_equal(p.reshape(-1, m) if m else p, j[:, :m] if m else p)
    assert np.allclose(d.reshape(-1, m) if m else d, r[:, :m] if m else d, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("bi", [0, 2])
@pytest.mark.parametrize("k", [1, 4, 12, 20])
def test_knn_matches_oracle(fgb, bi, k):
    b = BOXES[bi]
    x = W.small_random(20 + bi, 5000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.0)
    nl = nq.query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b, x, k), k)


def test_knn_perfect_fcc_ties(fgb):
    b = W.Box.cube(4 * 1.5874)
    x = W.lattice_points(None, b, 4)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.2)
    nl = nq.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    assert nl.escalations > 0
    assert_knn_equal(nl, oracle.knn(b, x, 12), 12)


def test_knn_few_points(fgb):
    b = W.Box.cube(20.0)
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.5]], np.float32)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.0)
    nl = nq.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b, x, 12), 12)
    far = np.array([[0.0, 0.0, 0.0], [9.9, 9.9, 9.9]], np.float32)
    with pytest.raises(fgb.FGBError) as e:
        fgb.NeighborQuery(b, dev(far), 2.0).query(None, dict(num_neighbors=1)).toNeighborList()
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL


# ------------------------------------------------------------------------ RDF


@pytest.mark.parametrize("bi", range(len(BOXES)))
def test_rdf_matches_oracle(fgb, bi):
    b = BOXES[bi]
    x = W.small_random(30 + bi, 6000, b)
    for bins, r_max, r_min, r_cell in [(50, 4.0, 0.0, 4.0), (173, 3.3, 0.7, 1.2)]:
        rdf = fgb.RDF(bins, r_max, r_min)
        rdf.compute(fgb.NeighborQuery(b, dev(x), r_cell=r_cell), reset=True)
        assert np.array_equal(rdf.bin_counts, oracle.rdf_counts(b, x, bins, r_max, r_min))


def test_rdf_c1_accumulate_and_normalise(fgb):
    w = W.c1()
    p = w.params
    y = W.uniform_points(np.random.default_rng(99), w.box, 4096)
    rdf = fgb.RDF(p["rdf_bins"], p["rdf_r_max"])
    for i, pts in enumerate((w.points, y)):
        rdf.compute(fgb.NeighborQuery(w.box, dev(pts), r_cell=4.0), reset=(i == 0))
    want = oracle.rdf_counts(w.box, w.points, 100, 4.0) + oracle.rdf_counts(w.box, y, 100, 4.0)
    assert np.array_equal(rdf.bin_counts, want)
    g_ref, c_ref = oracle.rdf_normalize(want, 2 * 4096, 4096, w.box.volume, 100, 0.0, 4.0)
    assert np.allclose(rdf.rdf, g_ref, rtol=1e-12) and np.allclose(rdf.bin_centers, c_ref)


def test_rdf_from_neighbor_list_and_query_points(fgb):
    b = BOXES[2]
    x = W.small_random(40, 4000, b)
    y = W.small_random(41, 500, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.5)
    nl = nq.query(None, dict(r_max=2.5, exclude_ii=True)).toNeighborList()
    rdf = fgb.RDF(64, 2.5, 0.2)
    rdf.compute(nq, neighbors=nl)
    assert np.array_equal(rdf.bin_counts, oracle.rdf_counts(b, x, 64, 2.5, 0.2))
    rdf2 = fgb.RDF(64, 2.5)
    rdf2.compute(nq, query_points=dev(y))
    assert np.array_equal(rdf2.bin_counts, oracle.rdf_counts(b, x, 64, 2.5, exclude_ii=False, query_points=y))


def test_rdf_dense_cells_duplicates_and_many_bins(fgb):
    # a tight blob puts hundreds of points in a few cells (several query passes per
    # cell in the tile kernel), exact duplicates give r = 0 pairs, and 3000 bins take the
    # kernel with shared or global histograms instead of the private per-warp ones
    b = W.Box.cube(20.0)
    rng = np.random.default_rng(7)
    blob = (rng.normal(size=(900, 3)) * 0.3).astype(np.float32)
    x = np.concatenate([W.small_random(50, 2000, b), blob, blob[:50]]).astype(np.float32)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=3.0)
    for bins, r_max, r_min in [(100, 3.0, 0.0), (3000, 3.0, 0.0), (77, 2.9, 0.4)]:
        rdf = fgb.RDF(bins, r_max, r_min)
        rdf.compute(nq)
        assert np.array_equal(rdf.bin_counts, oracle.rdf_counts(b, x, bins, r_max, r_min)), bins


def test_rdf_exact_edges(fgb):
    b = W.Box.cube(16.0)
    g = np.stack(np.meshgrid(*[np.arange(-8, 8)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    g = g * np.float32(0.5)
    rdf = fgb.RDF(16, 4.0)
    rdf.compute(fgb.NeighborQuery(b, dev(g), r_cell=4.0))
    assert np.array_equal(rdf.bin_counts, oracle.rdf_counts(b, g, 16, 4.0))
    assert rdf.escalations() > 0


# ----------------------------------------------------------------- Steinhardt


def q_close(q, q_ref):
    return np.all(np.abs(q - q_ref) <= Q_TOL * np.maximum(q_ref, 1e-2))


@pytest.mark.parametrize("l", [0, 2, 4, 6, 8, 12])
def test_steinhardt_nlist_matches_oracle(fgb, l):
    w = W.c2(n_cells=10)
    _, off, pj, _ = oracle.ball_query(w.box, w.points, 1.3)
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(l)
    st.compute(nq, neighbors=nl)
    q_ref, Q_ref = oracle.steinhardt(w.box, w.points, off, pj, l, with_qlm=True)
    assert q_close(st.particle_order.cpu().numpy(), q_ref)
    # stored Q_lm (m >= 0) follows the same convention as the definition
    assert np.allclose(st.qlm().cpu().numpy(), Q_ref, atol=2e-6)


def test_steinhardt_fused_and_liquid(fgb):
    w = W.c4(n_cells=8)
    _, off, pj, _ = oracle.ball_query(w.box, w.points, 1.3)
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=1.3)
    for l in (4, 6):
        st = fgb.Steinhardt(l)
        st.compute(nq, neighbors=dict(r_max=1.3, exclude_ii=True))
        assert q_close(st.particle_order.cpu().numpy(), oracle.steinhardt(w.box, w.points, off, pj, l))
        assert np.array_equal(st.neighbor_counts().cpu().numpy(), np.diff(off))


def test_steinhardt_perfect_fcc(fgb):
    b = W.Box.cube(6 * 1.5874)
    x = W.lattice_points(None, b, 6)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.3)
    for l, want in ((4, 0.19094), (6, 0.57452)):
        st = fgb.Steinhardt(l)
        st.compute(nq, neighbors=dict(num_neighbors=12, exclude_ii=True))
        assert np.allclose(st.particle_order.cpu().numpy(), want, atol=5e-5)


# ------------------------------------------------------------------- backward


def test_q6_backward_symmetric_nlist(fgb):
    w = W.c4(n_cells=8)
    _, off, pj, _ = oracle.ball_query(w.box, w.points, 1.3)
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(6)
    st.compute(nq, neighbors=nl)
    g = st.backward(1.0).cpu().numpy().astype(np.float64)
    g_ref = oracle.q_grad(w.box, w.points, off, pj, 6)
    assert np.linalg.norm(g - g_ref) <= G_TOL * np.linalg.norm(g_ref)
    assert np.all(np.abs(g - g_ref) <= G_TOL * np.abs(g_ref).max())


def test_q6_backward_autograd_and_knn_scatter(fgb):
    w = W.c4(n_cells=6)
    pts = dev(w.points).requires_grad_(True)
    nq = fgb.NeighborQuery(w.box, pts.detach(), r_cell=1.3)
    nl = nq.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    Q = fgb.Q6Mean.apply(pts, w.box, nl, 6)
    (2.0 * Q).backward()
    seg, pj, _, _ = nl_host(nl)
    g_ref = 2.0 * oracle.q_grad(w.box, w.points, seg, pj, 6)
    g = pts.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) <= G_TOL * np.linalg.norm(g_ref)
    q_ref = oracle.steinhardt(w.box, w.points, seg, pj, 6)
    assert abs(Q.item() - q_ref.mean()) <= 1e-6


def test_points_only_query_serves_list_computes(fgb):
    # Q6Mean's handle: the box and the points, no cell list; same q6 and gradient as a
    # cell-list NeighborQuery given the same list, and no query of its own
    w = W.c4(n_cells=6)
    pts = dev(w.points)
    nq = fgb.NeighborQuery(w.box, pts, r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    a, b = fgb.Steinhardt(6), fgb.Steinhardt(6)
    a.compute(nq, neighbors=nl)
    pq = fgb.PointsQuery(w.box, pts)
    b.compute(pq, neighbors=nl)
    assert torch.equal(a.particle_order, b.particle_order)
    assert torch.equal(a.backward(1.0), b.backward(1.0))
    with pytest.raises(fgb.FGBError) as e:
        pq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    assert e.value.code == fgb.ERR_UNSUPPORTED


# ---------------------------------------------- full-size workloads, sampled outputs


@pytest.mark.slow
def test_full_c3_ball_query_sampled(fgb):
    w = W.c3()
    r = w.params["r_max"]
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=r)
    nl = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    seg = nl.segments.cpu().numpy()
    pj = nl.point_indices
    d = nl.distances
    rng = np.random.default_rng(0)
    for q0 in rng.integers(0, len(w.points) - 500, size=4):
        c, off, p_ref, d_ref = oracle.ball_query(w.box, w.points, r, queries=(int(q0), int(q0) + 500))
        a, z = seg[q0], seg[q0 + 500]
        assert np.array_equal(seg[q0:q0 + 501] - a, off)
        assert np.array_equal(pj[a:z].cpu().numpy(), p_ref)
        assert np.allclose(d[a:z].cpu().numpy(), d_ref, atol=2e-6 * r)
    assert int(seg[-1]) > 2.2e8


@pytest.mark.slow
def test_full_c3_rdf_and_knn(fgb):
    w = W.c3()
    p = w.params
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=p["r_max"])
    rdf = fgb.RDF(p["rdf_bins"], p["rdf_r_max"])
    rdf.compute(nq)
    got = rdf.bin_counts
    want = oracle.rdf_counts(w.box, w.points, p["rdf_bins"], p["rdf_r_max"])
    assert np.array_equal(got, want)
    nk = fgb.NeighborQuery(w.box, dev(w.points), r_cell=1.6)
    nl = nk.query(None, dict(num_neighbors=p["k"], exclude_ii=True)).toNeighborList()
    pj = nl.point_indices.cpu().numpy().reshape(-1, p["k"])
    for q0 in (0, 1234567, 4_000_000):
        n, j, _ = oracle.knn(w.box, w.points, p["k"], queries=(q0, q0 + 400))
        assert np.array_equal(pj[q0:q0 + 400], j)


@pytest.mark.slow
def test_full_c2_steinhardt_and_c4_gradient_sampled(fgb):
    w = W.c2()
    nq = fgb.NeighborQuery(w.box, dev(w.points), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    seg, pj = nl.segments.cpu().numpy(), nl.point_indices.cpu().numpy()
    rng = np.random.default_rng(1)
    which = rng.choice(len(w.points), 3000, replace=False)
    for l in (4, 6):
        st = fgb.Steinhardt(l)
        st.compute(nq, neighbors=nl)
        q = st.particle_order.cpu().numpy()
        assert q_close(q[which], oracle.steinhardt(w.box, w.points, seg, pj, l, which=which))
    w4 = W.c4()
    nq4 = fgb.NeighborQuery(w4.box, dev(w4.points), r_cell=1.3)
    nl4 = nq4.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(6)
    st.compute(nq4, neighbors=nl4)
    g = st.backward(1.0).cpu().numpy().astype(np.float64)
    assert np.allclose(g.sum(0), 0.0, atol=1e-9)
    seg4, pj4 = nl4.segments.cpu().numpy(), nl4.point_indices.cpu().numpy()
    x = w4.points.astype(np.float64)
    n = len(x)
    h = 1e-3
    for k in rng.choice(n, 12, replace=False):
        aff = np.unique(np.concatenate([[k], pj4[seg4[k]:seg4[k + 1]]]))
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (oracle.steinhardt(w4.box, xp, seg4, pj4, 6, which=aff).sum()
                  - oracle.steinhardt(w4.box, xm, seg4, pj4, 6, which=aff).sum()) / (2 * h * n)
            assert abs(fd - g[k, c]) <= G_TOL * np.abs(g).max() + 1e-3 * abs(fd)


# Small grids run 8 lanes per query (or one thread per query with many queries) by
# default and large ones the cell-tile kernels; the environment switches force one
# family, or one variant inside it, so that every kernel stays covered at small sizes:
#   FGB_THREAD_KERNELS=1 (+ FGB_SPLIT_KERNELS=0: the single-lane count and write),
#   FGB_TILE_KERNELS=1 (the staged-sort write; + FGB_NL_STAGE_CAP=64: most cells to the
#   listed fallback; + FGB_NL_KERNELS=0: the earlier tile count and write;
#   + FGB_NL_QN=2 FGB_NL_QI=0: two queries per pass, query index filled by its own pass).
KERNEL_SWITCH_CHECKS = r"""
import numpy as np, torch, oracle, workloads as W, paper_1906_06317_gb300 as fgb
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
def ball(b, x, r, rc):
    nl = fgb.NeighborQuery(b, dev(x), r_cell=rc).query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    _, off, pj, d = oracle.ball_query(b, x, r)
    assert np.array_equal(nl.segments.cpu().numpy(), off)
    assert np.array_equal(nl.point_indices.cpu().numpy(), pj)
    assert np.array_equal(nl.query_point_indices.cpu().numpy(), np.repeat(np.arange(len(off) - 1), np.diff(off)))
    assert np.allclose(nl.distances.cpu().numpy(), d, atol=1e-5)
def rdf(b, x, bins, r, rc):
    h = fgb.RDF(bins, r); h.compute(fgb.NeighborQuery(b, dev(x), r_cell=rc))
    assert np.array_equal(h.bin_counts, oracle.rdf_counts(b, x, bins, r))
b = W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15)
x = W.small_random(90, 5000, b)
ball(b, x, 2.0, 2.0); rdf(b, x, 60, 3.9, 2.0)
w = W.c1()                                   # 3 x 3 x 3 cells, 150 points each
ball(w.box, w.points, 4.0, 4.0); rdf(w.box, w.points, 100, 4.0, 4.0)
c = W.Box.cube(20.0)
blob = (np.random.default_rng(7).normal(size=(900, 3)) * 0.3).astype(np.float32)
xd = np.concatenate([W.small_random(50, 2000, c), blob, blob[:50]]).astype(np.float32)
ball(c, xd, 1.5, 1.5); rdf(c, xd, 100, 3.0, 3.0)
g = np.stack(np.meshgrid(*[np.arange(-8, 8)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32) * 0.5
rdf(W.Box.cube(16.0), g, 16, 4.0, 2.0)       # thousands of pairs on bin edges
ball(W.Box.cube(16.0), g, 1.0, 1.0)          # and exactly on r_max
r1 = float(np.nextafter(1.0, 2.0))
ball(W.Box.cube(16.0), g, r1, r1)            # just inside r_max: found by the FP64 decision
k = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
_, kj, _ = oracle.knn(b, x, 12)
assert np.array_equal(k.point_indices.cpu().numpy().reshape(-1, 12), kj[:, :12])
print('ok')
"""


@pytest.mark.parametrize("switch", ["FGB_THREAD_KERNELS", "FGB_THREAD_KERNELS FGB_SPLIT_KERNELS=0",
                                    "FGB_TILE_KERNELS", "FGB_TILE_KERNELS FGB_NL_STAGE_CAP=64",
                                    "FGB_TILE_KERNELS FGB_NL_KERNELS=0",
                                    "FGB_TILE_KERNELS FGB_NL_QN=2 FGB_NL_QI=0"])
def test_kernel_family_switches(switch):
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    for item in switch.split():
        k, _, v = item.partition("=")
        env[k] = v or "1"
    r = subprocess.run([sys.executable, "-c", KERNEL_SWITCH_CHECKS], env=env, cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]


def test_ball_dense_rows_global_path(fgb):
    # blobs whose rows run from a few hundred to about 2,000 neighbors: the cell tiles
    # append them to the list and a shared-memory network sorts each row; the tree
    # query's row sort takes the same network
    b = W.Box.cube(40.0)
    rng = np.random.default_rng(77)
    bg = W.uniform_points(rng, b, 10000)
    centres = rng.uniform(-15, 15, size=(4, 3))
    blobs = (np.repeat(centres, 2500, axis=0) + rng.normal(0.0, 0.45, size=(10000, 3))).astype(np.float32)
    x = np.concatenate([bg, blobs]).astype(np.float32)
    ref = oracle.ball_query(b, x, 1.0)
    assert np.diff(ref[1]).max() > 1024 and np.diff(ref[1]).max() <= 16384
    nl = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(r_max=1.0, exclude_ii=True)).toNeighborList()
    assert_ball_equal(nl, ref, 1.0)
    tl = fgb.AABBQuery(b, dev(x)).query(None, dict(r_max=1.0, exclude_ii=True)).toNeighborList()
    assert_ball_equal(tl, ref, 1.0)


@pytest.mark.parametrize("k", [6, 12])
def test_knn_dense_clusters(fgb, k):
    # blob cells hold hundreds of points: the cell-tile kNN lists their queries and a warp
    # per query keeps the best candidates in a shared buffer trimmed to k + 1
    b = W.Box.cube(40.0)
    rng = np.random.default_rng(78)
    bg = W.uniform_points(rng, b, 10000)
    centres = rng.uniform(-15, 15, size=(4, 3))
    blobs = (np.repeat(centres, 2500, axis=0) + rng.normal(0.0, 0.45, size=(10000, 3))).astype(np.float32)
    x = np.concatenate([bg, blobs]).astype(np.float32)
    nl = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b, x, k), k)
    if k == 12:
        tl = fgb.AABBQuery(b, dev(x)).query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
        assert_knn_equal(tl, oracle.knn(b, x, k), k)
