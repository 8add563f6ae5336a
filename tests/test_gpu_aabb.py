"""GPU parity of the tree (AABB) NeighborQuery: ball queries against the FP64 oracle and
against the cell list, bit for bit in the pair sets and their order.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOXES = [
    W.Box.cube(12.0),
    W.Box(11.0, 9.5, 10.5, 0.1, 0.05, 0.0),
    W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15),
    W.Box(10.0, 10.0, 10.0, 0.2, -0.2, -0.2),
]


@pytest.fixture(scope="module")
def fgb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_06317_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def assert_ball_equal(nl, ref, r_max):
    _, off, pj, dist = ref
    seg = nl.segments.cpu().numpy()
    assert np.array_equal(seg, off), "segments differ"
    assert np.array_equal(nl.point_indices.cpu().numpy(), pj), "point indices differ"
    qi = nl.query_point_indices.cpu().numpy()
    assert np.array_equal(qi, np.repeat(np.arange(len(off) - 1), np.diff(off))), "query indices differ"
    assert np.all(np.abs(nl.distances.cpu().numpy() - dist) <= 2e-6 * r_max + 1e-7), "distances differ"


@pytest.mark.parametrize("bi", range(len(BOXES)))
def test_tree_ball_matches_oracle(fgb, bi):
    b = BOXES[bi]
    x = W.small_random(60 + bi, 5000, b)
    aq = fgb.AABBQuery(b, dev(x))
    for r in (0.9, 2.3, 4.4):  # 4.4 is within 8 % of half the smallest width of these boxes
        for excl in (True, False):
            nl = aq.query(None, dict(r_max=r, exclude_ii=excl)).toNeighborList()
            assert_ball_equal(nl, oracle.ball_query(b, x, r, exclude_ii=excl), r)


@pytest.mark.parametrize("bi", [0, 2])
def test_tree_equals_cell_list(fgb, bi):
    b = BOXES[bi]
    x = W.small_random(70 + bi, 20000, b)
    for r in (1.0, 2.5):
        a = fgb.AABBQuery(b, dev(x)).query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
        c = fgb.NeighborQuery(b, dev(x), r_cell=r).query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
        assert torch.equal(a.segments, c.segments)
        assert torch.equal(a.point_indices, c.point_indices)
        assert torch.equal(a.query_point_indices, c.query_point_indices)
        assert torch.allclose(a.distances, c.distances, rtol=0, atol=2e-6 * r + 1e-7)


def test_tree_query_points_outside_the_box(fgb):
    # points and query points up to one box length outside (wrapped by the tree build)
    b = BOXES[3]
    rng = np.random.default_rng(5)
    x = W.small_random(80, 3000, b)
    x[:200] += (b.matrix() @ rng.integers(-1, 2, size=(200, 3)).T).T.astype(np.float32)
    y = W.small_random(81, 700, b)
    y[:100] -= (b.matrix() @ rng.integers(-1, 2, size=(100, 3)).T).T.astype(np.float32)
    aq = fgb.AABBQuery(b, dev(x))
    for excl in (False, True):
        nl = aq.query(dev(y), dict(r_max=2.2, exclude_ii=excl)).toNeighborList()
        assert_ball_equal(nl, oracle.ball_query(b, x, 2.2, exclude_ii=excl, query_points=y), 2.2)
    nl = aq.query(None, dict(r_max=2.2)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, x, 2.2), 2.2)


def test_tree_dense_cluster_duplicates_and_tiny_inputs(fgb):
    b = W.Box.cube(20.0)
    rng = np.random.default_rng(9)
    blob = (rng.normal(size=(1500, 3)) * 0.2).astype(np.float32)
    x = np.concatenate([W.small_random(90, 1000, b), blob, blob[:40]]).astype(np.float32)
    nl = fgb.AABBQuery(b, dev(x)).query(None, dict(r_max=1.2)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, x, 1.2), 1.2)
    for n in (1, 2, 3):
        xs = W.small_random(91 + n, n, b)
        nl = fgb.AABBQuery(b, dev(xs)).query(None, dict(r_max=9.0, exclude_ii=False)).toNeighborList()
        assert_ball_equal(nl, oracle.ball_query(b, xs, 9.0, exclude_ii=False), 9.0)
    empty = fgb.AABBQuery(b, dev(np.zeros((0, 3), np.float32)))
    nl = empty.query(dev(xs), dict(r_max=1.0, exclude_ii=False)).toNeighborList()
    assert nl.n_pairs == 0 and nl.segments.cpu().numpy().tolist() == [0] * (len(xs) + 1)


def test_tree_exact_edges_on_a_lattice(fgb):
    # integer lattice: thousands of pairs exactly at r_max, decided by the FP64 sequence
    b = W.Box.cube(16.0)
    g = np.stack(np.meshgrid(*[np.arange(-8, 8)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    nl = fgb.AABBQuery(b, dev(g)).query(None, dict(r_max=2.0)).toNeighborList()
    assert_ball_equal(nl, oracle.ball_query(b, g, 2.0), 2.0)
    assert nl.escalations > 0


def test_tree_feeds_rdf_and_steinhardt(fgb):
    b = BOXES[1]
    x = W.small_random(95, 4000, b)
    aq = fgb.AABBQuery(b, dev(x))
    nl = aq.query(None, dict(r_max=2.5, exclude_ii=True)).toNeighborList()
    rdf = fgb.RDF(50, 2.5)
    rdf.compute(aq, neighbors=nl)
    assert np.array_equal(rdf.bin_counts, oracle.rdf_counts(b, x, 50, 2.5))
    st = fgb.Steinhardt(6)
    st.compute(aq, neighbors=nl)
    _, off, pj, _ = oracle.ball_query(b, x, 2.5)
    q_ref = oracle.steinhardt(b, x, off, pj, 6)
    q = st.particle_order.cpu().numpy()
    assert np.all(np.abs(q - q_ref) <= 1e-5 * np.maximum(q_ref, 1e-2))


def test_tree_unsupported_and_invalid(fgb):
    b = BOXES[0]
    x = W.small_random(96, 500, b)
    aq = fgb.AABBQuery(b, dev(x))
    with pytest.raises(fgb.FGBError) as e:
        aq.query(None, dict(num_neighbors=33)).toNeighborList()
    assert e.value.code == fgb.ERR_UNSUPPORTED
    with pytest.raises(fgb.FGBError) as e:
        fgb.RDF(10, 2.0).compute(aq)
    assert e.value.code == fgb.ERR_UNSUPPORTED
    with pytest.raises(fgb.FGBError) as e:
        aq.query(None, dict(r_max=6.5)).toNeighborList()
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL
    far = x.copy()
    far[0] += 100.0
    with pytest.raises(fgb.FGBError) as e:
        fgb.AABBQuery(b, dev(far))
    assert e.value.code == fgb.ERR_INVALID_ARG
    with pytest.raises(fgb.FGBError) as e:
        aq.query(dev(far[:5]), dict(r_max=1.0, exclude_ii=False)).toNeighborList()
    assert e.value.code == fgb.ERR_INVALID_ARG


def assert_knn_equal(nl, ref):
    n, j, r = ref
    m = int(n[0])
    assert np.all(n == m)
    assert np.array_equal(nl.segments.cpu().numpy(), np.arange(len(n) + 1) * m)
    assert np.array_equal(nl.point_indices.cpu().numpy().reshape(-1, m), j[:, :m])
    assert np.allclose(nl.distances.cpu().numpy().reshape(-1, m), r[:, :m], rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("bi", [0, 2, 3])
@pytest.mark.parametrize("k", [1, 4, 12, 20, 32])
def test_tree_knn_matches_oracle_and_cell_list(fgb, bi, k):
    b = BOXES[bi]
    x = W.small_random(100 + bi, 4000, b)
    nl = fgb.AABBQuery(b, dev(x)).query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b, x, k))
    c = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
    assert torch.equal(nl.point_indices, c.point_indices)


def test_tree_knn_ties_outside_points_and_query_points(fgb):
    # perfect FCC: 12 neighbors at one distance, decided by index through the FP64 path
    b = W.Box.cube(4 * 1.5874)
    xf = W.lattice_points(None, b, 4)
    nl = fgb.AABBQuery(b, dev(xf)).query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b, xf, 12))
    b3 = BOXES[3]
    rng = np.random.default_rng(12)
    x = W.small_random(110, 3000, b3)
    x[:150] += (b3.matrix() @ rng.integers(-1, 2, size=(150, 3)).T).T.astype(np.float32)
    y = W.small_random(111, 400, b3)
    aq = fgb.AABBQuery(b3, dev(x))
    for excl in (False, True):
        nl = aq.query(dev(y), dict(num_neighbors=8, exclude_ii=excl)).toNeighborList()
        assert_knn_equal(nl, oracle.knn(b3, x, 8, exclude_ii=excl, query_points=y))
    nl = aq.query(None, dict(num_neighbors=6, exclude_ii=False)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b3, x, 6, exclude_ii=False))
    # fewer points than k: rows of n - 1 (a tight cluster, so every distance is valid)
    xs = (np.random.default_rng(13).normal(size=(5, 3)) * 0.5).astype(np.float32)
    few = fgb.AABBQuery(b3, dev(xs))
    nl = few.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    assert_knn_equal(nl, oracle.knn(b3, xs, 12))
    with pytest.raises(fgb.FGBError) as e:  # 5 points spread over the box: a 4th neighbor too far
        fgb.AABBQuery(b3, dev(W.small_random(112, 5, b3))).query(None, dict(num_neighbors=4)).toNeighborList()
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL


TREE_THREAD_CHECK = r"""
import numpy as np, torch, oracle, workloads as W, paper_1906_06317_gb300 as fgb
b = W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15)
x = W.small_random(64, 5000, b)
aq = fgb.AABBQuery(b, torch.from_numpy(x).cuda())
for r in (0.9, 2.3):
    for excl in (True, False):
        nl = aq.query(None, dict(r_max=r, exclude_ii=excl)).toNeighborList()
        _, off, pj, d = oracle.ball_query(b, x, r, exclude_ii=excl)
        assert np.array_equal(nl.segments.cpu().numpy(), off)
        assert np.array_equal(nl.point_indices.cpu().numpy(), pj)
        assert np.all(np.abs(nl.distances.cpu().numpy() - d) <= 2e-6 * r + 1e-7)
print("ok")
"""


def test_tree_thread_per_query_kernels(fgb):
    # self queries take the warp-per-group walk by default; FGB_BVH_GROUP=0 keeps them on
    # the thread-per-query kernels, which other query sets use
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root, FGB_BVH_GROUP="0")
    r = subprocess.run([sys.executable, "-c", TREE_THREAD_CHECK], env=env, cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
