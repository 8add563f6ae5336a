"""GPU parity of the cluster module: cluster indices and sizes bit for bit against the
oracle (numbering by decreasing size, ties by smallest member); centres within 1e-4 and
gyration tensors within 1e-4 * (1 + |G_ref|) (FP32 positions, FP64 sums) for clusters
well below half the box (a box-spanning cluster has members near half a box from its
smallest member, where FP32 and FP64 may pick different images)."""
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


def check(fgb, b, x, r, mask=None, properties=True):
    nq = fgb.NeighborQuery(b, dev(x), r_cell=max(r, 0.5))
    nl = nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
    m = None if mask is None else torch.from_numpy(mask(nl.n_pairs).astype(np.uint8)).cuda()
    cl = fgb.Cluster().compute(nq, nl, bond_mask=m)
    qi = nl.query_point_indices.cpu().numpy()
    pj = nl.point_indices.cpu().numpy()
    idx, sizes = oracle.clusters(len(x), qi, pj, None if m is None else m.cpu().numpy().astype(bool))
    assert cl.num_clusters == len(sizes)
    assert np.array_equal(cl.cluster_idx.cpu().numpy(), idx)
    assert np.array_equal(cl.cluster_sizes.cpu().numpy(), sizes)
    if properties:
        c, g = cl.properties()
        c_ref, g_ref = oracle.cluster_properties(b, x, idx)
        dc = c.cpu().numpy() - c_ref
        # centres compare as points of the periodic box (one on a face may wrap either way)
        M = b.matrix()
        s = dc @ np.linalg.inv(M).T
        dc = (s - np.round(s)) @ M.T
        assert np.all(np.abs(dc) <= 1e-4), np.abs(dc).max()
        dg = np.abs(g.cpu().numpy() - g_ref)
        assert np.all(dg <= 1e-4 * (1 + np.abs(g_ref))), dg.max()
    return cl


@pytest.mark.parametrize("bi", [0, 1, 2])
def test_clusters_match_oracle(fgb, bi):
    boxes = [W.Box.cube(12.0), W.Box(11.0, 9.5, 10.5, 0.1, 0.05, 0.0), W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15)]
    b = boxes[bi]
    x = W.small_random(200 + bi, 6000, b)
    for r in (0.4, 0.5):  # many small clusters
        check(fgb, b, x, r)
    for r in (0.62, 0.75):  # near and above percolation: one spanning cluster
        check(fgb, b, x, r, properties=False)
    rng = np.random.default_rng(bi)
    check(fgb, b, x, 0.62, mask=lambda m: rng.random(m) < 0.4)


def test_clusters_across_the_boundary_and_degenerate(fgb):
    b = W.Box.cube(10.0)
    rng = np.random.default_rng(11)
    blobs = [rng.normal(size=(40, 3)) * 0.3 + c for c in ([4.9, 0.0, 0.0], [0.0, -4.9, 4.9], [1.0, 1.0, 1.0])]
    x = np.vstack(blobs + [rng.uniform(-5, 5, size=(20, 3))]).astype(np.float32)
    x = ((x + 5.0) % 10.0 - 5.0).astype(np.float32)
    cl = check(fgb, b, x, 0.5)
    assert cl.cluster_sizes.cpu().numpy()[0] >= 30
    one = np.zeros((1, 3), np.float32)
    assert check(fgb, b, one, 0.5).num_clusters == 1
