"""GPU parity of the solid-liquid order parameter: bond scores within 1e-6 (FP64 on the
device, stored as float32), solid-like bond counts, cluster indices and sizes bit for
bit against the FP64 oracle."""
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


def crystal_and_liquid(seed):
    """A perturbed FCC crystal in half of a triclinic box, a uniform liquid in the rest."""
    b = W.Box(8 * 1.5874, 8 * 1.5874, 8 * 1.5874, 0.1, 0.0, 0.05)
    rng = np.random.default_rng(seed)
    x = W.lattice_points(None, b, 8).astype(np.float64)
    s = x @ np.linalg.inv(b.matrix()).T
    keep = s[:, 2] < 0.0
    x = x[keep] + rng.normal(scale=0.06, size=(keep.sum(), 3))
    liquid = W.uniform_points(rng, b, 3000).astype(np.float64)
    ls = liquid @ np.linalg.inv(b.matrix()).T
    ncrystal = len(x)
    x = np.vstack([x, liquid[ls[:, 2] >= 0.05]])
    return b, x.astype(np.float32), ncrystal


@pytest.mark.parametrize("l,qt,st,norm", [(6, 0.7, 7, True), (4, 0.5, 4, True), (6, 0.05, 5, False)])
def test_solid_liquid_matches_oracle(fgb, l, qt, st, norm):
    b, x, ncrystal = crystal_and_liquid(7 + l)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.4)
    nl = nq.query(None, dict(r_max=1.4, exclude_ii=True)).toNeighborList()
    sl = fgb.SolidLiquid(l, qt, st, normalize_q=norm).compute(nq, nl)
    _, off, pj, _ = oracle.ball_query(b, x, 1.4)
    s, conn, idx, sizes = oracle.solid_liquid(b, x, off, pj, l, qt, st, normalize_q=norm)
    assert np.all(np.abs(sl.ql_ij.cpu().numpy() - s) <= 1e-6 * np.maximum(1.0, np.abs(s)))
    assert np.array_equal(sl.num_connections.cpu().numpy(), conn)
    assert np.array_equal(sl.cluster_idx.cpu().numpy(), idx)
    assert np.array_equal(sl.clusters.cluster_sizes.cpu().numpy(), sizes)
    if norm and l == 6:
        assert sl.largest_cluster_size > 0.7 * ncrystal  # the crystal half is one solid cluster


def test_solid_liquid_lone_points(fgb):
    b = W.Box.cube(10.0)
    x = np.array([[0.0, 0.0, 0.0], [0.3, -0.8, 0.5], [4.0, 4.0, 4.0]], np.float32)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.0)
    nl = nq.query(None, dict(r_max=1.0)).toNeighborList()
    sl = fgb.SolidLiquid(6, 0.5, 1).compute(nq, nl)
    assert np.allclose(sl.ql_ij.cpu().numpy(), 1.0, atol=1e-6)
    assert sl.num_connections.cpu().numpy().tolist() == [1, 1, 0]
    assert sl.clusters.num_clusters == 2 and sl.largest_cluster_size == 2
