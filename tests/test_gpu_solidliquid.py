"""GPU parity of the solid-liquid order parameter: solid-like bond counts, cluster
indices and sizes bit for bit against the FP64 oracle; bond scores at float32 accuracy
(each bond is screened in FP32 with a proven enclosure of its score and settled in FP64
only when the enclosure reaches the threshold)."""
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


S_TOL = 5e-5  # float32 scores: normalised products of FP32 Q_lm (FP64 near the threshold)


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
    assert np.all(np.abs(sl.ql_ij.cpu().numpy() - s) <= S_TOL * np.maximum(1.0, np.abs(s)))
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


def test_solid_liquid_thresholds_on_bond_scores(fgb):
    # thresholds 1e-10 above or below bond scores of the oracle: those bonds are decided
    # by a margin far inside any FP32 error (only the FP64 pass can decide them) and far
    # outside the 1e-12 by which two FP64 evaluations may differ
    b, x, _ = crystal_and_liquid(21)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.4)
    nl = nq.query(None, dict(r_max=1.4, exclude_ii=True)).toNeighborList()
    _, off, pj, _ = oracle.ball_query(b, x, 1.4)
    s_all, _, _, _ = oracle.solid_liquid(b, x, off, pj, 6, 0.7, 7)
    rng = np.random.default_rng(5)
    picks = s_all[rng.choice(len(s_all), 3, replace=False)]
    for qt in np.concatenate([picks - 1e-10, picks + 1e-10]):
        sl = fgb.SolidLiquid(6, float(qt), 6).compute(nq, nl)
        _, conn, idx, sizes = oracle.solid_liquid(b, x, off, pj, 6, float(qt), 6)
        assert np.array_equal(sl.num_connections.cpu().numpy(), conn)
        assert np.array_equal(sl.cluster_idx.cpu().numpy(), idx)
        assert np.array_equal(sl.clusters.cluster_sizes.cpu().numpy(), sizes)


SL_FP64_ONLY = r"""
import numpy as np, torch, oracle, workloads as W, paper_1906_06317_gb300 as fgb
import sys; sys.path.insert(0, 'tests')
from test_gpu_solidliquid import crystal_and_liquid, dev
b, x, _ = crystal_and_liquid(9)
nq = fgb.NeighborQuery(b, dev(x), r_cell=1.4)
nl = nq.query(None, dict(r_max=1.4, exclude_ii=True)).toNeighborList()
sl = fgb.SolidLiquid(6, 0.7, 7).compute(nq, nl)
_, off, pj, _ = oracle.ball_query(b, x, 1.4)
s, conn, idx, sizes = oracle.solid_liquid(b, x, off, pj, 6, 0.7, 7)
assert np.all(np.abs(sl.ql_ij.cpu().numpy() - s) <= 1e-6 * np.maximum(1.0, np.abs(s)))
assert np.array_equal(sl.num_connections.cpu().numpy(), conn)
assert np.array_equal(sl.cluster_idx.cpu().numpy(), idx)
print('ok')
"""


def test_solid_liquid_fp64_path():
    # FGB_SL_SCREEN=0: every bond and every Q_lm in FP64 (scores within 1e-6)
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root, FGB_SL_SCREEN="0")
    r = subprocess.run([sys.executable, "-c", SL_FP64_ONLY], env=env, cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
