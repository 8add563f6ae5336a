"""GPU parity of the Steinhardt variants (W_l, neighbor-averaged q_l) and of the per-bond
LocalDescriptors against the FP64 oracle.

Tolerances (FP32 sums of FP32 harmonics): normalised W_l within 1e-4 absolute and the
unnormalised one within 1e-4 * (sum_m |Q_lm|^2)^{3/2} (W_l is a sum of up to (2l+1)^2
products of three Q_lm, each off by ~1e-6 of |Q|); averaged q_l as q_l,
1e-5 * max(q_ref, 1e-2); descriptors within 2e-5 * max(1, |Y_ref|).
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


def fcc_liquid(seed):
    """Perturbed FCC crystal (c2-like, triclinic) next to a uniform liquid."""
    b = W.Box(4 * 1.5874, 4 * 1.5874, 4 * 1.5874, 0.1, 0.05, 0.0)
    rng = np.random.default_rng(seed)
    x = W.lattice_points(None, b, 4).astype(np.float64)
    x += rng.normal(scale=0.05, size=x.shape)
    liquid = W.uniform_points(rng, b, 200).astype(np.float64)
    return b, np.vstack([x, liquid]).astype(np.float32)


@pytest.mark.parametrize("l", [3, 4, 6, 8, 12])
def test_wl_matches_oracle(fgb, l):
    b, x = fcc_liquid(10 + l)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(l)
    st.compute(nq, neighbors=nl)
    _, off, pj, _ = oracle.ball_query(b, x, 1.3)
    _, Q = oracle.steinhardt(b, x, off, pj, l, with_qlm=True)
    w_ref = oracle.wl_from_qlm(Q, l, normalize=True)
    u_ref = oracle.wl_from_qlm(Q, l, normalize=False)
    s = np.abs(Q[:, 0]) ** 2 + 2 * np.sum(np.abs(Q[:, 1:]) ** 2, axis=1)
    w = st.wl(normalize=True).cpu().numpy()
    u = st.wl(normalize=False).cpu().numpy()
    assert np.all(np.abs(w - w_ref) <= 1e-4), np.abs(w - w_ref).max()
    assert np.all(np.abs(u - u_ref) <= 1e-4 * s ** 1.5 + 1e-12), np.abs(u - u_ref).max()


def test_wl_perfect_fcc_and_lone_points(fgb):
    b = W.Box.cube(4 * 1.5874)
    x = W.lattice_points(None, b, 4)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3)).toNeighborList()
    st = fgb.Steinhardt(6)
    st.compute(nq, neighbors=nl)
    assert np.allclose(st.wl().cpu().numpy(), -0.013161, atol=2e-5)
    lone = dev(np.array([[0.0, 0.0, 0.0], [3.0, 3.0, 3.0]]))
    nq2 = fgb.NeighborQuery(W.Box.cube(10.0), lone, r_cell=1.0)
    empty = nq2.query(None, dict(r_max=1.0)).toNeighborList()
    assert empty.n_pairs == 0  # an empty list is still a list (not "no list")
    st2 = fgb.Steinhardt(4)
    st2.compute(nq2, neighbors=empty)
    assert st2.wl().cpu().numpy().tolist() == [0.0, 0.0]
    assert st2.particle_order.cpu().numpy().tolist() == [0.0, 0.0]
    rdf = fgb.RDF(10, 1.0)
    rdf.compute(nq2, neighbors=empty)
    assert int(rdf.bin_counts.sum()) == 0


@pytest.mark.parametrize("l", [2, 4, 6, 12])
def test_average_matches_oracle_and_feeds_wl(fgb, l):
    b, x = fcc_liquid(30 + l)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.3)
    nl = nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(l)
    st.compute(nq, neighbors=nl)
    qb = st.average(nl).cpu().numpy()
    _, off, pj, _ = oracle.ball_query(b, x, 1.3)
    qb_ref, Qb = oracle.steinhardt_average(b, x, off, pj, l, with_qlm=True)
    assert np.all(np.abs(qb - qb_ref) <= 1e-5 * np.maximum(qb_ref, 1e-2)), np.abs(qb - qb_ref).max()
    w = st.wl().cpu().numpy()
    assert np.all(np.abs(w - oracle.wl_from_qlm(Qb, l)) <= 1e-4)
    with pytest.raises(fgb.FGBError) as e:
        st.backward()
    assert e.value.code == fgb.ERR_UNSUPPORTED


@pytest.mark.parametrize("l_max,neg", [(0, True), (4, False), (6, True), (12, True)])
def test_descriptors_match_oracle(fgb, l_max, neg):
    b = W.Box(9.0, 10.0, 11.0, 0.1, -0.15, 0.2)
    x = W.small_random(40 + l_max, 1500, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.6)
    nl = nq.query(None, dict(r_max=1.6, exclude_ii=True)).toNeighborList()
    ld = fgb.LocalDescriptors(l_max, negative_m=neg).compute(nq, nl)
    qi = nl.query_point_indices.cpu().numpy()
    pj = nl.point_indices.cpu().numpy()
    ref = oracle.local_descriptors(b, x, qi, pj, l_max, negative_m=neg)
    got = ld.sph.cpu().numpy()
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= 2e-5 * np.maximum(1.0, np.abs(ref))), np.abs(got - ref).max()


def test_descriptors_separate_query_points_and_empty(fgb):
    b = W.Box.cube(10.0)
    x = W.small_random(50, 800, b)
    y = W.small_random(51, 90, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.0)
    nl = nq.query(dev(y), dict(r_max=2.0, exclude_ii=False)).toNeighborList()
    ld = fgb.LocalDescriptors(6).compute(nq, nl, query_points=dev(y))
    ref = oracle.local_descriptors(b, x, nl.query_point_indices.cpu().numpy(), nl.point_indices.cpu().numpy(), 6,
                                   query_points=y)
    assert np.all(np.abs(ld.sph.cpu().numpy() - ref) <= 2e-5 * np.maximum(1.0, np.abs(ref)))
    far = dev(np.full((1, 3), 4.99, np.float32))  # almost surely nothing within 0.001
    empty = nq.query(far, dict(r_max=0.001, exclude_ii=False)).toNeighborList()
    assert fgb.LocalDescriptors(3).compute(nq, empty, query_points=far).sph.shape == (empty.n_pairs, 16)
