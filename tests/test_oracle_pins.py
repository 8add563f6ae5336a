"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each check is chosen so a plausible slip in the oracle (dropped image term, wrong tilt
index, off-by-one bin, sign of a spherical-harmonic phase, missing Legendre term,
transposed gradient) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.special import sph_harm_y

import oracle
import workloads as W
from tests.helpers import image_distances, legendre_p, nl_sets, q_from_bonds

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

BOXES = [
    W.Box.cube(10.0),
    W.Box(11.0, 9.5, 10.5, 0.1, 0.05, 0.0),
    W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15),
    W.Box(10.0, 10.0, 10.0, 0.2, -0.2, -0.2),
]


def _pairs(offsets, pj):
    qi = np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))
    return qi, pj


@pytest.mark.parametrize("bi", range(len(BOXES)))
def test_min_image_is_true_nearest_image(bi):
    b = BOXES[bi]
    rng = np.random.default_rng(10 + bi)
    x = W.uniform_points(rng, b, 60).astype(np.float64)
    x[:10] += 3.0 * rng.normal(size=(10, 3))          # some points outside the box
    ref = image_distances(b, x, x, reach=3)
    wmin = oracle.box_widths(b).min()
    for i in range(0, 60, 7):
        for j in range(60):
            d, r = oracle.min_image(b, x[i], x[j])
            if ref[i, j] < 0.5 * wmin:
                assert r == pytest.approx(ref[i, j], rel=1e-12, abs=1e-12)
            else:
                assert r >= ref[i, j] - 1e-12


def test_box_widths_closed_form():
    b = W.Box(12.0, 10.0, 11.0, -0.2, 0.2, 0.15)
    M = np.array([[12.0, -2.0, 2.2], [0.0, 10.0, 1.65], [0.0, 0.0, 11.0]])
    inv = np.linalg.inv(M)
    w = 1.0 / np.linalg.norm(inv, axis=1)              # plane spacing = 1/|reciprocal row|
    assert np.allclose(oracle.box_widths(b), w, rtol=1e-14)


@pytest.mark.parametrize("bi", range(len(BOXES)))
@pytest.mark.parametrize("r_max", [1.1, 2.3, 4.3])
def test_ball_cells_equal_brute(bi, r_max):
    b = BOXES[bi]
    x = W.small_random(20 + bi, 1200, b)
    c1, o1, p1, d1 = oracle.ball_query(b, x, r_max, brute=True)
    c2, o2, p2, d2 = oracle.ball_query(b, x, r_max)
    assert np.array_equal(o1, o2) and np.array_equal(p1, p2) and np.array_equal(d1, d2)
    assert all(np.all(np.diff(p1[o1[i]:o1[i + 1]]) > 0) for i in range(len(x)))


@pytest.mark.parametrize("bi", range(len(BOXES)))
def test_ball_matches_image_enumeration(bi):
    b = BOXES[bi]
    x = W.small_random(30 + bi, 400, b)
    r_max = 2.7
    ref = image_distances(b, x, x)
    np.fill_diagonal(ref, np.inf)
    _, o, pj, dist = oracle.ball_query(b, x, r_max)
    got = nl_sets(o, pj)
    margin = 1e-9
    for i in range(len(x)):
        sure = set(np.nonzero(ref[i] < r_max - margin)[0].tolist())
        maybe = set(np.nonzero(ref[i] < r_max + margin)[0].tolist())
        assert sure <= got[i] <= maybe
        assert np.allclose(dist[o[i]:o[i + 1]], ref[i, pj[o[i]:o[i + 1]]], rtol=1e-12)


def test_ball_matches_ckdtree_cubic():
    L = 12.0
    b = W.Box.cube(L)
    x = W.small_random(40, 3000, b).astype(np.float64)
    r_max = 1.7
    tree = cKDTree(x + L / 2, boxsize=L)
    ref = tree.query_pairs(r_max - 1e-9, output_type="ndarray")
    ref_hi = tree.query_pairs(r_max + 1e-9, output_type="ndarray")
    _, o, pj, _ = oracle.ball_query(b, x.astype(np.float32), r_max)
    qi, _ = _pairs(o, pj)
    got = {(int(a), int(c)) for a, c in zip(qi, pj) if a < c}
    lo = {(int(a), int(c)) for a, c in ref}
    hi = {(int(a), int(c)) for a, c in ref_hi}
    assert lo <= got <= hi and len(got) > 1000


def test_fcc_shell_counts():
    g = json.load(open(os.path.join(GOLDEN, "fcc_shells.json")))
    a = 1.5874
    n = 4
    b = W.Box.cube(n * a)
    x = W.lattice_points(None, b, n)
    radii = [a * s for s in g["shell_radius_over_a"]] + [1e9]
    for t, want in enumerate(g["cumulative_counts"]):
        r_max = 0.5 * (radii[t] + radii[t + 1]) if t + 1 < len(g["cumulative_counts"]) else radii[t] + 0.05
        c, *_ = oracle.ball_query(b, x, r_max)
        assert np.all(c == want), (t, np.unique(c))


def test_neighbor_list_symmetry_and_translation():
    b = W.Box(10.0, 10.0, 10.0, 0.15, -0.1, 0.05)
    x = W.small_random(50, 1500, b)
    _, o, pj, _ = oracle.ball_query(b, x, 2.2)
    qi, _ = _pairs(o, pj)
    fwd = set(zip(qi.tolist(), pj.tolist()))
    assert fwd == {(j, i) for i, j in fwd}
    # translation by whole box vectors is exact in FP64 here, so sets and order are identical
    M = W.Box(10.0, 10.0, 10.0, 0.15, -0.1, 0.05).matrix()
    rng = np.random.default_rng(0)
    xs = x.astype(np.float64) + (rng.integers(-2, 3, size=(len(x), 3)) @ M.T)
    _, o2, pj2, d2 = oracle.ball_query(b, xs, 2.2)
    assert np.array_equal(o, o2) and np.array_equal(pj, pj2)


@pytest.mark.parametrize("bi", [0, 2])
def test_knn_equals_full_sort(bi):
    b = BOXES[bi]
    x = W.small_random(60 + bi, 700, b)
    k = 12
    n1, j1, r1 = oracle.knn(b, x, k, brute=True)
    n2, j2, r2 = oracle.knn(b, x, k)
    assert np.array_equal(n1, n2) and np.array_equal(j1, j2) and np.array_equal(r1, r2)
    ref = image_distances(b, x, x)
    np.fill_diagonal(ref, np.inf)
    order = np.lexsort((np.broadcast_to(np.arange(len(x)), ref.shape), ref), axis=1)[:, :k]
    gaps = np.diff(np.sort(ref, axis=1)[:, : k + 1], axis=1).min(axis=1)
    clear = gaps > 1e-9                                  # no near-tie anywhere in the first k+1
    assert clear.mean() > 0.95
    assert np.array_equal(j1[clear], order[clear])
    assert np.allclose(r1, np.take_along_axis(ref, j1, axis=1), rtol=1e-12)


def test_knn_small_n_and_box_limits():
    b = W.Box.cube(20.0)
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.5]], np.float32)
    n, j, r = oracle.knn(b, x, 12)
    assert np.all(n == 3)
    assert j[0, :3].tolist() == [1, 2, 3] and np.allclose(r[0, :3], [1.0, 2.0, 3.5])
    n, j, r = oracle.knn(b, x[:1], 12)
    assert n[0] == 0
    far = np.array([[0.0, 0.0, 0.0], [9.9, 9.9, 9.9]], np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.knn(b, far, 1)
    assert e.value.code == oracle.ERR_BOX_TOO_SMALL
    with pytest.raises(oracle.OracleError) as e:
        oracle.ball_query(b, x, 10.0)
    assert e.value.code == oracle.ERR_BOX_TOO_SMALL


def test_rdf_histogram_against_numpy():
    b = W.Box(9.0, 10.0, 11.0, 0.1, 0.0, -0.1)
    x = W.small_random(70, 800, b)
    bins, r_min, r_max = 37, 0.3, 4.1
    ref = image_distances(b, x, x)
    np.fill_diagonal(ref, np.inf)
    delta = (r_max - r_min) / bins
    edges = np.array([r_min + k * delta for k in range(bins)] + [r_max])
    assert np.array_equal(edges, oracle.rdf_edges(bins, r_min, r_max))
    r = ref[np.isfinite(ref)]
    r = r[(r >= r_min) & (r < r_max)]
    want = np.histogram(r, bins=edges)[0]
    got = oracle.rdf_counts(b, x, bins, r_max, r_min)
    assert np.array_equal(got, want.astype(np.uint64))
    assert np.array_equal(oracle.rdf_counts(b, x, bins, r_max, r_min, brute=True), got)


def test_rdf_total_equals_neighbor_count():
    b = W.Box.cube(16.0)
    x = W.c1().points[:2048]
    c, *_ = oracle.ball_query(b, x, 4.0)
    h = oracle.rdf_counts(b, x, 100, 4.0)
    assert int(h.sum()) == int(c.sum())


def test_rdf_ideal_gas():
    w = W.c1()
    p = w.params
    counts = oracle.rdf_counts(w.box, w.points, p["rdf_bins"], p["rdf_r_max"])
    n = len(w.points)
    g, centers = oracle.rdf_normalize(counts, n, n, w.box.volume, p["rdf_bins"], 0.0, p["rdf_r_max"])
    e = oracle.rdf_edges(p["rdf_bins"], 0.0, p["rdf_r_max"])
    expect = n * (n - 1) / w.box.volume * 4.0 / 3.0 * math.pi * (e[1:] ** 3 - e[:-1] ** 3)
    ok = expect > 200
    sigma = np.sqrt(2.0 / expect[ok])
    assert np.all(np.abs(g[ok] - (1.0 - 1.0 / n)) < 5.0 * sigma)
    assert centers[0] == pytest.approx(0.02) and centers[-1] == pytest.approx(3.98)


def test_ylm_matches_scipy():
    rng = np.random.default_rng(80)
    for _ in range(20):
        v = rng.normal(size=3)
        th = math.acos(v[2] / np.linalg.norm(v))
        ph = math.atan2(v[1], v[0])
        for l in (0, 1, 2, 4, 6, 8, 12):
            for m in range(-l, l + 1):
                assert oracle.ylm(l, m, v) == pytest.approx(complex(sph_harm_y(l, m, th, ph)), abs=1e-12)


def _lattice_q(basis, nn, l):
    b = W.Box.cube(6.0)
    x = W.lattice_points(None, b, 6, basis=basis)
    shells = image_distances(b, x[:1], x)[0]
    r_first = np.sort(shells)[1]
    r_max = r_first * 1.05
    _, o, pj, _ = oracle.ball_query(b, x, r_max)
    assert np.all(np.diff(o) == nn)
    return oracle.steinhardt(b, x, o, pj, l), oracle.steinhardt_legendre(b, x, o, pj, l)


@pytest.mark.parametrize("name,basis,nn", [("fcc_12", W.FCC_BASIS, 12), ("bcc_8", W.BCC_BASIS, 8),
                                            ("sc_6", W.SC_BASIS, 6)])
def test_steinhardt_perfect_lattices(name, basis, nn):
    g = json.load(open(os.path.join(GOLDEN, "steinhardt_lattices.json")))[name]
    for l in (4, 6):
        q1, q2 = _lattice_q(basis, nn, l)
        assert np.allclose(q1, g[f"q{l}"], atol=g["tol"])
        assert np.allclose(q1, q2, atol=1e-12)


def test_steinhardt_closed_forms_numpy():
    # SC: dot products 1 (x6), -1 (x6), 0 (x24): q_l = sqrt(6 P(1) + 6 P(-1) + 24 P(0)) / 6
    for l in (4, 6):
        S = 6 * legendre_p(l, 1.0) + 6 * legendre_p(l, -1.0) + 24 * legendre_p(l, 0.0)
        sc = math.sqrt(S) / 6
        q1, _ = _lattice_q(W.SC_BASIS, 6, l)
        assert np.allclose(q1, sc, atol=1e-12)
    fcc_bonds = np.array([[a, b_, 0] for a in (1, -1) for b_ in (1, -1)] + [[a, 0, b_] for a in (1, -1) for b_ in (1, -1)]
                         + [[0, a, b_] for a in (1, -1) for b_ in (1, -1)], np.float64)
    for l in (4, 6):
        q1, _ = _lattice_q(W.FCC_BASIS, 12, l)
        assert np.allclose(q1, q_from_bonds(fcc_bonds, l), atol=1e-12)


def test_steinhardt_single_neighbor_and_empty():
    b = W.Box.cube(10.0)
    x = np.array([[0.0, 0.0, 0.0], [0.3, 1.1, -0.4], [4.0, 4.0, 4.0]], np.float64)
    off = np.array([0, 1, 2, 2])
    pj = np.array([1, 0])
    for l in (2, 4, 6, 8):
        q = oracle.steinhardt(b, x, off, pj, l)
        assert q[0] == pytest.approx(1.0, abs=1e-13) and q[1] == pytest.approx(1.0, abs=1e-13) and q[2] == 0.0
        assert np.allclose(oracle.steinhardt_legendre(b, x, off, pj, l), q, atol=1e-13)


def test_steinhardt_forms_agree_and_rotation_invariant():
    w = W.c2(n_cells=4)
    _, o, pj, _ = oracle.ball_query(w.box, w.points, 1.3)
    for l in (4, 6):
        q1 = oracle.steinhardt(w.box, w.points, o, pj, l)
        q2 = oracle.steinhardt_legendre(w.box, w.points, o, pj, l)
        assert np.allclose(q1, q2, atol=1e-12)
    # an isolated cluster in a big box: rotating it leaves q_l unchanged
    rng = np.random.default_rng(81)
    cl = rng.normal(size=(14, 3))
    big = W.Box.cube(100.0)
    off = np.array([0, 13] + [13] * 13)
    pj = np.arange(1, 14)
    R = W.random_rotation(rng)
    for l in (3, 4, 6, 10):
        a = oracle.steinhardt(big, cl, off, pj, l)[0]
        c = oracle.steinhardt(big, cl @ R.T, off, pj, l)[0]
        assert a == pytest.approx(c, abs=1e-12)
        assert a == pytest.approx(q_from_bonds(cl[1:] - cl[0], l), abs=1e-12)


def test_q_gradient_finite_differences():
    w = W.c4(n_cells=4)
    x = w.points.astype(np.float64)
    l = 6
    _, o, pj, _ = oracle.ball_query(w.box, w.points, 1.3)
    g = oracle.q_grad(w.box, x, o, pj, l)
    assert np.allclose(g.sum(axis=0), 0.0, atol=1e-14)
    n = len(x)
    h = 1e-3
    rng = np.random.default_rng(82)
    picks = rng.choice(n, 40, replace=False)
    for k in picks:
        affected = np.unique(np.concatenate([[k], pj[o[k]:o[k + 1]]]))
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            # only k and its neighbors change; the other terms of the mean cancel
            fp = oracle.steinhardt(w.box, xp, o, pj, l, which=affected).sum() / n
            fm = oracle.steinhardt(w.box, xm, o, pj, l, which=affected).sum() / n
            fd = (fp - fm) / (2 * h)
            assert fd == pytest.approx(g[k, c], rel=1e-4, abs=1e-4 * np.abs(g).max())


# ------------------------------------------------- Wigner 3j, W_l, averaged q_l, Y_lm


def _w3j_all_zero_m(l1, l2, l3):
    """(l1 l2 l3; 0 0 0) by its closed form: 0 for odd L = l1+l2+l3, else
    (-1)^(L/2) sqrt[(L-2l1)!(L-2l2)!(L-2l3)!/(L+1)!] (L/2)!/[(L/2-l1)!(L/2-l2)!(L/2-l3)!]."""
    L = l1 + l2 + l3
    if L % 2:
        return 0.0
    f = math.factorial
    g = L // 2
    return (-1) ** g * math.sqrt(f(L - 2 * l1) * f(L - 2 * l2) * f(L - 2 * l3) / f(L + 1)) * f(g) / (
        f(g - l1) * f(g - l2) * f(g - l3))


def test_wigner3j_closed_forms_and_symmetries():
    for l in range(0, 9):
        for m in range(-l, l + 1):  # (l l 0; m -m 0) = (-1)^(l-m) / sqrt(2l+1)
            assert oracle.wigner3j(l, l, 0, m, -m, 0) == pytest.approx((-1) ** (l - m) / math.sqrt(2 * l + 1),
                                                                        abs=1e-14)
    for l1, l2, l3 in [(4, 4, 4), (6, 6, 6), (2, 3, 3), (5, 6, 7), (12, 12, 12), (3, 4, 5)]:
        assert oracle.wigner3j(l1, l2, l3, 0, 0, 0) == pytest.approx(_w3j_all_zero_m(l1, l2, l3), abs=1e-14)
    # column permutations: cyclic ones keep the value, odd ones and m -> -m give (-1)^L
    rng = np.random.default_rng(1)
    for _ in range(40):
        l1, l2 = rng.integers(0, 7, 2)
        l3 = int(rng.integers(abs(l1 - l2), l1 + l2 + 1))
        m1 = int(rng.integers(-l1, l1 + 1))
        m2 = int(rng.integers(-l2, l2 + 1))
        m3 = -m1 - m2
        if abs(m3) > l3:
            continue
        v = oracle.wigner3j(l1, l2, l3, m1, m2, m3)
        sg = (-1) ** (l1 + l2 + l3)
        assert oracle.wigner3j(l2, l3, l1, m2, m3, m1) == pytest.approx(v, abs=1e-14)
        assert oracle.wigner3j(l2, l1, l3, m2, m1, m3) == pytest.approx(sg * v, abs=1e-14)
        assert oracle.wigner3j(l1, l2, l3, -m1, -m2, -m3) == pytest.approx(sg * v, abs=1e-14)


def test_wigner3j_orthogonality():
    # sum_{m1,m2} (l1 l2 l3; m1 m2 m3)(l1 l2 l3'; m1 m2 m3') = delta delta / (2 l3 + 1)
    for l1, l2 in [(3, 4), (6, 6)]:
        for l3 in range(abs(l1 - l2), l1 + l2 + 1, 3):
            for l3b in (l3, min(l1 + l2, l3 + 1)):
                for m3 in (-min(l3, l3b), 0, min(l3, l3b)):
                    s = sum(oracle.wigner3j(l1, l2, l3, m1, -m1 - m3, m3) * oracle.wigner3j(l1, l2, l3b, m1, -m1 - m3, m3)
                            for m1 in range(-l1, l1 + 1) if abs(m1 + m3) <= l2)
                    want = 1.0 / (2 * l3 + 1) if l3 == l3b else 0.0
                    assert s == pytest.approx(want, abs=1e-13)


def test_wl_single_bond_and_lattices():
    # one bond: Q_lm = Y_lm(u), which rotates into delta_m0 sqrt((2l+1)/4pi), so the
    # normalised W_l is (l l l; 0 0 0) for every direction
    b = W.Box.cube(10.0)
    rng = np.random.default_rng(4)
    x = np.vstack([[0.0, 0.0, 0.0], rng.normal(size=(1, 3))])
    off, pj = np.array([0, 1, 2]), np.array([1, 0])
    for l in (2, 3, 4, 6, 8):
        w = oracle.wl(b, x, off, pj, l)
        assert np.allclose(w, _w3j_all_zero_m(l, l, l), atol=1e-12)
    g = json.load(open(os.path.join(GOLDEN, "wl_lattices.json")))
    bf = W.Box.cube(4 * 1.5874)
    xf = W.lattice_points(None, bf, 4)
    _, o, pj, _ = oracle.ball_query(bf, xf, 1.3)
    for l in (4, 6):
        assert np.allclose(oracle.wl(bf, xf, o, pj, l), g["fcc_12"][f"w{l}"], atol=g["fcc_12"]["tol"])
    phi = (1 + 5 ** 0.5) / 2
    v = np.array([p for s1 in (-1, 1) for s2 in (-1, 1) for p in ((0, s1, s2 * phi), (s1, s2 * phi, 0),
                                                                  (s2 * phi, 0, s1))], np.float64)
    v /= np.linalg.norm(v[0])
    xi = np.vstack([[0.0, 0.0, 0.0], v])
    oi, pi = np.array([0] + [12] * 13), np.arange(1, 13)
    bi = W.Box.cube(20.0)
    ico = g["icosahedral_12"]
    assert oracle.wl(bi, xi, oi, pi, 6)[0] == pytest.approx(ico["w6"], abs=ico["tol"])
    assert oracle.steinhardt(bi, xi, oi, pi, 6)[0] == pytest.approx(ico["q6"], abs=ico["tol"])


def test_wl_rotation_invariant_and_unnormalised_scale():
    b = W.Box.cube(30.0)
    rng = np.random.default_rng(6)
    bonds = rng.normal(size=(9, 3))
    R = W.random_rotation(np.random.default_rng(7))
    x1, x2 = np.vstack([[0, 0, 0], bonds]), np.vstack([[0, 0, 0], bonds @ R.T])
    off, pj = np.array([0] + [9] * 10), np.arange(1, 10)
    for l in (4, 6):
        w1, w2 = oracle.wl(b, x1, off, pj, l), oracle.wl(b, x2, off, pj, l)
        assert w1[0] == pytest.approx(w2[0], abs=1e-12)
        _, Q = oracle.steinhardt(b, x1, off, pj, l, with_qlm=True)
        s = np.abs(Q[0, 0]) ** 2 + 2 * np.sum(np.abs(Q[0, 1:]) ** 2)
        assert oracle.wl(b, x1, off, pj, l, normalize=False)[0] == pytest.approx(w1[0] * s ** 1.5, abs=1e-12)


def test_average_pair_lattice_and_isolated():
    b = W.Box.cube(10.0)
    # two points, each the other's only neighbor: Qbar = (Y(u) + Y(-u)) / 2, so qbar_l is
    # 1 for even l (a single bond has q_l = 1) and 0 for odd l; a lone point gives 0
    x = np.array([[0.0, 0.0, 0.0], [0.4, -1.0, 0.7], [4.0, 4.0, 4.0]])
    off, pj = np.array([0, 1, 2, 2]), np.array([1, 0])
    for l in (1, 2, 3, 4, 5, 6):
        qb = oracle.steinhardt_average(b, x, off, pj, l)
        want = 1.0 if l % 2 == 0 else 0.0
        assert np.allclose(qb[:2], want, atol=1e-12) and qb[2] == 0.0
    bf = W.Box.cube(4 * 1.5874)
    xf = W.lattice_points(None, bf, 4)
    _, o, pj, _ = oracle.ball_query(bf, xf, 1.3)
    for l in (4, 6):  # every particle of a perfect crystal has the same Q_lm
        assert np.allclose(oracle.steinhardt_average(bf, xf, o, pj, l), oracle.steinhardt(bf, xf, o, pj, l), atol=1e-12)


def test_descriptors_addition_theorem_and_axes():
    b = W.Box.cube(10.0)
    x = W.small_random(8, 300, b).astype(np.float64)
    _, o, pj, _ = oracle.ball_query(b, x, 2.0)
    qi = np.repeat(np.arange(len(x)), np.diff(o))
    Y = oracle.local_descriptors(b, x, qi, pj, 6)
    k = 0
    for l in range(7):  # sum_m |Y_lm|^2 = (2l+1)/(4 pi) for every bond
        assert np.allclose(np.sum(np.abs(Y[:, k:k + 2 * l + 1]) ** 2, axis=1), (2 * l + 1) / (4 * math.pi),
                           atol=1e-12)
        k += 2 * l + 1
    z = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.5], [1.5, 0.0, 0.0]])
    Yz = oracle.local_descriptors(b, z, [0, 0], [1, 2], 3, negative_m=False)
    k = 0
    for l in range(4):  # along z only m = 0: sqrt((2l+1)/4pi); along x, Y_11 = -sqrt(3/8pi)
        assert Yz[0, k] == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), abs=1e-13)
        assert np.allclose(Yz[0, k + 1:k + l + 1], 0, atol=1e-13)
        k += l + 1
    assert Yz[1, 2] == pytest.approx(-math.sqrt(3 / (8 * math.pi)), abs=1e-13)


def test_clusters_match_connected_components_and_ordering():
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    b = W.Box(10.0, 9.0, 11.0, 0.1, 0.0, -0.1)
    x = W.small_random(21, 1500, b)
    _, o, pj, _ = oracle.ball_query(b, x, 0.55)
    qi = np.repeat(np.arange(len(x)), np.diff(o))
    rng = np.random.default_rng(2)
    for mask in (None, rng.random(len(qi)) < 0.6):
        idx, sizes = oracle.clusters(len(x), qi, pj, mask)
        keep = np.ones(len(qi), bool) if mask is None else mask
        g = coo_matrix((np.ones(keep.sum()), (qi[keep], pj[keep])), shape=(len(x), len(x)))
        ncc, lab = connected_components(g, directed=True, connection="weak")
        assert len(sizes) == ncc and sizes.sum() == len(x)
        # same partition: the pairs of labels form a bijection
        assert len(set(zip(idx.tolist(), lab.tolist()))) == ncc
        assert np.all(np.diff(sizes) <= 0)
        firsts = np.array([np.nonzero(idx == c)[0][0] for c in range(len(sizes))])
        same = np.diff(sizes) == 0
        assert np.all(np.diff(firsts)[same] > 0), "ties not ordered by smallest member"


def test_cluster_properties_closed_forms_and_periodic_shift():
    b = W.Box.cube(10.0)
    # a pair 0.6 apart through the x face (x = 4.8 and -4.6): centre 5.1, wrapped to -4.9;
    # offsets from it are -+0.3 along x, so the gyration tensor is diag(0.09, 0, 0)
    x = np.array([[4.8, 1.0, -2.0], [-4.6, 1.0, -2.0], [0.0, 0.0, 0.0]])
    c, g = oracle.cluster_properties(b, x, np.array([0, 0, 1]))
    assert np.allclose(c[0], [-4.9, 1.0, -2.0], atol=1e-12)
    assert np.allclose(g[0], np.diag([0.3 ** 2, 0.0, 0.0]), atol=1e-12)
    assert np.allclose(g[1], 0.0) and np.allclose(c[1], 0.0)
    # translating a cluster across the box moves its centre by the same amount (mod the
    # box) and leaves its gyration tensor unchanged; the tensor is the population covariance
    rng = np.random.default_rng(3)
    blob = rng.normal(size=(30, 3)) * 0.5
    t = np.array([4.7, -3.2, 4.9])
    c1, g1 = oracle.cluster_properties(b, blob, np.zeros(30, np.int64))
    c2, g2 = oracle.cluster_properties(b, blob + t, np.zeros(30, np.int64))
    dc = (c2[0] - c1[0] - t + 5.0) % 10.0 - 5.0
    assert np.allclose(dc, 0.0, atol=1e-10) and np.allclose(g1, g2, atol=1e-10)
    assert np.allclose(g1[0], np.cov((blob - blob.mean(0)).T, bias=True), atol=1e-12)


def test_solid_liquid_crystal_pair_and_symmetry():
    # perfect FCC: every particle has the same Q_lm, so s_ij = 1 on every bond, all 12
    # bonds are solid-like and the crystal is one cluster; unnormalised, s_ij = sum_m
    # |Q_lm|^2 = (2l+1)/(4 pi) q_l^2
    b = W.Box.cube(4 * 1.5874)
    x = W.lattice_points(None, b, 4)
    _, o, pj, _ = oracle.ball_query(b, x, 1.3)
    s, conn, idx, sizes = oracle.solid_liquid(b, x, o, pj, 6, 0.7, 7)
    assert np.allclose(s, 1.0, atol=1e-12) and np.all(conn == 12)
    assert len(sizes) == 1 and sizes[0] == len(x)
    q6 = oracle.steinhardt(b, x, o, pj, 6)
    su, _, _, _ = oracle.solid_liquid(b, x, o, pj, 6, 0.0, 1, normalize_q=False)
    assert np.allclose(su, 13 / (4 * math.pi) * q6[0] ** 2, atol=1e-12)
    # two points, each the other's only neighbor: Q(2) = Y(-u) = (-1)^l Y(u), s = (-1)^l
    b2 = W.Box.cube(10.0)
    x2 = np.array([[0.0, 0.0, 0.0], [0.3, -0.8, 0.5], [4.0, 4.0, 4.0]])
    o2, pj2 = np.array([0, 1, 2, 2]), np.array([1, 0])
    for l in (3, 4, 6):
        s2, conn2, idx2, _ = oracle.solid_liquid(b2, x2, o2, pj2, l, 0.5, 1)
        assert np.allclose(s2, (-1) ** l, atol=1e-12)
        assert list(conn2) == ([1, 1, 0] if l % 2 == 0 else [0, 0, 0])
        assert (idx2[0] == idx2[1]) == (l % 2 == 0)
    # symmetric list: s_ij = s_ji
    xr = W.small_random(31, 800, b2)
    _, o3, pj3, _ = oracle.ball_query(b2, xr, 1.5)
    s3, _, _, _ = oracle.solid_liquid(b2, xr, o3, pj3, 6, 0.7, 7)
    qi3 = np.repeat(np.arange(len(xr)), np.diff(o3))
    fwd = dict(zip(zip(qi3.tolist(), pj3.tolist()), s3.tolist()))
    assert all(fwd[(j, i)] == v for (i, j), v in fwd.items())
