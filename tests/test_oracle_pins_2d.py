"""Pins of the oracle's 2D boxes and PMFT(x, y) against facts fixed outside it (CPU only).

A 2D box (Lz = 0) has parallelogram widths, no z period and annulus RDF shells; the PMFT
counts bonds in the frame of the query particle.  Plausible slips that a check here
catches: a z reduction by Lz = 0, the 3D shell volume in 2D, a bond rotated by +theta
instead of -theta, x and y bins swapped, an off-by-one bin, the bond taken as
q_i - x_j, the bond turned by the orientation of the wrong particle.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import workloads as W
from tests.helpers import image_vectors_2d

BOXES2 = [W.Box.square(12.0), W.Box(11.0, 9.0, 0.0, 0.25), W.Box(10.0, 12.5, 0.0, -0.3)]


def _qi(off):
    return np.repeat(np.arange(len(off) - 1), np.diff(off))


def test_2d_box_widths_closed_form():
    b = W.Box(10.0, 8.0, 0.0, 0.3)
    a2 = np.array([0.3 * 8.0, 8.0])
    w = oracle.box_widths(b)
    assert w[0] == pytest.approx(80.0 / np.linalg.norm(a2), rel=1e-14)
    assert w[1] == pytest.approx(8.0, rel=1e-14) and math.isinf(w[2])


@pytest.mark.parametrize("bi", range(len(BOXES2)))
def test_2d_min_image_is_nearest_image(bi):
    b = BOXES2[bi]
    rng = np.random.default_rng(300 + bi)
    x = W.uniform_points(rng, b, 50).astype(np.float64)
    x[:8, :2] += 4.0 * rng.normal(size=(8, 2))        # some points outside the box
    ref = image_vectors_2d(b, x, x)
    wmin = oracle.box_widths(b)[:2].min()
    for i in range(0, 50, 5):
        for j in range(50):
            d, r = oracle.min_image(b, x[i], x[j])
            assert d[2] == 0.0
            if np.linalg.norm(ref[i, j]) < 0.5 * wmin:
                assert np.allclose(d[:2], ref[i, j], atol=1e-12)


@pytest.mark.parametrize("bi", range(len(BOXES2)))
def test_2d_ball_query_brute_and_slab(bi):
    b = BOXES2[bi]
    x = W.small_random(310 + bi, 900, b)
    assert np.all(x[:, 2] == 0.0)
    r = 1.7
    c, off, pj, dist = oracle.ball_query(b, x, r)
    c2, off2, pj2, dist2 = oracle.ball_query(b, x, r, brute=True)
    assert np.array_equal(off, off2) and np.array_equal(pj, pj2) and np.array_equal(dist, dist2)
    ref = np.linalg.norm(image_vectors_2d(b, x, x), axis=-1)
    np.fill_diagonal(ref, np.inf)
    want = [np.flatnonzero(row < r) for row in ref]
    assert np.array_equal(np.diff(off), [len(w) for w in want])
    assert np.array_equal(pj, np.concatenate(want))
    # the same points in a 3D slab thicker than 2 r (no z image within reach)
    slab = W.Box(b.Lx, b.Ly, 5.0, b.xy)
    _, off3, pj3, dist3 = oracle.ball_query(slab, x, r)
    assert np.array_equal(off, off3) and np.array_equal(pj, pj3) and np.array_equal(dist, dist3)


def test_2d_ball_query_matches_periodic_kdtree():
    b = W.Box.square(15.0)
    x = W.small_random(320, 1500, b)
    _, off, pj, _ = oracle.ball_query(b, x, 1.3)
    t = cKDTree(x[:, :2].astype(np.float64) + 7.5, boxsize=15.0)
    ref = t.query_ball_point(x[:, :2].astype(np.float64) + 7.5, 1.3 - 1e-12)
    for i in range(len(x)):
        assert sorted(set(ref[i]) - {i}) == pj[off[i]:off[i + 1]].tolist()


def test_2d_knn_equals_full_sort():
    b = BOXES2[1]
    x = W.small_random(330, 600, b)
    k = 7
    n_found, idx, dist = oracle.knn(b, x, k)
    ref = np.linalg.norm(image_vectors_2d(b, x, x), axis=-1)
    np.fill_diagonal(ref, np.inf)
    for i in range(0, 600, 13):
        order = np.lexsort((np.arange(600), ref[i]))[:k]
        assert np.array_equal(idx[i], order)
        assert np.allclose(dist[i], ref[i, order], atol=1e-12)


def test_2d_rdf_histogram_and_ideal_gas():
    b = BOXES2[1]
    x = W.small_random(340, 800, b)
    bins, r_max = 30, 4.0
    ref = np.linalg.norm(image_vectors_2d(b, x, x), axis=-1)
    np.fill_diagonal(ref, np.inf)
    r = ref[ref < r_max]
    want = np.histogram(r, bins=oracle.rdf_edges(bins, 0.0, r_max))[0]
    assert np.array_equal(oracle.rdf_counts(b, x, bins, r_max), want.astype(np.uint64))
    f = W.p6(seed=341, n=20000, n_frames=1)[0]
    n = len(f.points)
    counts = oracle.rdf_counts(f.box, f.points, 50, 5.0)
    g, _ = oracle.rdf_normalize(counts, n, n, f.box.area, 50, 0.0, 5.0, dim=2)
    e = oracle.rdf_edges(50, 0.0, 5.0)
    expect = n * (n - 1) / f.box.area * math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    ok = expect > 500
    assert ok.sum() > 40
    assert np.all(np.abs(g[ok] - (1.0 - 1.0 / n)) < 5.0 * np.sqrt(2.0 / expect[ok]))


def test_pmft_hand_worked_bonds():
    # particle 0 at the origin, particle 1 at (0.75, 0.3); x_max = y_max = 1, 4 x 4 bins
    # of 0.5.  theta = (0, 0): bond 0->1 = (0.75, 0.3) -> bin (3, 2); bond 1->0 =
    # (-0.75, -0.3) -> bin (0, 1).  theta_0 = pi/2: bond 0->1 turned by -pi/2 is
    # (0.3, -0.75) -> bin (2, 0).
    b = W.Box.square(10.0)
    x = np.array([[0.0, 0.0, 0.0], [0.75, 0.3, 0.0]], np.float32)
    c = oracle.pmftxy(b, x, np.zeros(2, np.float32), 1.0, 1.0, 4, 4)
    want = np.zeros((4, 4), np.int64)
    want[3, 2] = want[0, 1] = 1
    assert np.array_equal(c, want)
    c = oracle.pmftxy(b, x, np.array([np.pi / 2, 0.0], np.float32), 1.0, 1.0, 4, 4)
    want = np.zeros((4, 4), np.int64)
    want[2, 0] = want[0, 1] = 1
    assert np.array_equal(c, want)
    # across the periodic boundary: 0 at x = -4.9, 1 at x = 4.7 -> bond 0->1 = (-0.4, 0)
    # -> bin (1, 2); bond 1->0 = (0.4, 0) -> bin (2, 2)
    x = np.array([[-4.9, 0.1, 0.0], [4.7, 0.1, 0.0]], np.float32)
    c, xy, qi, pj = oracle.pmftxy(b, x, np.zeros(2, np.float32), 1.0, 1.0, 4, 4, with_xy=True)
    e0 = int(np.flatnonzero(qi == 0)[0])
    assert xy[e0, 0] == pytest.approx(-0.4, abs=1e-6) and xy[e0, 1] == pytest.approx(0.0, abs=1e-7)
    assert c[1, 2] == 1 and c[2, 2] == 1 and c.sum() == 2


def _numpy_pmft(b, x, theta, x_max, y_max, bx, by):
    """Histogram2d of every ordered pair's nearest-image bond turned by -theta_i."""
    v = image_vectors_2d(b, x, x)
    n = len(x)
    i, j = np.nonzero(~np.eye(n, dtype=bool))
    d = v[i, j]
    c, s = np.cos(theta[i].astype(np.float64)), np.sin(theta[i].astype(np.float64))
    xr = c * d[:, 0] + s * d[:, 1]
    yr = c * d[:, 1] - s * d[:, 0]
    ex = np.linspace(-x_max, x_max, bx + 1)
    ey = np.linspace(-y_max, y_max, by + 1)
    # bonds within 1e-9 of an edge could fall either way between two FP64 evaluations
    gap = min(np.abs(xr[:, None] - ex[None]).min(), np.abs(yr[:, None] - ey[None]).min())
    inside = (xr >= -x_max) & (xr < x_max) & (yr >= -y_max) & (yr < y_max)
    h = np.histogram2d(xr[inside], yr[inside], bins=[ex, ey])[0].astype(np.int64)
    return h, gap


@pytest.mark.parametrize("bi", range(len(BOXES2)))
@pytest.mark.parametrize("orient", ["zero", "same", "random"])
def test_pmft_against_numpy_histogram2d(bi, orient):
    b = BOXES2[bi]
    rng = np.random.default_rng(350 + bi)
    n = 700
    x = W.uniform_points(rng, b, n)
    theta = {"zero": np.zeros(n), "same": np.full(n, 0.7),
             "random": rng.uniform(-np.pi, np.pi, n)}[orient].astype(np.float32)
    x_max, y_max, bx, by = 2.0, 1.5, 16, 9
    want, gap = _numpy_pmft(b, x, theta, x_max, y_max, bx, by)
    assert gap > 1e-9
    got = oracle.pmftxy(b, x, theta, x_max, y_max, bx, by)
    assert np.array_equal(got, want)
    if orient == "zero":  # bond j->i is minus bond i->j: point symmetry of the histogram
        assert np.array_equal(got, got[::-1, ::-1])


def test_pmft_frame_rotation_and_explicit_list():
    # turning the whole square system by 90 degrees and every orientation by 90 degrees
    # leaves every bond's local coordinates unchanged
    b = W.Box.square(11.0)
    rng = np.random.default_rng(360)
    x = W.uniform_points(rng, b, 500)
    theta = rng.uniform(-np.pi, np.pi, 500).astype(np.float32)
    xr = np.stack([-x[:, 1], x[:, 0], x[:, 2]], 1).astype(np.float32)
    _, xy1, qi1, pj1 = oracle.pmftxy(b, x, theta, 1.5, 1.5, 10, 10, with_xy=True)
    _, xy2, qi2, pj2 = oracle.pmftxy(b, xr, (theta + np.float32(np.pi / 2)).astype(np.float32), 1.5, 1.5, 10, 10,
                                     with_xy=True)
    assert np.array_equal(qi1, qi2) and np.array_equal(pj1, pj2)
    assert np.allclose(xy1, xy2, atol=2e-5)
    # an explicit list gives the same counts as the default query; bonds outside the
    # square are dropped
    _, off, pj, _ = oracle.ball_query(b, x, 3.0)
    c_list = oracle.pmftxy(b, x, theta, 1.5, 1.5, 10, 10, qi=_qi(off), pj=pj)
    assert np.array_equal(c_list, oracle.pmftxy(b, x, theta, 1.5, 1.5, 10, 10))


def test_pmft_query_points_and_ideal_gas():
    f = W.p6(seed=370, n=20000, n_frames=1)[0]
    p = W.P6_PARAMS
    c = oracle.pmftxy(f.box, f.points, f.theta, 1.0, 1.0, 20, 20)
    n = len(f.points)
    pcf, pmft = oracle.pmft_normalize(c, n * n / f.box.area, 1.0, 1.0)
    expect = n * (n - 1) / f.box.area * (0.1 * 0.1)
    assert np.all(np.abs(pcf - (1.0 - 1.0 / n)) < 5.0 * np.sqrt(1.0 / expect))
    assert np.allclose(pmft, -np.log(pcf))
    # other query points: no exclusion, orientation per query point
    q = f.points[:300] + np.float32(0.01)
    q[:, 2] = 0.0
    th = f.theta[:300]
    cq, xy, qi, pj = oracle.pmftxy(f.box, f.points, th, 1.0, 1.0, 20, 20, query_points=q, with_xy=True)
    v = image_vectors_2d(f.box, q, f.points)[qi, pj]
    cs, sn = np.cos(th[qi].astype(np.float64)), np.sin(th[qi].astype(np.float64))
    assert np.allclose(xy[:, 0], cs * v[:, 0] + sn * v[:, 1], atol=1e-12)
    assert np.allclose(xy[:, 1], cs * v[:, 1] - sn * v[:, 0], atol=1e-12)
    assert cq.sum() == np.count_nonzero((np.abs(xy[:, 0]) < 1.0) & (np.abs(xy[:, 1]) < 1.0))
    assert p["bins_x"] == 100
