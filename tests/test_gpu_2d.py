"""GPU parity for 2D boxes (Lz = 0) and PMFT(x, y), through the C ABI, against the oracle.

Neighbor sets, their order, RDF counts and PMFT counts must match bit for bit; stored
float32 distances within 2e-6 relative; q_l within 1e-5 * max(q_ref, 1e-2).  The PMFT
decides every bond in FP64; its inputs are drawn so that no bond lies within 1e-9 of a
bin edge (checked from the oracle's rotated bonds), where two FP64 evaluations of
cos/sin (the device's and the host library's) could disagree in the last bit.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOXES2 = [W.Box.square(30.0), W.Box(28.0, 24.0, 0.0, 0.3), W.Box(25.0, 31.0, 0.0, -0.25)]


@pytest.fixture(scope="module")
def fgb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_06317_gb300 as m
    m.lib()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def pts2d(seed, n, b):
    x = W.small_random(seed, n, b)
    assert np.all(x[:, 2] == 0.0)
    return x


def assert_ball(nl, b, x, r):
    _, off, pj, dist = oracle.ball_query(b, x, r)
    assert np.array_equal(nl.segments.cpu().numpy(), off), "segments differ"
    assert np.array_equal(nl.point_indices.cpu().numpy(), pj), "point indices differ"
    assert np.array_equal(nl.query_point_indices.cpu().numpy(), np.repeat(np.arange(len(off) - 1), np.diff(off))), \
        "query indices differ"
    assert np.all(np.abs(nl.distances.cpu().numpy() - dist) <= 2e-6 * r + 1e-7), "distances differ"


# --------------------------------------------------------------------- 2D boxes


@pytest.mark.parametrize("bi", range(len(BOXES2)))
@pytest.mark.parametrize("r", [1.0, 2.5])
def test_2d_ball_matches_oracle(fgb, bi, r):
    b = BOXES2[bi]
    x = pts2d(400 + bi, 6000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=r)
    assert nq.cell_dims()[2] == 3
    assert_ball(nq.query(None, dict(r_max=r, exclude_ii=True)).toNeighborList(), b, x, r)
    # a wider query on the same grid, and other query points (no exclusion)
    assert_ball(nq.query(None, dict(r_max=1.6 * r, exclude_ii=True)).toNeighborList(), b, x, 1.6 * r)
    q = pts2d(410 + bi, 500, b)
    nl = nq.query(dev(q), dict(r_max=r)).toNeighborList()
    _, off, pj, _ = oracle.ball_query(b, x, r, exclude_ii=False, query_points=q)
    assert np.array_equal(nl.segments.cpu().numpy(), off)
    assert np.array_equal(nl.point_indices.cpu().numpy(), pj)


@pytest.mark.parametrize("bi", [0, 1])
@pytest.mark.parametrize("k", [1, 6, 12])
def test_2d_knn_matches_oracle(fgb, bi, k):
    b = BOXES2[bi]
    x = pts2d(420 + bi, 5000, b)
    nl = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(num_neighbors=k, exclude_ii=True)).toNeighborList()
    n, j, d = oracle.knn(b, x, k)
    assert np.array_equal(nl.point_indices.cpu().numpy().reshape(-1, k), j[:, :k])
    assert np.allclose(nl.distances.cpu().numpy().reshape(-1, k), d[:, :k], rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("bi", range(len(BOXES2)))
def test_2d_rdf_matches_oracle(fgb, bi):
    b = BOXES2[bi]
    x = pts2d(430 + bi, 8000, b)
    for bins, r, rc in ((100, 5.0, 5.0), (300, 3.0, 1.0)):
        h = fgb.RDF(bins, r)
        h.compute(fgb.NeighborQuery(b, dev(x), r_cell=rc))
        c = oracle.rdf_counts(b, x, bins, r)
        assert np.array_equal(h.bin_counts, c)
        g, centers = oracle.rdf_normalize(c, len(x), len(x), b.area, bins, 0.0, r, dim=2)
        assert np.allclose(h.rdf, g, rtol=1e-12, atol=0)
        assert np.allclose(h.bin_centers, centers)


def test_2d_rdf_frames_share_a_dimension(fgb):
    b2, b3 = BOXES2[0], W.Box.cube(12.0)
    h = fgb.RDF(50, 2.0)
    h.compute(fgb.NeighborQuery(b2, dev(pts2d(440, 3000, b2)), r_cell=2.0))
    with pytest.raises(fgb.FGBError) as e:
        h.compute(fgb.NeighborQuery(b3, dev(W.small_random(441, 3000, b3)), r_cell=2.0), reset=False)
    assert e.value.code == fgb.ERR_INVALID_ARG
    h.compute(fgb.NeighborQuery(b3, dev(W.small_random(441, 3000, b3)), r_cell=2.0), reset=True)


def test_2d_steinhardt_and_tree(fgb):
    b = BOXES2[1]
    x = pts2d(450, 6000, b)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.5)
    nl = nq.query(None, dict(r_max=1.5, exclude_ii=True)).toNeighborList()
    _, off, pj, _ = oracle.ball_query(b, x, 1.5)
    for l in (4, 6):
        st = fgb.Steinhardt(l)
        st.compute(nq, neighbors=nl)
        q_ref = oracle.steinhardt(b, x, off, pj, l)
        q = st.particle_order.cpu().numpy()
        assert np.all(np.abs(q - q_ref) <= 1e-5 * np.maximum(q_ref, 1e-2))
    tree = fgb.AABBQuery(b, dev(x))
    assert_ball(tree.query(None, dict(r_max=1.5, exclude_ii=True)).toNeighborList(), b, x, 1.5)
    kn = tree.query(None, dict(num_neighbors=8, exclude_ii=True)).toNeighborList()
    _, j, _ = oracle.knn(b, x, 8)
    assert np.array_equal(kn.point_indices.cpu().numpy().reshape(-1, 8), j[:, :8])


def test_2d_box_rules(fgb):
    x = dev(np.zeros((4, 3), np.float32))
    with pytest.raises(fgb.FGBError) as e:
        fgb.NeighborQuery(W.Box(10.0, 10.0, 0.0, 0.0, 0.1, 0.0), x, 1.0)
    assert e.value.code == fgb.ERR_INVALID_ARG
    b = W.Box(20.0, 6.0, 0.0, 0.0)           # in-plane width 6: r_max must stay below 3
    nq = fgb.NeighborQuery(b, dev(pts2d(460, 500, b)), 1.0)
    nq.query(None, dict(r_max=2.9, exclude_ii=True)).toNeighborList()
    with pytest.raises(fgb.FGBError) as e:
        nq.query(None, dict(r_max=3.1, exclude_ii=True)).toNeighborList()
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL


# ------------------------------------------------------------------------- PMFT


def pmft_ref(b, x, theta, x_max, y_max, bx, by, **kw):
    c, xy, qi, pj = oracle.pmftxy(b, x, theta, x_max, y_max, bx, by, with_xy=True, **kw)
    ex = np.linspace(-x_max, x_max, bx + 1)
    ey = np.linspace(-y_max, y_max, by + 1)
    # theta = 0 turns nothing (cos 1, sin 0 exactly): such bonds may sit on an edge
    xy = xy[theta[qi] != 0]
    gap = min(np.abs(xy[:, :1] - ex[None]).min(), np.abs(xy[:, 1:] - ey[None]).min()) if len(xy) else 1.0
    assert gap > 1e-9, "an input bond sits on a bin edge; pick another seed"
    return c, qi, pj


@pytest.mark.parametrize("bi", range(len(BOXES2)))
@pytest.mark.parametrize("orient", ["zero", "random"])
def test_pmft_self_matches_oracle(fgb, bi, orient):
    b = BOXES2[bi]
    rng = np.random.default_rng(500 + bi)
    x = pts2d(500 + bi, 6000, b)
    th = (np.zeros(6000) if orient == "zero" else rng.uniform(-np.pi, np.pi, 6000)).astype(np.float32)
    x_max, y_max, bx, by = 2.0, 1.5, 40, 30
    want, _, _ = pmft_ref(b, x, th, x_max, y_max, bx, by)
    p = fgb.PMFTXY(x_max, y_max, (bx, by))
    p.compute((b, dev(x)), dev(th))
    got = p.bin_counts
    assert np.array_equal(got, want.astype(np.uint64))
    n = len(x)
    pcf, pm = oracle.pmft_normalize(want, n * n / b.area, x_max, y_max)
    assert np.allclose(p.pcf, pcf, rtol=1e-12, atol=0)
    assert np.array_equal(np.isinf(p.pmft), np.isinf(pm))
    fin = np.isfinite(pm)
    assert np.allclose(p.pmft[fin], pm[fin], rtol=1e-12, atol=1e-12)


def test_pmft_lists_query_points_and_tree(fgb):
    b = BOXES2[1]
    rng = np.random.default_rng(510)
    x = pts2d(510, 7000, b)
    th = rng.uniform(-np.pi, np.pi, 7000).astype(np.float32)
    want, _, _ = pmft_ref(b, x, th, 1.2, 2.0, 24, 20)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.0)
    # a wider list than needed: bonds outside the rectangle are dropped
    nl = nq.query(None, dict(r_max=3.0, exclude_ii=True)).toNeighborList()
    p = fgb.PMFTXY(1.2, 2.0, (24, 20))
    p.compute(nq, dev(th), neighbors=nl)
    assert np.array_equal(p.bin_counts, want.astype(np.uint64))
    tree = fgb.AABBQuery(b, dev(x))
    p.compute(tree, dev(th))
    assert np.array_equal(p.bin_counts, want.astype(np.uint64))
    # other query points with their own orientations (no exclusion)
    q = pts2d(511, 900, b)
    tq = rng.uniform(-np.pi, np.pi, 900).astype(np.float32)
    wq, _, _ = pmft_ref(b, x, tq, 1.2, 2.0, 24, 20, query_points=q)
    p.compute(nq, dev(tq), query_points=dev(q))
    assert np.array_equal(p.bin_counts, wq.astype(np.uint64))


def test_pmft_accumulates_fig6_frames(fgb):
    frames = W.p6(seed=520, n=20000, n_frames=3)
    prm = W.P6_PARAMS
    x_max, y_max, bx, by = prm["x_max"], prm["y_max"], prm["bins_x"], prm["bins_y"]
    p = fgb.PMFTXY(x_max, y_max, (bx, by))
    total = np.zeros((bx, by), np.int64)
    for k, f in enumerate(frames):
        c, _, _ = pmft_ref(f.box, f.points, f.theta, x_max, y_max, bx, by)
        total += c
        p.compute((f.box, dev(f.points)), dev(f.theta), reset=(k == 0))
    assert np.array_equal(p.bin_counts, total.astype(np.uint64))
    n = 20000
    pcf, _ = oracle.pmft_normalize(total, 3 * n * n / frames[0].box.area, x_max, y_max)
    assert np.allclose(p.pcf, pcf, rtol=1e-12, atol=0)
    assert np.array_equal(p.counts_device().cpu().numpy(), total)


def test_pmft_fused_edges_escalate(fgb):
    # square lattice of spacing 0.5 with theta = 0 and bins of 0.5: every bond lies on a
    # bin edge, so the fused kernel must leave them to its FP64 pass
    g = np.arange(80) * 0.5 - 20.0
    x = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    x = np.concatenate([x, np.zeros((len(x), 1))], 1).astype(np.float32)
    b = W.Box.square(40.0)
    th = np.zeros(len(x), np.float32)
    p = fgb.PMFTXY(1.5, 1.5, 6)
    p.compute((b, dev(x)), dev(th))
    assert p.escalations() > 0
    assert np.array_equal(p.bin_counts, oracle.pmftxy(b, x, th, 1.5, 1.5, 6, 6).astype(np.uint64))
    # the list route on the same bonds (FP32 binning, FP64 for bonds near an edge)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=2.2)
    nl = nq.query(None, dict(r_max=2.2, exclude_ii=True)).toNeighborList()
    p.compute(nq, dev(th), neighbors=nl)
    assert np.array_equal(p.bin_counts, oracle.pmftxy(b, x, th, 1.5, 1.5, 6, 6).astype(np.uint64))
    # the same lattice turned by 90 degrees per particle: cos is -4.4e-8, not 0
    th = np.full(len(x), np.pi / 2, np.float32)
    p.compute((b, dev(x)), dev(th))
    want = oracle.pmftxy(b, x, th, 1.5, 1.5, 6, 6).astype(np.uint64)
    assert np.array_equal(p.bin_counts, want)
    p.compute(nq, dev(th), neighbors=nl)
    assert np.array_equal(p.bin_counts, want)


@pytest.mark.parametrize("bins", [(7, 3), (128, 128), (200, 100)])
def test_pmft_bin_counts_across_routes(fgb, bins):
    # the fused kernel keeps at most 16384 bins in shared memory; more take the list route
    f = W.p6(seed=525, n=20000, n_frames=1)[0]
    bx, by = bins
    want, _, _ = pmft_ref(f.box, f.points, f.theta, 1.3, 0.9, bx, by)
    p = fgb.PMFTXY(1.3, 0.9, bins)
    p.compute((f.box, dev(f.points)), dev(f.theta))
    assert np.array_equal(p.bin_counts, want.astype(np.uint64))


def test_pmft_dense_cluster(fgb):
    # thousands of points in a few cells next to a uniform background: long candidate
    # streams per cell, heavy contention on the shared counts, and (angles 0) many bonds
    # exactly on bin edges from the duplicated float32 coordinates
    b = W.Box.square(60.0)
    rng = np.random.default_rng(535)
    bg = W.uniform_points(rng, b, 12000)
    cl = np.zeros((4000, 3), np.float32)
    cl[:, :2] = (rng.random((4000, 2)) * 1.6 - 0.8).astype(np.float32)
    x = np.concatenate([bg, cl]).astype(np.float32)
    th = np.zeros(len(x), np.float32)
    p = fgb.PMFTXY(1.0, 1.0, 40)
    p.compute((b, dev(x)), dev(th))
    want = oracle.pmftxy(b, x, th, 1.0, 1.0, 40, 40).astype(np.uint64)
    assert np.array_equal(p.bin_counts, want)
    nq = fgb.NeighborQuery(b, dev(x), r_cell=1.5)
    p.compute(nq, dev(th), neighbors=nq.query(None, dict(r_max=1.5, exclude_ii=True)).toNeighborList())
    assert np.array_equal(p.bin_counts, want)


def test_pmft_errors_and_empty(fgb):
    b3 = W.Box.cube(12.0)
    x3 = dev(W.small_random(530, 100, b3))
    p = fgb.PMFTXY(1.0, 1.0, 10)
    with pytest.raises(fgb.FGBError) as e:
        p.compute((b3, x3), dev(np.zeros(100, np.float32)))
    assert e.value.code == fgb.ERR_INVALID_ARG
    b = W.Box.square(5.0)
    with pytest.raises(fgb.FGBError) as e:
        fgb.PMFTXY(2.0, 2.0, 10).compute((b, dev(pts2d(531, 50, b))), dev(np.zeros(50, np.float32)))
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL
    with pytest.raises(fgb.FGBError) as e:
        fgb.PMFTXY(0.0, 1.0, 10)
    assert e.value.code == fgb.ERR_INVALID_ARG
    one = dev(np.zeros((1, 3), np.float32))
    p.compute((b, one), dev(np.zeros(1, np.float32)))
    assert p.bin_counts.sum() == 0 and np.all(np.isinf(p.pmft))


# Small 2D grids run one thread per query by default and large ones the cell-tile
# kernels; each switch forces one family.
SWITCH_CHECKS_2D = r"""
import numpy as np, torch, oracle, workloads as W, paper_1906_06317_gb300 as fgb
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
for b in (W.Box.square(30.0), W.Box(28.0, 24.0, 0.0, 0.3)):
    x = W.small_random(540, 6000, b)
    for r in (1.0, 2.2):
        nl = fgb.NeighborQuery(b, dev(x), r_cell=r).query(None, dict(r_max=r, exclude_ii=True)).toNeighborList()
        _, off, pj, _ = oracle.ball_query(b, x, r)
        assert np.array_equal(nl.segments.cpu().numpy(), off)
        assert np.array_equal(nl.point_indices.cpu().numpy(), pj)
        assert np.array_equal(nl.query_point_indices.cpu().numpy(), np.repeat(np.arange(len(off) - 1), np.diff(off)))
        h = fgb.RDF(120, r); h.compute(fgb.NeighborQuery(b, dev(x), r_cell=r))
        assert np.array_equal(h.bin_counts, oracle.rdf_counts(b, x, 120, r))
    k = fgb.NeighborQuery(b, dev(x), r_cell=1.0).query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
    _, kj, _ = oracle.knn(b, x, 12)
    assert np.array_equal(k.point_indices.cpu().numpy().reshape(-1, 12), kj[:, :12])
    th = np.random.default_rng(541).uniform(-np.pi, np.pi, 6000).astype(np.float32)
    p = fgb.PMFTXY(1.5, 1.5, 30); p.compute((b, dev(x)), dev(th))
    assert np.array_equal(p.bin_counts, oracle.pmftxy(b, x, th, 1.5, 1.5, 30, 30).astype(np.uint64))
print('ok')
"""


@pytest.mark.parametrize("switch", ["FGB_THREAD_KERNELS", "FGB_TILE_KERNELS"])
def test_2d_kernel_family_switches(switch):
    import os
    import subprocess
    import sys
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    env[switch] = "1"
    r = subprocess.run([sys.executable, "-c", SWITCH_CHECKS_2D], env=env, cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
