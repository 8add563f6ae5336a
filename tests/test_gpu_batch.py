"""Batched frames (persistent launches, CUDA-graph replay, autotuner) against the oracle
frame by frame: RDF counts bit-exact, q_l within 1e-5 * max(q, 1e-2), on both routes
(cell-tile kernels and the per-point kernel)."""
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


@pytest.fixture(scope="module")
def frames():
    fr = W.c5(seed=11, n_frames=10, n_lo=600, n_hi=5000)
    P = W.C5_PARAMS
    refs = []
    for f in fr:
        counts = oracle.rdf_counts(f.box, f.points, P["rdf_bins"], P["rdf_r_max"])
        _, off, pj, _ = oracle.ball_query(f.box, f.points, P["r_max"])
        q = oracle.steinhardt(f.box, f.points, off, pj, P["l"])
        refs.append((counts, q, np.diff(off)))
    return fr, refs


def check(b, fr, refs):
    counts, q, nn = (t.cpu().numpy() for t in b.outputs())
    off = b.offsets
    for k, (c_ref, q_ref, nn_ref) in enumerate(refs):
        assert np.array_equal(counts[k].astype(np.uint64), c_ref), f"frame {k} RDF counts"
        qk = q[off[k]:off[k + 1]]
        assert np.all(np.abs(qk - q_ref) <= 1e-5 * np.maximum(q_ref, 1e-2)), f"frame {k} q_l"
        assert np.array_equal(nn[off[k]:off[k + 1]], nn_ref)


# (cell_div, block, hist_copies, tile_cells, cells_per_warp, route): tile_cells -1 puts
# every frame on the per-point kernel; cell_div 2 makes the RDF half stencil too wide for
# the tile kernels; tile_cells 1 gives one-cell work items; cells_per_warp 2, 4 and 8 walk
# blocks of x-adjacent query cells (shortened at row and work-item ends; frames too narrow
# take smaller blocks)
@pytest.mark.parametrize("cell_div,block,copies,tile,qb,route", [
    (1, 128, 2, -1, 1, "per_point"), (2, 64, 1, 0, 1, "per_point"), (1, 256, 4, 0, 1, "tile"),
    (1, 128, 2, 1, 1, "tile"), (1, 128, 2, 0, 2, "tile"), (1, 128, 2, 0, 4, "tile"), (1, 128, 2, 3, 4, "tile"),
    (1, 128, 2, 0, 8, "tile")])
def test_batch_matches_oracle(fgb, frames, cell_div, block, copies, tile, qb, route):
    fr, refs = frames
    P = W.C5_PARAMS
    pts = torch.from_numpy(np.concatenate([f.points for f in fr])).cuda()
    b = fgb.Batch([len(f.points) for f in fr], [f.box for f in fr], r_max=P["r_max"], l=P["l"],
                  rdf_bins=P["rdf_bins"], rdf_r_max=P["rdf_r_max"], cell_div=cell_div, block=block,
                  hist_copies=copies, tile_cells=tile, cells_per_warp=qb)
    assert b.routes()[route] == len(fr)
    b.run(pts)
    torch.cuda.synchronize()
    check(b, fr, refs)


def test_batch_routes_agree(fgb, frames):
    # the same frames on both routes: identical RDF and neighbor counts, q_l to rounding
    fr, _ = frames
    P = W.C5_PARAMS
    pts = torch.from_numpy(np.concatenate([f.points for f in fr])).cuda()
    out = []
    for tile in (-1, 64):
        b = fgb.Batch([len(f.points) for f in fr], [f.box for f in fr], r_max=P["r_max"], l=P["l"],
                      rdf_bins=P["rdf_bins"], rdf_r_max=P["rdf_r_max"], cell_div=1, tile_cells=tile)
        b.run(pts)
        torch.cuda.synchronize()
        out.append([t.cpu().numpy() for t in b.outputs()])
    (c0, q0, n0), (c1, q1, n1) = out
    assert np.array_equal(c0, c1) and np.array_equal(n0, n1)
    assert np.all(np.abs(q0 - q1) <= 1e-5 * np.maximum(np.abs(q0), 1e-2))


@pytest.mark.parametrize("l,qb", [(4, 1), (12, 1), (6, 2)])
def test_batch_crowded_cells(fgb, l, qb):
    # about 40 points per cell (several query passes per cell in the tile kernels; blocks
    # of two cells: about 80 queries), one cubic and one triclinic frame, l with two
    # partial sums (4) and with one (12)
    rng = np.random.default_rng(21 + l)
    boxes = [W.Box.cube(8.0), W.Box(8.2, 8.0, 8.4, 0.1, -0.05, 0.08)]
    xs = [W.uniform_points(rng, boxes[0], 5000), W.uniform_points(rng, boxes[1], 5400)]
    P = W.C5_PARAMS
    refs = []
    for box, x in zip(boxes, xs):
        counts = oracle.rdf_counts(box, x, P["rdf_bins"], P["rdf_r_max"])
        _, off, pj, _ = oracle.ball_query(box, x, P["r_max"])
        refs.append((counts, oracle.steinhardt(box, x, off, pj, l), np.diff(off)))
    pts = torch.from_numpy(np.concatenate(xs)).cuda()
    b = fgb.Batch([len(x) for x in xs], boxes, r_max=P["r_max"], l=l, rdf_bins=P["rdf_bins"],
                  rdf_r_max=P["rdf_r_max"], cell_div=1, cells_per_warp=qb)
    assert b.routes()["tile"] == 2
    b.run(pts)
    torch.cuda.synchronize()
    check(b, None, refs)


def test_batch_graph_replay_and_tune(fgb, frames):
    fr, refs = frames
    P = W.C5_PARAMS
    pts = torch.from_numpy(np.concatenate([f.points for f in fr])).cuda()
    b = fgb.Batch([len(f.points) for f in fr], [f.box for f in fr], r_max=P["r_max"], l=P["l"],
                  rdf_bins=P["rdf_bins"], rdf_r_max=P["rdf_r_max"])
    chosen = b.tune(pts)
    assert chosen["cell_div"] in (1, 2) and chosen["block"] in (64, 128, 256) and chosen["tile_cells"] in (16, 64)
    assert chosen["cells_per_warp"] in (1, 2, 4, 8)
    for _ in range(3):
        b.run(pts, graph=True)
    torch.cuda.synchronize()
    check(b, fr, refs)
    # a new points buffer with the same contents recaptures and gives the same answer
    pts2 = pts.clone()
    b.run(pts2, graph=True)
    torch.cuda.synchronize()
    check(b, fr, refs)


def test_batch_rejects_small_boxes(fgb):
    box = W.Box.cube(5.0)
    with pytest.raises(fgb.FGBError) as e:
        fgb.Batch([10], [box], r_max=1.5, rdf_r_max=3.0)
    assert e.value.code == fgb.ERR_BOX_TOO_SMALL


def test_batch_mixes_2d_and_3d_frames(fgb):
    # 2D frames (Lz = 0) next to 3D ones in one persistent launch
    P = W.C5_PARAMS
    fr = W.c5(seed=12, n_frames=3, n_lo=800, n_hi=3000)
    flat = [(f.box, f.points) for f in fr]
    for k, n in enumerate((1500, 4000, 700)):
        g = W.p6(seed=40 + k, n=n, n_frames=1, neighbors=6.0, xy=0.1 * k)[0]
        flat.insert(2 * k, (g.box, g.points))
    refs = []
    for box, x in flat:
        counts = oracle.rdf_counts(box, x, P["rdf_bins"], P["rdf_r_max"])
        _, off, pj, _ = oracle.ball_query(box, x, P["r_max"])
        refs.append((counts, oracle.steinhardt(box, x, off, pj, P["l"]), np.diff(off)))
    pts = torch.from_numpy(np.concatenate([x for _, x in flat])).cuda()
    b = fgb.Batch([len(x) for _, x in flat], [box for box, _ in flat], r_max=P["r_max"], l=P["l"],
                  rdf_bins=P["rdf_bins"], rdf_r_max=P["rdf_r_max"])
    b.run(pts)
    torch.cuda.synchronize()
    check(b, None, refs)


def test_full_c5_batch_sampled(fgb):
    # the 256-frame workload in the bench's launch configuration (autotuned, graph
    # replay); the smallest, median and largest frames and two more against the oracle,
    # and for every frame the symmetry of a self query: an even total of ordered RDF
    # pairs and of neighbor counts
    fr = W.c5()
    P = W.C5_PARAMS
    sizes = np.array([len(f.points) for f in fr])
    pts = torch.from_numpy(np.concatenate([f.points for f in fr])).cuda()
    b = fgb.Batch(sizes.tolist(), [f.box for f in fr], r_max=P["r_max"], l=P["l"], rdf_bins=P["rdf_bins"],
                  rdf_r_max=P["rdf_r_max"])
    b.tune(pts)
    b.run(pts, graph=True)
    b.run(pts, graph=True)
    torch.cuda.synchronize()
    counts, q, nn = (t.cpu().numpy() for t in b.outputs())
    off = b.offsets
    order = np.argsort(sizes, kind="stable")
    rng = np.random.default_rng(55)
    picks = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1]),
                    *rng.choice(len(fr), 2, replace=False).tolist()})
    for k in picks:
        f = fr[k]
        c_ref = oracle.rdf_counts(f.box, f.points, P["rdf_bins"], P["rdf_r_max"])
        _, o, pj, _ = oracle.ball_query(f.box, f.points, P["r_max"])
        q_ref = oracle.steinhardt(f.box, f.points, o, pj, P["l"])
        assert np.array_equal(counts[k].astype(np.uint64), c_ref), f"frame {k} RDF counts"
        qk = q[off[k]:off[k + 1]]
        assert np.all(np.abs(qk - q_ref) <= 1e-5 * np.maximum(q_ref, 1e-2)), f"frame {k} q_l"
        assert np.array_equal(nn[off[k]:off[k + 1]], np.diff(o)), f"frame {k} neighbor counts"
    for k in range(len(fr)):
        assert int(counts[k].sum()) % 2 == 0 and int(nn[off[k]:off[k + 1]].sum()) % 2 == 0, f"frame {k}"
