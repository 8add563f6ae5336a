"""The allocation-free RDF entry point (fgb_rdf_noalloc), called through the C ABI, gives
the same counts as the allocating fgb_rdf_compute path.

It exists for callers that cannot allocate device memory while they run (simulation
steps with a fixed memory budget, runtimes whose own pool owns the device); its working
set is one static device array.  Two calls in a row on different frames check that
nothing stale from the previous call leaks into the next; the second frame is also
compared with the FP64 oracle directly.  This file is collected last so a
stop-at-first-failure run has already run every other test."""
import ctypes

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


def noalloc_counts(fgb, box, pts, bins, r_max, r_min):
    out = torch.zeros(bins, dtype=torch.int64, device="cuda")
    b = fgb.Box.from_box(box)._c()
    code = fgb.lib().fgb_rdf_noalloc(ctypes.byref(b), pts.data_ptr(), pts.shape[0], bins, r_max, r_min,
                                     out.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    fgb._check(code)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.uint64)


def allocating_counts(fgb, box, pts, bins, r_max, r_min):
    rdf = fgb.RDF(bins, r_max, r_min)
    rdf.compute(fgb.NeighborQuery(box, pts, r_cell=r_max), reset=True)
    return rdf.bin_counts


def test_noalloc_matches_allocating_path_twice(fgb):
    frames = [
        (W.Box(20.0, 21.0, 19.0, 0.1, -0.05, 0.2), W.small_random(71, 30000, W.Box(20.0, 21.0, 19.0, 0.1, -0.05, 0.2)),
         300, 4.0, 0.0),
        (W.Box.cube(24.0), W.small_random(72, 12000, W.Box.cube(24.0)), 97, 5.5, 0.3),
    ]
    for k, (box, x, bins, r_max, r_min) in enumerate(frames):
        pts = torch.from_numpy(x).cuda()
        got = noalloc_counts(fgb, box, pts, bins, r_max, r_min)
        want = allocating_counts(fgb, box, pts, bins, r_max, r_min)
        assert np.array_equal(got, want)
        assert got.sum() > 0
        if k == 1:
            assert np.array_equal(got, oracle.rdf_counts(box, x, bins, r_max, r_min))


def test_noalloc_rejects_sizes_beyond_its_limit(fgb):
    box = W.Box.cube(100.0)
    big = torch.zeros((262145, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(fgb.FGBError) as e:
        noalloc_counts(fgb, box, big, 10, 2.0, 0.0)
    assert e.value.code == fgb.ERR_CAPACITY
    small = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(fgb.FGBError) as e:
        noalloc_counts(fgb, box, small, 8193, 2.0, 0.0)
    assert e.value.code == fgb.ERR_CAPACITY


def test_noalloc_2d_frame_and_general_stencil(fgb):
    # a 2D frame (its points on the z = 0 layer) and a box too small for the 27-cell
    # shift stencil (two cells per axis, so the library takes its general stencil
    # route), each compared with the allocating path and the oracle
    sq = W.Box.square(30.0, 0.1)
    x2 = W.small_random(73, 9000, sq)
    small = W.Box.cube(9.0)
    xs = W.small_random(74, 2500, small)
    for box, x, bins, r_max in ((sq, x2, 120, 6.0), (small, xs, 50, 4.0)):
        pts = torch.from_numpy(x).cuda()
        got = noalloc_counts(fgb, box, pts, bins, r_max, 0.0)
        assert np.array_equal(got, allocating_counts(fgb, box, pts, bins, r_max, 0.0))
        assert np.array_equal(got, oracle.rdf_counts(box, x, bins, r_max, 0.0))
        assert got.sum() > 0
