"""Single-reference MVS (through the C ABI) against the oracle (Sec. III-A, Eq. 4): census codes,
plane maps, cost volume, SGM aggregate, kept flags, depths and fused points bit-exact (integer
work, and floating point whose every operation is prescribed on both sides); the depth range and
the reference choice exact, Eq. 4 scores to 1e-12 (libm functions); ragged sizes, plane counts
that do not fill a warp, the widest plane count, and the error paths."""
import numpy as np
import pytest

from oracle import mvs as M
from paper_2601_17354_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2601_17354_gb300 import mvs
    return mvs


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _check_view(V, sc, target, D, full=True):
    cams = sc.cameras
    W, H = cams[target].width, cams[target].height
    mv = V.MultiViewStereo(W, H, D)
    pts = _cuda(sc.sparse.astype(np.float32))
    d_min, d_max, med = mv.depth_range(cams[target], pts)
    o_min, o_max, o_med = M.depth_range(sc.sparse.astype(np.float32), cams[target])
    assert (d_min, d_max, med) == (o_min, o_max, o_med)
    ref, scores = mv.select_reference(cams, target, med)
    o_scores = M.reference_scores(cams, target, o_med)
    assert ref == int(np.argmax(o_scores))
    fin = np.isfinite(o_scores)
    assert np.array_equal(np.isfinite(scores), fin)
    assert np.allclose(scores[fin], o_scores[fin], rtol=1e-12, atol=0)
    img_t, img_r = _cuda(sc.images[target]), _cuda(sc.images[ref])
    depth, kept = mv.depth(cams[target], cams[ref], img_t, img_r, d_min, d_max)
    torch.cuda.synchronize()
    inv_far, step = M.inverse_depths(o_min, o_max, D)
    cen_t, cen_r = M.census(M.luma(sc.images[target])), M.census(M.luma(sc.images[ref]))
    assert np.array_equal(_u64(mv.read(0)), cen_t)
    assert np.array_equal(_u64(mv.read(1)), cen_r)
    maps = M.plane_maps(cams[target], cams[ref], inv_far, step, D)
    assert np.array_equal(mv.read(4).cpu().numpy(), maps)
    C = M.cost_volume(cen_t, cen_r, maps)
    assert np.array_equal(mv.read(2).cpu().numpy(), C)
    Sv = M.sgm(C)
    assert np.array_equal(mv.read(3).cpu().numpy().view(np.uint16), Sv)
    k1, o_kept, o_depth = M.select_depth(Sv, inv_far, step)
    g = depth.cpu().numpy()
    assert kept == int(o_kept.sum())
    assert np.array_equal(np.isfinite(g), o_kept)
    assert np.array_equal(g[o_kept], o_depth[o_kept])
    pts_g, pix_g = mv.fuse(cams[target], depth)
    P, idx = M.back_project(o_depth, cams[target])
    assert np.array_equal(pix_g.cpu().numpy(), idx)
    assert np.array_equal(pts_g.cpu().numpy(), P)
    return mv, o_kept, g


def test_full_size_keyframe_bit_exact(V):
    sc = S.mvs_scene(3, views=[3, 4, 5])
    _, kept, depth = _check_view(V, sc, 4, 64)
    gt = sc.depths[4]
    fg = kept & np.isfinite(gt)
    rel = np.abs(depth[fg] - gt[fg]) / gt[fg]
    assert np.median(rel) < 0.01 and (rel < 0.02).mean() > 0.9


@pytest.mark.parametrize("D", [3, 40, 128])
def test_ragged_sizes_and_plane_counts(V, D):
    sc = S.mvs_scene(8, n_cameras=24, width=77, height=45, focal=60.0, n_sparse=3000, views=[9, 10, 11])
    _check_view(V, sc, 10, D)


def test_errors_and_capacity(V):
    from paper_2601_17354_gb300 import _lib as L
    sc = S.mvs_scene(9, n_cameras=16, width=96, height=64, focal=75.0, n_sparse=2000, views=[2, 3])
    mv = V.MultiViewStereo(96, 64, 32)
    cam = sc.cameras[2]
    far = _cuda(np.array([[100.0, 100.0, 100.0]], np.float32))          # behind / outside every view
    with pytest.raises(L.PgsError) as e:
        mv.depth_range(cam, far)
    assert e.value.code == L.PGS_ERR_INVALID_ARG
    img = _cuda(sc.images[2])
    with pytest.raises(L.PgsError):
        mv.depth(cam, sc.cameras[3], img, img, 0.0, 5.0)                 # d_min must be positive
    with pytest.raises(ValueError):
        mv.depth(cam, sc.cameras[3], img[:, :32], img, 1.0, 5.0)         # wrong image size
    d_min, d_max, _ = mv.depth_range(cam, _cuda(sc.sparse.astype(np.float32)))
    depth, kept = mv.depth(cam, sc.cameras[3], img, _cuda(sc.images[3]), d_min, d_max)
    assert kept > 10
    with pytest.raises(L.PgsError) as e:
        mv.fuse(cam, depth, capacity=5)
    assert e.value.code == L.PGS_ERR_CAPACITY
    pts, pix = mv.fuse(cam, depth)
    assert len(pix) == kept
