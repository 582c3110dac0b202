"""Union of cell bounds (ar_bounds_union) and the partitioned render
(ar_render_abstract_partitioned) on the GPU: the union is bit-exact against
numpy's elementwise min / max; the partitioned render equals the union of
ar_render_abstract over the same pieces bit for bit, matches the oracle's
union within the parity tolerance of test_gpu_parity, and is sound."""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def arlib():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    assert torch.cuda.is_available()
    return ar


@pytest.mark.parametrize("nc,W,H", [(5, 7, 5), (3, 8, 6), (1, 16, 9), (70, 33, 17)])
def test_union_matches_numpy(arlib, nc, W, H):
    ar = arlib
    g = torch.Generator().manual_seed(nc * 1000 + W)
    lo = torch.rand((nc, H, W, 3), generator=g).cuda()
    hi = lo + torch.rand((nc, H, W, 3), generator=g).cuda()
    olo = torch.full((H, W, 3), -1.0, device="cuda")
    ohi = torch.full_like(olo, -1.0)
    ar.ar_bounds_union(lo, hi, nc, W, H, olo, ohi)
    torch.cuda.synchronize()
    assert np.array_equal(olo.cpu().numpy(), lo.cpu().numpy().min(axis=0))
    assert np.array_equal(ohi.cpu().numpy(), hi.cpu().numpy().max(axis=0))


@pytest.mark.parametrize("W,H", [(8, 6), (7, 5)])   # the 16-byte and the one-float kernels
def test_union_propagates_nan(arlib, W, H):
    """A NaN bound of any piece (which would mean an unsound piece) reaches
    the joined image, as numpy's minimum / maximum let it, instead of being
    hidden by the other pieces' finite bounds."""
    ar = arlib
    nc = 3
    g = torch.Generator().manual_seed(5)
    lo = torch.rand((nc, H, W, 3), generator=g)
    hi = lo + torch.rand((nc, H, W, 3), generator=g)
    lo[1, 2, 3, 1] = float("nan")
    hi[2, 0, 1, 0] = float("nan")
    hi[0, 4, 4, 2] = float("nan")
    olo = torch.full((H, W, 3), -1.0, device="cuda")
    ohi = torch.full_like(olo, -1.0)
    ar.ar_bounds_union(lo.cuda(), hi.cuda(), nc, W, H, olo, ohi)
    torch.cuda.synchronize()
    want_lo, want_hi = np.minimum.reduce(lo.numpy()), np.maximum.reduce(hi.numpy())
    got_lo, got_hi = olo.cpu().numpy(), ohi.cpu().numpy()
    assert np.isnan(got_lo[2, 3, 1]) and np.isnan(got_hi[0, 1, 0]) and np.isnan(got_hi[4, 4, 2])
    assert np.array_equal(np.isnan(got_lo), np.isnan(want_lo)) and np.array_equal(np.isnan(got_hi), np.isnan(want_hi))
    f = ~np.isnan(want_lo)
    assert np.array_equal(got_lo[f], want_lo[f])
    f = ~np.isnan(want_hi)
    assert np.array_equal(got_hi[f], want_hi[f])


def test_union_rejects_bad_arguments(arlib):
    ar = arlib
    lo = torch.zeros((2, 4, 4, 3), device="cuda")
    hi = torch.zeros_like(lo)
    out = torch.zeros((4, 4, 3), device="cuda")
    with pytest.raises(ar.ArError):
        ar.ar_bounds_union(lo, hi, 0, 4, 4, out, out.clone())
    with pytest.raises(ar.ArError):
        ar.ar_bounds_union(lo, hi, 2, 4, 4, lo[1], out)          # output inside an input
    with pytest.raises(ar.ArError):
        ar.ar_bounds_union(lo, hi, 2, 4, 4, out, out)            # outputs overlap


def _scene():
    sc = synth.object_scene(1500, 6)
    cam = synth.look_camera(50, 38, 60.0, centre=(0, 0, -4))
    box_lo = np.array([-0.02, 0.0, -0.02, 0.0, -0.006, 0.0])
    return sc, cam, box_lo, -box_lo


@pytest.mark.parametrize("parts", [[2, 1, 2, 1, 1, 1], [4, 1, 4, 1, 5, 1]])   # 4 and 80 pieces (two chunks)
def test_partitioned_equals_union_of_pieces(arlib, orc, parts):
    ar = arlib
    sc, cam, box_lo, box_hi = _scene()
    s = ar.Scene(sc)
    intr, pose = ar.make_intrinsics(cam), ar.make_pose(cam)
    box = ar.make_cells(box_lo, box_hi)[0]
    plo = torch.full((cam.height, cam.width, 3), -7.0, device="cuda")
    phi = torch.full_like(plo, -7.0)
    ar.ar_render_abstract_partitioned(s.handle, intr, pose, box, parts, 16, plo, phi)
    # the same pieces through ar_render_abstract, joined by ar_bounds_union
    clo, chi = orc.partition_cells(box_lo, box_hi, parts)
    n = clo.shape[0]
    cells = ar.make_cells(clo, chi)
    a_lo = torch.empty((n, cam.height, cam.width, 3), device="cuda")
    a_hi = torch.empty_like(a_lo)
    ar.ar_render_abstract(s.handle, intr, pose, cells, n, 16, a_lo, a_hi)
    ulo = torch.empty_like(plo)
    uhi = torch.empty_like(plo)
    ar.ar_bounds_union(a_lo, a_hi, n, cam.width, cam.height, ulo, uhi)
    torch.cuda.synchronize()
    assert torch.equal(plo, ulo) and torch.equal(phi, uhi)
    # finer pieces give bounds at least as tight as the whole box, up to the early-exit widening
    w_lo = torch.empty((1, cam.height, cam.width, 3), device="cuda")
    w_hi = torch.empty_like(w_lo)
    ar.ar_render_abstract(s.handle, intr, pose, ar.make_cells(box_lo, box_hi), 1, 16, w_lo, w_hi)
    torch.cuda.synchronize()
    assert float((phi - plo).mean()) < float((w_hi - w_lo).mean())
    s.close()


def test_partitioned_parity_and_soundness(arlib, orc):
    ar = arlib
    sc, cam, box_lo, box_hi = _scene()
    parts = [2, 1, 2, 1, 1, 1]
    s = ar.Scene(sc)
    plo = torch.empty((cam.height, cam.width, 3), device="cuda")
    phi = torch.empty_like(plo)
    ar.ar_render_abstract_partitioned(s.handle, ar.make_intrinsics(cam), ar.make_pose(cam),
                                      ar.make_cells(box_lo, box_hi)[0], parts, 0, plo, phi)
    torch.cuda.synchronize()
    glo, ghi = plo.double().cpu().numpy(), phi.double().cpu().numpy()
    s.close()
    olo, ohi, frag = orc.render_abstract_partitioned(sc, cam, box_lo, box_hi, parts)
    ok = frag == 0
    e = np.maximum(np.abs(glo - olo), np.abs(ghi - ohi)).max(axis=-1)
    assert (e[ok] > TOL).sum() / max(1, ok.sum()) <= 1e-3, e[ok].max()
    assert e[ok].max() < 1e-3
    rng = np.random.default_rng(32)
    worst, nv = orc.check_samples(sc, cam, synth.sample_poses(rng, box_lo, box_hi, 400), glo, ghi)
    assert nv == 0, worst


def test_refined_render(arlib, orc):
    """Adaptive refinement: the pieces cover the box; the bounds are never
    looser than the box's own, at least as tight as the union of the last
    round's pieces, deterministic, and sound at sampled poses."""
    ar = arlib
    sc, cam, box_lo, box_hi = _scene()
    s = ar.Scene(sc)
    intr, pose = ar.make_intrinsics(cam), ar.make_pose(cam)
    box = ar.make_cells(box_lo, box_hi)[0]
    shape = (cam.height, cam.width, 3)
    rlo = torch.full(shape, -7.0, device="cuda")
    rhi = torch.full_like(rlo, -7.0)
    llo, lhi = ar.ar_render_abstract_refined(s.handle, intr, pose, box, 3, 16, rlo, rhi)
    assert llo.shape == (5, 6)                      # 1 -> 2 -> 3 -> 5 pieces
    act = box_hi > box_lo
    assert np.all(llo >= box_lo) and np.all(lhi <= box_hi) and np.all(llo <= lhi)
    vol = np.prod((lhi - llo)[:, act], axis=1).sum() / np.prod((box_hi - box_lo)[act])
    assert abs(vol - 1.0) < 1e-12
    one_lo = torch.empty((1,) + shape, device="cuda")
    one_hi = torch.empty_like(one_lo)
    ar.ar_render_abstract(s.handle, intr, pose, ar.make_cells(box_lo, box_hi), 1, 16, one_lo, one_hi)
    p_lo = torch.empty((5,) + shape, device="cuda")
    p_hi = torch.empty_like(p_lo)
    ar.ar_render_abstract(s.handle, intr, pose, ar.make_cells(llo, lhi), 5, 16, p_lo, p_hi)
    ulo = torch.empty(shape, device="cuda")
    uhi = torch.empty_like(ulo)
    ar.ar_bounds_union(p_lo, p_hi, 5, cam.width, cam.height, ulo, uhi)
    torch.cuda.synchronize()
    assert torch.all(rlo >= one_lo[0]) and torch.all(rhi <= one_hi[0])
    assert torch.all(rlo >= ulo) and torch.all(rhi <= uhi)
    assert float((rhi - rlo).mean()) < float((one_hi - one_lo).mean())
    r2lo = torch.empty_like(rlo)
    r2hi = torch.empty_like(rlo)
    l2lo, l2hi = ar.ar_render_abstract_refined(s.handle, intr, pose, box, 3, 16, r2lo, r2hi)
    torch.cuda.synchronize()
    assert np.array_equal(l2lo, llo) and np.array_equal(l2hi, lhi)
    assert torch.equal(r2lo, rlo) and torch.equal(r2hi, rhi)
    with pytest.raises(ar.ArError):
        ar.ar_render_abstract_refined(s.handle, intr, pose, box, 13, 16, r2lo, r2hi)
    glo, ghi = rlo.double().cpu().numpy(), rhi.double().cpu().numpy()
    s.close()
    rng = np.random.default_rng(33)
    worst, nv = orc.check_samples(sc, cam, synth.sample_poses(rng, box_lo, box_hi, 400), glo, ghi)
    assert nv == 0, worst
