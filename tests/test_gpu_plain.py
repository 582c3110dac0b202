"""The plain FP64 path (ar_render_abstract_plain_fp64) against the oracle and
against the batched FP32 path.

The plain path runs the same relaxation with FP64 records and FP64 per-pixel
arithmetic, one cell per launch sequence, with no early stopping: away from
fragile pixels it matches the FP64 oracle far inside the 1e-4 contract, and
the batched FP32 path stays within the contract of it.
"""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
PLAIN_TOL = 1e-6   # FP64 path vs FP64 oracle, non-fragile pixels


@pytest.fixture(scope="module")
def arlib():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    assert torch.cuda.is_available()
    return ar


def render(ar, scene, cam, lo, hi, plain, tile=0):
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 6)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 6)
    s = ar.Scene(scene)
    out_lo = torch.full((lo.shape[0], cam.height, cam.width, 3), -7.0, dtype=torch.float32, device="cuda")
    out_hi = torch.full_like(out_lo, -7.0)
    (s.render_plain_fp64 if plain else s.render)(cam, lo, hi, out_lo, out_hi, tile=tile)
    stats = ar.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    r = out_lo.double().cpu().numpy(), out_hi.double().cpu().numpy()
    s.close()
    return r[0], r[1], stats


def check_vs_oracle(orc, scene, cam, lo_c, hi_c, glo, ghi, tol):
    olo, ohi, frag = orc.render_abstract(scene, cam, lo_c, hi_c)
    ok = ~np.isnan(olo[..., 0]) & (frag == 0)
    e = np.maximum(np.abs(glo - olo), np.abs(ghi - ohi)).max(axis=-1)
    assert np.all(e[ok] <= tol), e[ok].max()
    return e[ok].max(initial=0.0), ok


def test_plain_tiny64(arlib, orc):
    w = synth.tiny64()
    glo, ghi, st = render(arlib, w.scene, w.camera, w.cells_lo, w.cells_hi, plain=True)
    assert np.all(glo >= 0) and np.all(ghi <= 1) and np.all(glo <= ghi)
    err, _ = check_vs_oracle(orc, w.scene, w.camera, w.cells_lo[0], w.cells_hi[0], glo[0], ghi[0], PLAIN_TOL)
    print("plain tiny64 max |err| =", err)
    assert st["n_records"] > 0
    rng = np.random.default_rng(5)
    poses = synth.sample_poses(rng, w.cells_lo[0], w.cells_hi[0], 2000)
    worst, nv = orc.check_samples(w.scene, w.camera, poses, glo[0], ghi[0], tol=0.0)
    assert nv == 0, worst


@pytest.mark.parametrize("hw,splits", [
    ([0.05, 0.05, 0.05, 0.0, 0.0175, 0.0], [2, 1, 1, 1, 2, 1]),
    ([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087], [1, 1, 1, 1, 2, 2]),
])
def test_plain_object_and_batched(arlib, orc, hw, splits):
    sc = synth.object_scene(2500, 4)
    cam = synth.look_camera(72, 56, 80.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid(hw, splits)
    plo, phi, st = render(arlib, sc, cam, lo, hi, plain=True, tile=8)
    assert st["n_launches"] >= 4 * lo.shape[0]   # one launch sequence per cell
    blo, bhi, _ = render(arlib, sc, cam, lo, hi, plain=False)
    worst = 0.0
    for c in range(lo.shape[0]):
        err, ok = check_vs_oracle(orc, sc, cam, lo[c], hi[c], plo[c], phi[c], PLAIN_TOL)
        worst = max(worst, err)
        # the batched FP32 path within the contract of the plain FP64 one
        d = np.maximum(np.abs(blo[c] - plo[c]), np.abs(bhi[c] - phi[c])).max(axis=-1)
        assert np.all(d[ok] <= TOL + PLAIN_TOL), d[ok].max()
    print("plain object max |err| =", worst)
    rng = np.random.default_rng(11)
    c = lo.shape[0] - 1
    worst_s, nv = orc.check_samples(sc, cam, synth.sample_poses(rng, lo[c], hi[c], 200), plo[c], phi[c])
    assert nv == 0, worst_s


def test_plain_empty_and_point(arlib, orc):
    cam = synth.look_camera(20, 17, 24.0, centre=(0, 0, -3))
    lo = np.zeros((1, 6))
    glo, ghi, _ = render(arlib, synth.cube_scene(0, 0), cam, lo, lo, plain=True)
    assert np.all(glo == 0) and np.all(ghi == 0)
    w = synth.tiny64()
    d = np.array([0.004, -0.003, 0.01, 0.002, -0.004, 0.003])
    glo, ghi, _ = render(arlib, w.scene, w.camera, d, d, plain=True)
    img = orc.render_concrete(w.scene, w.camera, d, "sort")
    _, _, frag = orc.render_abstract(w.scene, w.camera, d, d)
    ok = frag == 0
    assert np.abs(glo[0] - img)[ok].max() < PLAIN_TOL and np.abs(ghi[0] - img)[ok].max() < PLAIN_TOL
