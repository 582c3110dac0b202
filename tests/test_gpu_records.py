"""The decision part of the records (Algorithm 1 lines 2-7 with set-valued
variables): which pairs reach the image, near-plane straddles, depth-key
intervals and pixel boxes.  These are integer or FP64 outputs that decide
integer outcomes (which Gaussians a pixel sees, the three-valued Ind), so the
CUDA path must reproduce the FP64 oracle's values bit for bit."""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import arlib  # noqa: E402,F401


def _check(arlib, orc, sc, cam, clo, chi):
    s = arlib.Scene(sc)
    g = s.debug_records(cam, clo, chi)
    s.close()
    o = orc.records(sc, cam, clo, chi)
    valid = o["valid"] > 0
    assert np.array_equal(g[:, 0] > 0, valid), (int((g[:, 0] > 0).sum()), int(valid.sum()))
    assert np.array_equal(g[valid, 1] > 0, o["straddle"][valid] > 0)
    for j, k in [(2, "klo"), (3, "khi"), (4, "px0"), (5, "px1"), (6, "py0"), (7, "py1")]:
        assert np.array_equal(g[valid, j], o[k][valid]), (k, np.abs(g[valid, j] - o[k][valid]).max())
    # the expansion point of the pixel stage is a pixel centre
    assert np.all(np.mod(g[valid, 8:10], 1.0) == 0.5)
    return int(valid.sum())


@pytest.mark.parametrize("hw", [
    [0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087],
    [0.05, 0.0, 0.05, 0.0, 0.0175, 0.0],
    [0.0, 0.0, 0.01, 0.0, 0.0, 0.0],
])
def test_object_records_bit_exact(arlib, orc, hw):
    sc = synth.object_scene(20000, 2)
    cam = synth.look_camera(400, 300, 500.0, centre=(0, 0, -4))
    clo = -np.array(hw)
    assert _check(arlib, orc, sc, cam, clo, -clo) > 10000


def test_near_and_guard_records_bit_exact(arlib, orc):
    rng = np.random.default_rng(17)
    sc = synth.cube_scene(3000, 5, half=1.0, logscale_mu=-1.8)
    sc.uw[:, 0] = rng.uniform(-3.0, 3.0, size=3000).astype(np.float32)
    sc.uw[:, 2] = rng.uniform(-0.9, 1.0, size=3000).astype(np.float32)
    cam = synth.look_camera(160, 120, 140.0, centre=(0, 0, -1.0))
    clo = np.array([-0.05, -0.02, -0.05, 0.0, -0.0087, 0.0])
    o = orc.records(sc, cam, clo, -clo)
    assert o["straddle"].sum() > 10
    _check(arlib, orc, sc, cam, clo, -clo)


def test_unbounded_records_bit_exact(arlib, orc):
    w = synth.unbounded750k()
    sc = w.scene.subset(np.arange(100000))
    for c in (0, 77, 255):
        _check(arlib, orc, sc, w.camera, w.cells_lo[c], w.cells_hi[c])
