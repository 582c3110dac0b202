"""MatrixInv with the adjustments of Sec. 3.1 on the CUDA path: the adaptive
Taylor order and input splitting where the assertion of Algorithm 3 fails on
a whole pose cell.  Parity with the FP64 oracle (same tolerance as
test_gpu_parity), the split counted in the render statistics, and soundness at
sampled poses."""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import arlib, compare, gpu_render  # noqa: E402,F401


def _near_scene():
    sc = synth.cube_scene(60, 3, half=0.3)
    cam = synth.look_camera(32, 32, 28.0, centre=(0, 0, -1.2))
    clo = np.array([-0.05, -0.05, -0.05, -2.5 * synth.DEG, -2.5 * synth.DEG, -2.5 * synth.DEG])
    return sc, cam, clo


def test_split_parity_and_counts(arlib, orc):
    sc, cam, clo = _near_scene()
    rec = orc.records(sc, cam, clo, -clo)
    v = rec["valid"] > 0
    n_split = int((v & (rec["pieces"] > 0)).sum())
    n_fb = int((v & (rec["fallback"] > 0)).sum())
    assert n_split >= 2
    # the plain FP64 path builds every record: its counts match the oracle's
    s = arlib.Scene(sc)
    lo64 = torch.zeros((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    hi64 = torch.zeros_like(lo64)
    arlib.ar_set_profiling(s.handle, True)
    s.render_plain_fp64(cam, clo.reshape(1, 6), -clo.reshape(1, 6), lo64, hi64)
    st = arlib.ar_last_render_stats(s.handle)
    s.close()
    assert st["n_split"] == n_split and st["n_fallback"] == n_fb, (st["n_split"], n_split, st["n_fallback"], n_fb)
    # the batched FP32 path: parity and soundness
    glo, ghi, st32 = gpu_render(arlib, sc, cam, clo, -clo, return_stats=True)
    assert st32["n_split"] <= n_split and st32["n_fallback"] <= n_fb
    compare(orc, sc, cam, clo, -clo, glo[0], ghi[0])
    compare(orc, sc, cam, clo, -clo, lo64.double().cpu().numpy()[0], hi64.double().cpu().numpy()[0])
    rng = np.random.default_rng(4)
    poses = synth.sample_poses(rng, clo, -clo, 3000)
    worst, nv = orc.check_samples(sc, cam, poses, glo[0], ghi[0], tol=0.0)
    assert nv == 0, worst


def test_split_unbounded_slice(arlib, orc):
    # camera inside a 20 x 5 x 20 m scene: near-camera pairs fail MatrixInv on
    # the whole cell; a 64 x 64 window of the first cell against the oracle
    w = synth.unbounded750k()
    sc = w.scene.subset(np.arange(20000))
    lo, hi = w.cells_lo[:2], w.cells_hi[:2]
    glo, ghi, st = gpu_render(arlib, sc, w.camera, lo, hi, return_stats=True)
    assert st["n_split"] > 0
    win = (608, 671, 328, 391)
    for c in range(2):
        compare(orc, sc, w.camera, lo[c], hi[c], glo[c], ghi[c], window=win)
