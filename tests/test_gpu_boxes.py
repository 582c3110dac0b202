"""Scene-parameter boxes (Sec. 4.5) on the CUDA path: parity with the FP64
oracle (same tolerance as test_gpu_parity), bit-exact record decisions with a
mean box, soundness at sampled (pose, scene) pairs, and the argument checks."""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import arlib, compare  # noqa: E402,F401


def _box_array(b):
    return np.concatenate([b["uw_lo"], b["uw_hi"], b["o_lo"][:, None], b["o_hi"][:, None], b["c_lo"], b["c_hi"]],
                          axis=1).astype(np.float64)


def _render(ar, sc, cam, lo, hi, boxes):
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 6)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 6)
    s = ar.Scene(sc)
    s.set_boxes(boxes)
    out_lo = torch.full((lo.shape[0], cam.height, cam.width, 3), -7.0, dtype=torch.float32, device="cuda")
    out_hi = torch.full_like(out_lo, -7.0)
    s.render(cam, lo, hi, out_lo, out_hi)
    torch.cuda.synchronize()
    r = out_lo.double().cpu().numpy(), out_hi.double().cpu().numpy()
    s.close()
    return r


def _sample_scene(sc, b, rng):
    lo, hi = b["uw_lo"].astype(np.float64), b["uw_hi"].astype(np.float64)
    uw = lo + (hi - lo) * rng.uniform(size=lo.shape)
    o = b["o_lo"] + (b["o_hi"].astype(np.float64) - b["o_lo"]) * rng.uniform(size=sc.n)
    c = b["c_lo"] + (b["c_hi"].astype(np.float64) - b["c_lo"]) * rng.uniform(size=(sc.n, 3))
    return synth.Scene(uw, sc.logscale.astype(np.float64), sc.quat.astype(np.float64), o, c)


KINDS = {"colour": dict(red_add=0.5), "mean": dict(mean_d=(0.0, 0.08, 0.0)),
         "opacity": dict(opacity_scale=0.5, opacity_add=0.1),
         "all": dict(red_add=0.3, mean_d=(0.03, 0.03, 0.0), opacity_scale=0.8, opacity_add=0.1)}


@pytest.mark.parametrize("kind", list(KINDS))
def test_boxes_parity_and_soundness(arlib, orc, kind):
    sc = synth.object_scene(1500, 11, logscale_mu=-3.0)
    cam = synth.look_camera(56, 48, 66.0, centre=(0, 0, -3))
    lo, hi = synth.cell_grid([0.01, 0.01, 0.01, 0.0, 0.003, 0.0], [2, 1, 1, 1, 1, 1])
    b = synth.scene_boxes(sc, 5, frac=0.4, **KINDS[kind])
    glo, ghi = _render(arlib, sc, cam, lo, hi, b)
    assert np.all(glo >= 0) and np.all(ghi <= 1) and np.all(glo <= ghi)
    orc.set_boxes(_box_array(b))
    try:
        for c in range(lo.shape[0]):
            compare(orc, sc, cam, lo[c], hi[c], glo[c], ghi[c])
    finally:
        orc.set_boxes(None)
    rng = np.random.default_rng(9)
    for k in range(24):
        c = k % lo.shape[0]
        s2 = _sample_scene(sc, b, rng)
        pose = synth.sample_poses(rng, lo[c], hi[c], 1)[0]
        img = orc.render_concrete(s2, cam, pose, "ind")
        assert np.all(img >= glo[c]) and np.all(img <= ghi[c]), (kind, k)


def test_mean_box_records_bit_exact(arlib, orc):
    sc = synth.object_scene(6000, 4)
    cam = synth.look_camera(200, 160, 240.0, centre=(0, 0, -4))
    clo = -np.array([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087])
    b = synth.scene_boxes(sc, 2, frac=0.5, mean_d=(0.05, -0.04, 0.06))
    s = arlib.Scene(sc)
    s.set_boxes(b)
    g = s.debug_records(cam, clo, -clo)
    s.close()
    orc.set_boxes(_box_array(b))
    try:
        o = orc.records(sc, cam, clo, -clo)
    finally:
        orc.set_boxes(None)
    valid = o["valid"] > 0
    assert np.array_equal(g[:, 0] > 0, valid)
    for j, k in [(1, "straddle"), (2, "klo"), (3, "khi"), (4, "px0"), (5, "px1"), (6, "py0"), (7, "py1")]:
        assert np.array_equal(g[valid, j], o[k][valid]), k


def test_nominal_boxes_and_reset(arlib):
    sc = synth.object_scene(800, 6)
    cam = synth.look_camera(40, 36, 48.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.02, 0.0, 0.02, 0.0, 0.005, 0.0], [2, 1, 1, 1, 1, 1])
    a_lo, a_hi = _render(arlib, sc, cam, lo, hi, None)
    nominal = synth.scene_boxes(sc, 1, frac=0.0)
    b_lo, b_hi = _render(arlib, sc, cam, lo, hi, nominal)
    assert np.array_equal(a_lo, b_lo) and np.array_equal(a_hi, b_hi)
    # a box, then back to the nominal scene
    s = arlib.Scene(sc)
    s.set_boxes(synth.scene_boxes(sc, 1, frac=0.5, red_add=0.4))
    s.set_boxes(None)
    c_lo = torch.empty((2, cam.height, cam.width, 3), device="cuda")
    c_hi = torch.empty_like(c_lo)
    s.render(cam, lo, hi, c_lo, c_hi)
    torch.cuda.synchronize()
    s.close()
    assert np.array_equal(c_lo.double().cpu().numpy(), a_lo) and np.array_equal(c_hi.double().cpu().numpy(), a_hi)


def test_box_argument_errors(arlib):
    sc = synth.object_scene(50, 1)
    s = arlib.Scene(sc)
    b = synth.scene_boxes(sc, 1, frac=1.0, red_add=0.2)
    with pytest.raises(Exception):
        s.set_boxes({"uw_lo": b["uw_lo"]})                       # half a pair
    bad = dict(b)
    bad["o_lo"] = b["o_hi"] + 0.01                                # lo > hi
    with pytest.raises(Exception):
        s.set_boxes(bad)
    bad = dict(b)
    bad["c_hi"] = np.minimum(b["c_hi"] + 0.5, 1.5).astype(np.float32)   # colour above 1
    with pytest.raises(Exception):
        s.set_boxes(bad)
    s.close()
