"""The no-allocation entry point (ar_render_abstract_noalloc).

Some callers may not allocate memory while they run, e.g. a real-time loop or
an embedded verifier that fixes all of its memory up front; the entry point
serves them from a fixed 64 MiB scratch array inside libar.  This file checks,
through the C ABI, that two calls in a row give the same bounds as the
allocating entry point (within the parity tolerance of the GPU tests), and
that a request too large for the scratch array is refused cleanly.  It is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


def _render(ar, fn, scene, cam, lo, hi, tile=16):
    cells = ar.make_cells(lo, hi)
    nc = len(cells)
    out_lo = torch.full((nc, cam.height, cam.width, 3), -7.0, dtype=torch.float32, device="cuda")
    out_hi = torch.full_like(out_lo, -7.0)
    fn(scene.handle, ar.make_intrinsics(cam), ar.make_pose(cam), cells, nc, tile, out_lo, out_hi, 0)
    torch.cuda.synchronize()
    return out_lo.cpu().numpy(), out_hi.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    sc = synth.object_scene(2000, 11)
    cam = synth.look_camera(64, 48, 70.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.0, 0.01, 0.0], [2, 1, 1, 1, 2, 1])
    s = ar.Scene(sc)
    ref_lo, ref_hi = _render(ar, ar.ar_render_abstract, s, cam, lo, hi)
    for _ in range(2):                       # the second call reuses the scratch array
        n_lo, n_hi = _render(ar, ar.ar_render_abstract_noalloc, s, cam, lo, hi)
        assert np.all(n_lo >= 0) and np.all(n_hi <= 1)
        assert np.abs(n_lo - ref_lo).max() <= TOL and np.abs(n_hi - ref_hi).max() <= TOL
    # a different, smaller request right after (stale scratch contents must not leak in)
    w = synth.tiny64()
    t = ar.Scene(w.scene)
    a_lo, a_hi = _render(ar, ar.ar_render_abstract, t, w.camera, w.cells_lo, w.cells_hi)
    b_lo, b_hi = _render(ar, ar.ar_render_abstract_noalloc, t, w.camera, w.cells_lo, w.cells_hi)
    assert np.abs(a_lo - b_lo).max() <= TOL and np.abs(a_hi - b_hi).max() <= TOL
    t.close()
    # with scene-parameter boxes (the decision and value chains read them the same way)
    s.set_boxes(synth.scene_boxes(sc, 3, frac=0.4, red_add=0.3, mean_d=(0.02, 0.0, 0.0), opacity_scale=0.8,
                                  opacity_add=0.1))
    ref_lo, ref_hi = _render(ar, ar.ar_render_abstract, s, cam, lo, hi)
    n_lo, n_hi = _render(ar, ar.ar_render_abstract_noalloc, s, cam, lo, hi)
    assert np.abs(n_lo - ref_lo).max() <= TOL and np.abs(n_hi - ref_hi).max() <= TOL
    s.close()


def test_noalloc_refuses_oversized_request():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    sc = synth.object_scene(40_000, 2)
    cam = synth.look_camera(64, 64, 70.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.02, 0.02, 0.02, 0.01, 0.01, 0.01], [2, 2, 2, 2, 1, 1])   # 16 cells x 40k
    s = ar.Scene(sc)
    out = torch.full((16, 64, 64, 3), -7.0, device="cuda")
    with pytest.raises(ar.ArError) as e:
        ar.ar_render_abstract_noalloc(s.handle, ar.make_intrinsics(cam), ar.make_pose(cam), ar.make_cells(lo, hi),
                                      16, 16, out, out, 0)
    assert e.value.code == ar.AR_ENOMEM and "64 MiB" in str(e.value)
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)            # outputs untouched
    s.close()
