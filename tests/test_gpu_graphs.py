"""CUDA graphs for repeated renders (ar_scene_set_graphs): after the first
render of a shape, a cell batch's binning and windowed rounds are replayed
from a captured graph, with bounds bit-identical to enqueueing them, on the
legacy default stream and on a torch stream, across blend modes, FP64
thresholds and cell batching."""
import numpy as np
import pytest

from paper_2503_00308_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arlib():
    from paper_2503_00308_gb300 import _build, ar
    _build.build()
    assert torch.cuda.is_available()
    return ar


def _renders(ar, sc, cam, lo, hi, graphs, n, stream=None, blend=None, thr=None, limit=0):
    s = ar.Scene(sc)
    ar.ar_scene_set_graphs(s.handle, graphs)
    ar.ar_set_profiling(s.handle, True)
    if blend is not None:
        ar.ar_scene_set_blend(s.handle, blend)
    if thr is not None:
        ar.ar_scene_set_fp64_alpha(s.handle, thr)
    if limit:
        ar.ar_set_workspace_limit(s.handle, limit)
    out = []
    # the same output buffers every time: they are part of a graph's key
    a = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    for _ in range(n):
        if stream is None:
            a.fill_(-7.0)
            b.fill_(-7.0)
            s.render(cam, lo, hi, a, b, tile=16)
        else:
            with torch.cuda.stream(stream):       # outputs filled and rendered on the same stream
                a.fill_(-7.0)
                b.fill_(-7.0)
                s.render(cam, lo, hi, a, b, tile=16, stream=stream.cuda_stream)
        st = ar.ar_last_render_stats(s.handle)
        torch.cuda.synchronize()
        out.append((a.cpu().numpy(), b.cpu().numpy(), st))
    s.close()
    return out


def test_graph_replay_is_bit_identical(arlib):
    ar = arlib
    w = synth.object10k()
    ref = _renders(ar, w.scene, w.camera, w.cells_lo, w.cells_hi, False, 1)[0]
    assert ref[2]["n_graph_replays"] == 0
    got = _renders(ar, w.scene, w.camera, w.cells_lo, w.cells_hi, True, 4)
    assert max(g[2]["n_graph_replays"] for g in got) > 0      # replays once the learned window settles
    for a, b, st in got:
        assert np.array_equal(a, ref[0]) and np.array_equal(b, ref[1])
        assert st["n_evaluated"] == ref[2]["n_evaluated"] and st["ms_render"] > 0


@pytest.mark.parametrize("case", ["torch_stream", "relational", "fp64_all", "batched"])
def test_graph_replay_variants(arlib, case):
    ar = arlib
    sc = synth.object_scene(2500, 4)
    cam = synth.look_camera(72, 56, 80.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.05, 0.05, 0.05, 0.0, 0.0175, 0.0], [2, 1, 2, 1, 2, 1])
    kw = {}
    if case == "torch_stream":
        kw["stream"] = torch.cuda.Stream()
    elif case == "relational":
        kw["blend"] = ar.AR_BLEND_RELATIONAL
    elif case == "fp64_all":
        kw["thr"] = 0.0
    else:
        kw["limit"] = 2 << 20      # several cell batches, each with its own graph
    ref = _renders(ar, sc, cam, lo, hi, False, 1, **kw)[0]
    got = _renders(ar, sc, cam, lo, hi, True, 4, **kw)
    assert max(g[2]["n_graph_replays"] for g in got) > 0
    for a, b, _ in got:
        assert np.array_equal(a, ref[0]) and np.array_equal(b, ref[1])


def test_graphs_argument_checks(arlib):
    ar = arlib
    s = ar.Scene(synth.cube_scene(4, 0))
    assert ar.lib().ar_scene_set_graphs(s.handle, 2) == ar.AR_EINVAL      # the raw C call: only 0 or 1
    s.close()
    with pytest.raises(ar.ArError):
        ar.ar_scene_set_graphs(None, 1)
