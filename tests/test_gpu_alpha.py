"""The per-pixel effective-opacity relaxation (Algorithm 1 lines 9-10 with
Table 2's Exp) of single (Gaussian, pixel, cell) triples, through the
ar_debug_alpha hook, against the oracle's pixel_alpha, and the FP64
re-evaluation of wide Mahalanobis intervals (ar_scene_set_fp64_alpha).

Per triple, in FP64 (precision 2, from the same FP32 record the renderer
reads) the opacity bounds and forms match the oracle's to 1e-4; in FP32 they
match to within the renderer's own deviation estimate (the quantity that
decides where it takes FP64), so that estimate is checked to bound the real
single-precision error."""
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


def _triples(orc, w, c, pixels):
    gi, px, py, ref = [], [], [], []
    for x, y in pixels:
        d = orc.pixel_detail(w.scene, w.camera, w.cells_lo[c], w.cells_hi[c], x, y, cap=20000)
        for row in d:
            if row[10] != 0:      # MatrixInv fallback or near-plane straddle: constant forms
                continue
            g = int(row[0])
            gi.append(g), px.append(x), py.append(y)
            ref.append(orc.pixel_alpha(w.scene, w.camera, w.cells_lo[c], w.cells_hi[c], g, x, y))
    return np.array(gi), np.array(px), np.array(py), ref


def _form_gap(a, b, rng):
    """max over the cell's corners and random poses of |a(p) - b(p)| (7-forms)."""
    p = np.concatenate([np.sign(rng.normal(size=(64, 6))), rng.uniform(-1, 1, size=(64, 6))])
    return float(np.abs(p @ (a[:6] - b[:6]) + (a[6] - b[6])).max())


@pytest.mark.parametrize("name,cell,pixels", [
    ("object10k", 0, [(4, 69), (100, 100), (90, 110), (140, 80)]),
    ("object10k", 11, [(60, 125), (120, 60)]),
])
def test_opacity_relaxation_per_triple(arlib, orc, name, cell, pixels):
    w = synth.WORKLOADS[name]()
    gi, px, py, ref = _triples(orc, w, cell, pixels)
    assert len(gi) > 50
    s = arlib.Scene(w.scene)
    g32 = s.debug_alpha(w.camera, w.cells_lo[cell], w.cells_hi[cell], gi, px, py, 0)
    g64 = s.debug_alpha(w.camera, w.cells_lo[cell], w.cells_hi[cell], gi, px, py, 2)
    s.close()
    rng = np.random.default_rng(4)
    worst32 = worst64 = ratio = 0.0
    for t, r in enumerate(ref):
        assert g32[t, 39] == 1 and g64[t, 39] == 3          # valid; FP64 taken in the second
        # the m interval and the opacity enclosure
        e64 = max(abs(g64[t, 16] - r["alo"]), abs(g64[t, 17] - r["ahi"]))
        e32 = max(abs(g32[t, 16] - r["alo"]), abs(g32[t, 17] - r["ahi"]))
        assert e64 <= 1e-4, (t, e64, r)
        # the opacity forms over the cell
        f64 = max(_form_gap(g64[t, 0:7], r["L"], rng), _form_gap(g64[t, 7:14], r["U"], rng))
        assert f64 <= 1e-4, (t, f64)
        # single precision within its own deviation estimate (plus the FP64 floor)
        dev = g32[t, 18]
        assert e32 <= 1.5 * dev + e64 + 2e-6, (t, e32, dev)
        worst32, worst64 = max(worst32, e32), max(worst64, e64)
        if dev > 1e-5:
            ratio = max(ratio, (e32 - e64) / dev)
    print("%s cell %d: %d triples, max opacity error FP32 %.3g, FP64 %.3g, worst error / estimate %.3g"
          % (name, cell, len(ref), worst32, worst64, ratio))


def test_fp64_threshold_controls_precision(arlib, orc):
    """Lowering the threshold takes more evaluations in FP64 and never moves
    the bounds by more than the contract; a huge threshold takes none; the
    threshold is validated; bounds stay within the parity tolerance of the
    oracle at the default."""
    w = synth.object10k()
    cells = [0, 5]
    lo, hi = w.cells_lo[cells], w.cells_hi[cells]
    s = arlib.Scene(w.scene)
    arlib.ar_set_profiling(s.handle, True)
    res = {}
    for thr in (3e38, 1e-4, 1e-5, 0.0):
        arlib.ar_scene_set_fp64_alpha(s.handle, thr)
        a = torch.empty((2, 200, 200, 3), device="cuda")
        b = torch.empty_like(a)
        s.render(w.camera, lo, hi, a, b, tile=16)
        st = arlib.ar_last_render_stats(s.handle)
        torch.cuda.synchronize()
        res[thr] = (a.double().cpu().numpy(), b.double().cpu().numpy(), st["n_fp64"], st["n_fp64_segments"])
    assert res[3e38][2] == 0 and res[3e38][3] == 0
    assert 0 < res[1e-4][2] < res[1e-5][2] < res[0.0][2]
    for thr in (1e-4, 1e-5):
        d = max(np.abs(res[thr][0] - res[0.0][0]).max(), np.abs(res[thr][1] - res[0.0][1]).max())
        assert d <= 1e-4, (thr, d)
    with pytest.raises(arlib.ArError):
        arlib.ar_scene_set_fp64_alpha(s.handle, -1.0)
    with pytest.raises(arlib.ArError):
        arlib.ar_scene_set_fp64_alpha(s.handle, float("nan"))
    s.close()


def test_fp64_reevaluation_is_tile_and_batch_invariant(arlib):
    """The FP64 decision depends only on the pixel's own sweep: the same
    bounds (to the early stop's 2e-5) at tile 8 and 16, and bit for bit when
    the cells are split into batches."""
    w = synth.object10k()
    cells = [0, 3, 12]
    lo, hi = w.cells_lo[cells], w.cells_hi[cells]
    out = {}
    for tile, limit in ((16, 0), (8, 0), (16, 1 << 20)):
        s = arlib.Scene(w.scene)
        if limit:
            arlib.ar_set_workspace_limit(s.handle, limit)
        arlib.ar_set_profiling(s.handle, True)
        a = torch.empty((3, 200, 200, 3), device="cuda")
        b = torch.empty_like(a)
        s.render(w.camera, lo, hi, a, b, tile=tile)
        st = arlib.ar_last_render_stats(s.handle)
        torch.cuda.synchronize()
        out[(tile, limit)] = (a.double().cpu().numpy(), b.double().cpu().numpy(), st["n_fp64"])
        s.close()
    assert out[(16, 0)][2] > 0
    a, b = out[(16, 0)], out[(8, 0)]
    assert np.abs(a[0] - b[0]).max() <= 2e-5 and np.abs(a[1] - b[1]).max() <= 2e-5
    c = out[(16, 1 << 20)]
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])


@pytest.mark.parametrize("name,cells", [("tiny64", (0,)), ("object10k", (0, 11)), ("object300k", (0, 37)),
                                        ("unbounded750k", (5, 200))])
def test_packed_chain_is_bit_identical(arlib, name, cells):
    """The renderer's FP32 chain to the Mahalanobis term holds each (lower,
    upper) constant pair as (-lo, hi) and moves both ends with one packed
    operation rounded up; since RD(x) = -RU(-x) for every IEEE operation, each
    end carries the bits of the scalar directed-rounding step it replaces.
    Every output of the opacity stage (forms, radii, enclosure, deviation
    estimate, m interval) agrees bit for bit, signed zeros included, with the
    scalar chain (precision 3) on sampled triples of one, four and six pose
    variables."""
    w = synth.WORKLOADS[name]()
    s = arlib.Scene(w.scene)
    rng = np.random.default_rng(11)
    total = 0
    for c in cells:
        recs = s.debug_records(w.camera, w.cells_lo[c], w.cells_hi[c])
        valid = np.nonzero(recs[:, 0] == 1)[0]
        pick = np.sort(rng.choice(valid, size=min(4000, len(valid)), replace=False))
        x0, x1, y0, y1 = (recs[pick, k] for k in (4, 5, 6, 7))
        px = (x0 + np.floor(rng.uniform(size=len(pick)) * (x1 - x0 + 1))).astype(np.int32)
        py = (y0 + np.floor(rng.uniform(size=len(pick)) * (y1 - y0 + 1))).astype(np.int32)
        gi = pick.astype(np.int64)
        packed = s.debug_alpha(w.camera, w.cells_lo[c], w.cells_hi[c], gi, px, py, 0)
        scalar = s.debug_alpha(w.camera, w.cells_lo[c], w.cells_hi[c], gi, px, py, 3)
        assert np.all(packed[:, 39] >= 1)
        assert np.array_equal(packed.view(np.uint64), scalar.view(np.uint64)), (name, c)
        total += len(pick)
    with pytest.raises(arlib.ArError):
        s.debug_alpha(w.camera, w.cells_lo[0], w.cells_hi[0], gi[:1], px[:1], py[:1], 4)
    s.close()
    print("%s: %d triples bit-identical" % (name, total))
