"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, and its soundness.

Tolerance, per colour channel, against the oracle's bounds: |gpu - oracle| <=
1e-4 at every pixel that is not fragile.  A pixel is fragile where a threshold
decision that the GPU takes in single precision (MatrixInv's assertion on a
cell or a split piece, a cutoff ramp narrower than 0.05) lies within its
rounding band, so that both outcomes are sound; fragile pixels are checked for
soundness instead, and at most 1 % of the compared pixels may be fragile.
Every comparison prints its largest error and its fragile fraction.
Soundness: concrete FP64 renders at sampled poses lie inside the GPU bounds.
Invariances: cell batching is bit-exact; the tile size moves the bounds by at
most 2e-5 (early stopping).
"""
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


def gpu_render(ar, scene, cam, lo, hi, tile=0, return_stats=False):
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 6)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 6)
    nc = lo.shape[0]
    s = ar.Scene(scene)
    out_lo = torch.full((nc, cam.height, cam.width, 3), -7.0, dtype=torch.float32, device="cuda")
    out_hi = torch.full_like(out_lo, -7.0)
    ar.ar_set_profiling(s.handle, True)
    s.render(cam, lo, hi, out_lo, out_hi, tile=tile)
    stats = ar.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    r = out_lo.double().cpu().numpy(), out_hi.double().cpu().numpy()
    s.close()
    return (r + (stats,)) if return_stats else r


FRAG_MAX = 0.01


def compare(orc, scene, cam, lo_c, hi_c, glo, ghi, window=None, label=""):
    """Oracle bounds of one cell vs the GPU's; returns (max err, fragile fraction)."""
    olo, ohi, frag = orc.render_abstract(scene, cam, lo_c, hi_c, window=window)
    m = ~np.isnan(olo[..., 0])
    ok = m & (frag == 0)
    e = np.maximum(np.abs(glo - olo), np.abs(ghi - ohi)).max(axis=-1)
    fr = float((m & (frag != 0)).sum()) / max(1, int(m.sum()))
    err = float(e[ok].max(initial=0.0))
    print("parity %s: max |gpu - oracle| = %.3g over %d pixels, fragile %.4f" % (label, err, int(ok.sum()), fr))
    assert np.all(e[ok] <= TOL), (err, np.argwhere(e > TOL)[:5])
    assert fr <= FRAG_MAX, fr
    assert np.all(glo[m] <= ghi[m])
    return err, fr


def test_tiny64_parity_and_soundness(arlib, orc):
    w = synth.tiny64()
    glo, ghi = gpu_render(arlib, w.scene, w.camera, w.cells_lo, w.cells_hi)
    assert glo.shape == (1, 32, 32, 3) and np.all(glo >= 0) and np.all(ghi <= 1) and np.all(glo <= ghi)
    compare(orc, w.scene, w.camera, w.cells_lo[0], w.cells_hi[0], glo[0], ghi[0])
    rng = np.random.default_rng(0)
    poses = synth.sample_poses(rng, w.cells_lo[0], w.cells_hi[0], 10_000)
    worst, nv = orc.check_samples(w.scene, w.camera, poses, glo[0], ghi[0], tol=0.0)
    assert nv == 0, worst


def test_point_cell_is_concrete(arlib, orc):
    w = synth.tiny64()
    d = np.array([0.004, -0.003, 0.01, 0.002, -0.004, 0.003])
    glo, ghi = gpu_render(arlib, w.scene, w.camera, d, d)
    img = orc.render_concrete(w.scene, w.camera, d, "sort")
    _, _, frag = orc.render_abstract(w.scene, w.camera, d, d)
    ok = frag == 0
    assert np.abs(glo[0] - img)[ok].max() < TOL and np.abs(ghi[0] - img)[ok].max() < TOL
    assert np.all(glo[0] <= img + 1e-12) and np.all(img <= ghi[0] + 1e-12)


@pytest.mark.parametrize("hw,splits", [
    ([0.05, 0.05, 0.05, 0.0, 0.0175, 0.0], [2, 1, 2, 1, 2, 1]),   # 4-DoF like the 10k object
    ([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087], [1, 2, 1, 1, 1, 2]),  # 6-DoF
])
def test_object_parity_ragged_tiles(arlib, orc, hw, splits):
    sc = synth.object_scene(2500, 4)
    cam = synth.look_camera(72, 56, 80.0, centre=(0, 0, -4))   # 72x56: ragged 16x16 and 8x8 tiles
    lo, hi = synth.cell_grid(hw, splits)
    glo, ghi = gpu_render(arlib, sc, cam, lo, hi)
    for c in range(lo.shape[0]):
        compare(orc, sc, cam, lo[c], hi[c], glo[c], ghi[c])
    rng = np.random.default_rng(3)
    c = lo.shape[0] - 1
    worst, nv = orc.check_samples(sc, cam, synth.sample_poses(rng, lo[c], hi[c], 300), glo[c], ghi[c])
    assert nv == 0, worst


def test_tile_and_batch_invariance(arlib):
    sc = synth.object_scene(1500, 6)
    cam = synth.look_camera(50, 38, 60.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.0, 0.01, 0.0], [2, 1, 2, 1, 1, 1])
    a_lo, a_hi = gpu_render(arlib, sc, cam, lo, hi, tile=16)
    b_lo, b_hi = gpu_render(arlib, sc, cam, lo, hi, tile=8)
    # tiles differ only in where a pixel may stop early (each stop widens by <= 1e-5)
    assert np.abs(a_lo - b_lo).max() <= 2e-5 and np.abs(a_hi - b_hi).max() <= 2e-5
    for c in [0, 3]:
        c_lo, c_hi = gpu_render(arlib, sc, cam, lo[c:c + 1], hi[c:c + 1], tile=16)
        assert np.array_equal(c_lo[0], a_lo[c]) and np.array_equal(c_hi[0], a_hi[c])


def test_edge_cases(arlib, orc):
    cam = synth.look_camera(20, 17, 24.0, centre=(0, 0, -3))
    lo = np.array([[-0.01, 0, 0, 0, 0, 0]])
    hi = -lo
    # empty scene
    empty = synth.cube_scene(0, 0)
    glo, ghi = gpu_render(arlib, empty, cam, lo, hi)
    assert np.all(glo == 0) and np.all(ghi == 0)
    # single Gaussian
    one = synth.cube_scene(1, 3, logscale_mu=-1.5)
    glo, ghi = gpu_render(arlib, one, cam, lo, hi)
    compare(orc, one, cam, lo[0], hi[0], glo[0], ghi[0])
    assert ghi.max() > 0.05
    # all Gaussians behind the camera
    back = synth.cube_scene(30, 1)
    back.uw[:, 2] = -5.0
    glo, ghi = gpu_render(arlib, back, cam, lo, hi)
    assert np.all(glo == 0) and np.all(ghi == 0)
    # opacities below the 1/255 cutoff never contribute
    faint = synth.cube_scene(30, 2)
    faint.opacity[:] = 0.003
    glo, ghi = gpu_render(arlib, faint, cam, lo, hi)
    assert np.all(ghi == 0)
    # near-plane straddle
    near = synth.cube_scene(30, 2, half=0.25, logscale_mu=-2.5)
    near.uw[:, 2] = np.linspace(-0.85, -0.65, 30).astype(np.float32)
    camn = synth.look_camera(24, 24, 20.0, centre=(0, 0, -1.0))
    lo2 = np.array([[-0.02, -0.02, -0.08, 0, 0, 0]])
    glo, ghi = gpu_render(arlib, near, camn, lo2, -lo2)
    compare(orc, near, camn, lo2[0], -lo2[0], glo[0], ghi[0])
    rng = np.random.default_rng(9)
    worst, nv = orc.check_samples(near, camn, synth.sample_poses(rng, lo2[0], -lo2[0], 500), glo[0], ghi[0])
    assert nv == 0, worst


def test_bad_arguments_rejected(arlib):
    ar = arlib
    sc = synth.cube_scene(4, 0)
    s = ar.Scene(sc)
    cam = synth.look_camera(8, 8, 8.0)
    out = torch.zeros((1, 8, 8, 3), device="cuda")
    with pytest.raises(ar.ArError) as e:
        s.render(cam, [[0.1, 0, 0, 0, 0, 0]], [[0.0, 0, 0, 0, 0, 0]], out, out)   # lo > hi
    assert e.value.code == ar.AR_EINVAL
    with pytest.raises(ar.ArError):
        s.render(cam, [[0] * 6], [[0] * 6], out, out, tile=12)
    bad = synth.cube_scene(4, 0)
    bad.opacity[0] = 1.5
    with pytest.raises(ar.ArError):
        ar.Scene(bad)
    s.close()


def test_object10k_all_cells(arlib, orc):
    """The 10k-Gaussian, 200x200, 16-cell workload in one launch, every pixel
    of every cell against the oracle (the wide Mahalanobis intervals of this
    workload are where the FP64 re-evaluation of the opacity stage is
    needed), one cell also for soundness."""
    w = synth.object10k()
    glo, ghi, st = gpu_render(arlib, w.scene, w.camera, w.cells_lo, w.cells_hi, return_stats=True)
    assert st["n_records"] > 0 and st["m_vars"] == 4
    assert st["n_fp64"] > 0 and st["n_fp64_segments"] > 0
    for c in range(w.n_cells):
        compare(orc, w.scene, w.camera, w.cells_lo[c], w.cells_hi[c], glo[c], ghi[c], label="object10k cell %d" % c)
    rng = np.random.default_rng(5)
    c = 7
    worst, nv = orc.check_samples(w.scene, w.camera, synth.sample_poses(rng, w.cells_lo[c], w.cells_hi[c], 64),
                                  glo[c], ghi[c])
    assert nv == 0, worst


def test_object300k_full_size_sampled(arlib, orc):
    """The 300k-Gaussian, 800x800, 64-cell workload in the launch configuration
    the benchmark times (tile chosen by the autotuner); the oracle on eight
    seeded 32x32 windows of eight cells, one at the image centre."""
    w = synth.object300k()
    glo, ghi, st = gpu_render(arlib, w.scene, w.camera, w.cells_lo, w.cells_hi, return_stats=True)
    assert st["m_vars"] == 6 and st["n_fallback"] < st["n_records"] // 100
    rng = np.random.default_rng(1)
    cells = rng.choice(64, size=8, replace=False)
    xs, ys = rng.integers(250, 520, size=8), rng.integers(250, 520, size=8)
    xs[0] = ys[0] = 384
    for c, x, y in zip(cells, xs, ys):
        compare(orc, w.scene, w.camera, w.cells_lo[c], w.cells_hi[c], glo[c], ghi[c],
                window=(int(x), int(x) + 31, int(y), int(y) + 31), label="object300k cell %d at (%d, %d)" % (c, x, y))
    assert np.all(glo <= ghi)


def test_unbounded750k_slice(arlib, orc):
    """750k Gaussians in a 20 x 5 x 20 m box around the camera, 1280x720, four
    of the 256 cells of the +-10 cm / +-2 deg box rendered in one launch; the
    oracle on a 24x24 window of each."""
    w = synth.unbounded750k()
    rng = np.random.default_rng(2)
    cells = np.sort(rng.choice(w.n_cells, size=4, replace=False))
    glo, ghi, st = gpu_render(arlib, w.scene, w.camera, w.cells_lo[cells], w.cells_hi[cells], return_stats=True)
    assert st["m_vars"] == 6
    xs, ys = rng.integers(100, 1150, size=4), rng.integers(100, 590, size=4)
    for i, (c, x, y) in enumerate(zip(cells, xs, ys)):
        compare(orc, w.scene, w.camera, w.cells_lo[c], w.cells_hi[c], glo[i], ghi[i],
                window=(int(x), int(x) + 23, int(y), int(y) + 23), label="unbounded750k cell %d at (%d, %d)" % (c, x, y))


def test_cell_batches_are_bit_identical(arlib):
    """A small workspace limit splits the cells into batches; bounds must not change."""
    ar = arlib
    sc = synth.object_scene(3000, 12)
    cam = synth.look_camera(60, 44, 70.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.01, 0.0, 0.0], [2, 1, 2, 2, 1, 1])
    ref_lo, ref_hi = gpu_render(ar, sc, cam, lo, hi)
    s = ar.Scene(sc)
    ar.ar_set_workspace_limit(s.handle, 4 << 20)     # records of about one cell per batch
    out_lo = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
    out_hi = torch.empty_like(out_lo)
    ar.ar_set_profiling(s.handle, True)
    s.render(cam, lo, hi, out_lo, out_hi)
    st = ar.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    assert np.array_equal(out_lo.double().cpu().numpy(), ref_lo)
    assert np.array_equal(out_hi.double().cpu().numpy(), ref_hi)
    assert st["n_records"] > 0 and st["ms_render"] > 0
    s.close()


def test_batches_split_on_entry_overflow(arlib):
    """A cell batch whose tile entries would overflow the bins' 32-bit indices
    is split in halves and rendered again: with a low cap every batch splits
    down to one cell, with bounds bit-identical to one batch; a single cell
    over the cap is refused with AR_ENOMEM."""
    ar = arlib
    sc = synth.object_scene(3000, 12)
    cam = synth.look_camera(60, 44, 70.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.01, 0.0, 0.0], [2, 1, 2, 2, 1, 1])
    ref_lo, ref_hi, ref_st = gpu_render(ar, sc, cam, lo, hi, tile=16, return_stats=True)
    s = ar.Scene(sc)
    per_cell = ref_st["n_entries"] * 2 // lo.shape[0]
    ar.ar_debug_set_entry_cap(s.handle, int(1.9 * per_cell))     # two cells' entries do not fit
    out_lo = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
    out_hi = torch.empty_like(out_lo)
    ar.ar_set_profiling(s.handle, True)
    s.render(cam, lo, hi, out_lo, out_hi, tile=16)
    st = ar.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    assert np.array_equal(out_lo.double().cpu().numpy(), ref_lo)
    assert np.array_equal(out_hi.double().cpu().numpy(), ref_hi)
    assert st["n_entries"] == ref_st["n_entries"] and st["n_evaluated"] == ref_st["n_evaluated"]
    ar.ar_debug_set_entry_cap(s.handle, 10)
    with pytest.raises(ar.ArError) as e:
        s.render(cam, lo, hi, out_lo, out_hi, tile=16)
    assert e.value.code == ar.AR_ENOMEM
    s.close()


def test_host_outputs_match_device_outputs(arlib):
    """ar_render_abstract_host: page-locked buffers (written by the render
    kernel itself), pageable buffers (staged and copied), one of each (copied),
    and an empty scene all give the device call's bounds bit for bit."""
    ar = arlib
    sc = synth.object_scene(2500, 4)
    cam = synth.look_camera(72, 56, 80.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.0, 0.01, 0.0], [2, 1, 2, 1, 1, 1])
    nc = lo.shape[0]
    ref_lo, ref_hi = gpu_render(ar, sc, cam, lo, hi)
    s = ar.Scene(sc)
    intr, pose, cells = ar.make_intrinsics(cam), ar.make_pose(cam), ar.make_cells(lo, hi)
    shape = (nc, cam.height, cam.width, 3)
    p_lo = torch.full(shape, -7.0, dtype=torch.float32).pin_memory()
    p_hi = torch.full(shape, -7.0, dtype=torch.float32).pin_memory()
    ar.ar_render_abstract_host(s.handle, intr, pose, cells, nc, 0, p_lo, p_hi)
    assert np.array_equal(p_lo.double().numpy(), ref_lo) and np.array_equal(p_hi.double().numpy(), ref_hi)
    n_lo, n_hi = np.full(shape, -7.0, np.float32), np.full(shape, -7.0, np.float32)
    ar.ar_render_abstract_host(s.handle, intr, pose, cells, nc, 0, n_lo, n_hi)
    assert np.array_equal(n_lo.astype(np.float64), ref_lo) and np.array_equal(n_hi.astype(np.float64), ref_hi)
    # one page-locked and one pageable buffer: the staged copy path
    mixed_hi = np.full(shape, -7.0, np.float32)
    p_lo.fill_(-7.0)
    ar.ar_render_abstract_host(s.handle, intr, pose, cells, nc, 0, p_lo, mixed_hi)
    assert np.array_equal(p_lo.double().numpy(), ref_lo) and np.array_equal(mixed_hi.astype(np.float64), ref_hi)
    s.close()
    e = ar.Scene(synth.cube_scene(0, 0))
    p_lo.fill_(-7.0)
    p_hi.fill_(-7.0)
    ar.ar_render_abstract_host(e.handle, intr, pose, cells, nc, 0, p_lo, p_hi)
    assert float(p_lo.abs().max()) == 0.0 and float(p_hi.abs().max()) == 0.0
    e.close()


def test_windowed_rounds_restart(arlib, orc):
    """Faint, dense scenes: tiles never stop early, so sweeps outgrow the first
    (512-entry) and second (8192-entry) windows of built records and are swept
    again; the bounds match the oracle and the plain FP64 path."""
    sc = synth.object_scene(4500, 9, mean_sd=0.15, logscale_mu=-2.6)
    sc.opacity[:] = np.float32(0.02)
    cam = synth.look_camera(40, 24, 60.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.01, 0.0, 0.01, 0.0, 0.0, 0.0], [1, 1, 1, 1, 1, 1])
    glo, ghi, st = gpu_render(arlib, sc, cam, lo, hi, tile=16, return_stats=True)
    assert st["n_restarted"] > 0, st
    assert st["n_built"] == st["n_records"]          # every record is reached
    compare(orc, sc, cam, lo[0], hi[0], glo[0], ghi[0], window=(8, 4, 16, 12))
    s = arlib.Scene(sc)
    plo = torch.empty((1, cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    phi = torch.empty_like(plo)
    s.render_plain_fp64(cam, lo, hi, plo, phi)
    torch.cuda.synchronize()
    d = np.maximum(np.abs(glo - plo.double().cpu().numpy()), np.abs(ghi - phi.double().cpu().numpy()))
    assert d.max() <= 2 * TOL, d.max()
    s.close()


def test_guard_band_parity(arlib, orc):
    """Gaussians spread far beyond the frustum and close to the camera plane:
    the guard band drops or half-keeps them identically on both sides."""
    rng = np.random.default_rng(17)
    sc = synth.cube_scene(400, 5, half=1.0, logscale_mu=-1.8)
    sc.uw[:, 0] = rng.uniform(-3.0, 3.0, size=400).astype(np.float32)
    sc.uw[:, 2] = rng.uniform(-0.6, 1.0, size=400).astype(np.float32)
    cam = synth.look_camera(40, 32, 36.0, centre=(0, 0, -1.0))
    lo, hi = synth.cell_grid([0.05, 0.02, 0.05, 0.0, 0.0087, 0.0], [2, 1, 1, 1, 1, 1])
    rec = orc.records(sc, cam, lo[0], hi[0])
    assert rec["straddle"].sum() > 0
    glo, ghi = gpu_render(arlib, sc, cam, lo, hi)
    for c in range(lo.shape[0]):
        compare(orc, sc, cam, lo[c], hi[c], glo[c], ghi[c])
        poses = synth.sample_poses(np.random.default_rng(c), lo[c], hi[c], 300)
        worst, nv = orc.check_samples(sc, cam, poses, glo[c], ghi[c])
        assert nv == 0, worst


def test_autotuned_tile(arlib):
    """tile = 0: the autotuner picks a (tile edge, chunk) once per (size, pose
    variables), the same on later calls with bit-identical bounds, and those
    bounds are within the early stop's 2e-5 of an explicit tile's."""
    sc = synth.object_scene(1500, 6)
    cam = synth.look_camera(50, 38, 60.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.0, 0.01, 0.0], [2, 1, 2, 1, 1, 1])
    s = arlib.Scene(sc)
    arlib.ar_set_profiling(s.handle, True)
    outs = []
    for tile in (0, 0):
        a = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
        b = torch.empty_like(a)
        s.render(cam, lo, hi, a, b, tile=tile)
        st = arlib.ar_last_render_stats(s.handle)
        outs.append((a, b, st["tile"], st["chunk"]))
    assert (outs[0][2], outs[0][3]) in ((16, 16), (16, 8), (16, 32), (8, 16))
    assert outs[1][2:] == outs[0][2:]
    torch.cuda.synchronize()
    assert torch.equal(outs[1][0], outs[0][0]) and torch.equal(outs[1][1], outs[0][1])
    a = torch.empty_like(outs[0][0])
    b = torch.empty_like(a)
    s.render(cam, lo, hi, a, b, tile=outs[0][2])
    st = arlib.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    assert st["chunk"] == 16
    assert float((a - outs[0][0]).abs().max()) <= 2e-5 and float((b - outs[0][1]).abs().max()) <= 2e-5
    s.close()


@pytest.mark.parametrize("chunk", [8, 32])
def test_chunk_sizes_parity(arlib, orc, chunk):
    """The sweep's other chunk sizes (which the autotuner may pick) keep parity
    with the oracle and stay within 2e-5 of chunks of 16."""
    sc = synth.object_scene(2500, 4)
    cam = synth.look_camera(72, 56, 80.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087], [1, 2, 1, 1, 1, 2])
    ref_lo, ref_hi = gpu_render(arlib, sc, cam, lo, hi, tile=16)
    s = arlib.Scene(sc)
    out_lo = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
    out_hi = torch.empty_like(out_lo)
    assert arlib.lib().ar_debug_set_chunk(s.handle, chunk) == 0
    s.render(cam, lo, hi, out_lo, out_hi, tile=16)
    st = arlib.ar_last_render_stats(s.handle)
    torch.cuda.synchronize()
    assert st["chunk"] == chunk
    glo, ghi = out_lo.double().cpu().numpy(), out_hi.double().cpu().numpy()
    s.close()
    assert np.abs(glo - ref_lo).max() <= 2e-5 and np.abs(ghi - ref_hi).max() <= 2e-5
    for c in range(lo.shape[0]):
        compare(orc, sc, cam, lo[c], hi[c], glo[c], ghi[c], label="chunk %d cell %d" % (chunk, c))


def test_depth_prefix_phases_are_bit_identical(arlib):
    """Two-phase binning: the first phase bins each cell's first 1/2^s of its
    depth-sorted events, segments that need more restart with full lists.
    Every prefix (and the learned one) gives bounds bit-identical to one
    phase, and a small prefix does restart segments."""
    ar = arlib
    w = synth.object10k()
    lo, hi = w.cells_lo[:6], w.cells_hi[:6]
    outs = {}
    for shift in (0, 1, 3, 6, -1):
        s = ar.Scene(w.scene)
        ar.ar_set_profiling(s.handle, True)
        ar.ar_debug_set_prefix(s.handle, shift)
        out_lo = torch.full((len(lo), w.camera.height, w.camera.width, 3), -7.0, device="cuda")
        out_hi = torch.full_like(out_lo, -7.0)
        for _ in range(2):                     # the second render uses the learned prefix (shift -1)
            s.render(w.camera, lo, hi, out_lo, out_hi, tile=16)
        st = ar.ar_last_render_stats(s.handle)
        torch.cuda.synchronize()
        outs[shift] = (out_lo.cpu().numpy(), out_hi.cpu().numpy(), st)
        s.close()
    ref_lo, ref_hi, ref_st = outs[0]
    assert ref_st["n_restarted"] <= 2
    for shift, (o_lo, o_hi, st) in outs.items():
        assert np.array_equal(o_lo, ref_lo) and np.array_equal(o_hi, ref_hi), shift
        assert st["n_evaluated"] == ref_st["n_evaluated"], shift
    assert outs[6][2]["n_restarted"] > 100      # the second phase did run
    with pytest.raises(ar.ArError):
        ar.ar_debug_set_prefix(None, 3)


def test_depth_prefix_with_batches_and_scene_boxes(arlib):
    """The prefix is per cell, so batch splits (a small workspace limit) and
    scene-parameter boxes keep the bounds bit-identical too."""
    ar = arlib
    sc = synth.object_scene(3000, 12)
    cam = synth.look_camera(60, 44, 70.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.03, 0.0, 0.03, 0.01, 0.0, 0.0], [2, 1, 2, 2, 1, 1])
    res = []
    for shift, limit in ((0, 0), (4, 0), (4, 4 << 20)):
        s = ar.Scene(sc)
        s.set_boxes(synth.scene_boxes(sc, 5, frac=0.3, red_add=0.2, mean_d=(0.01, 0.0, 0.0), opacity_scale=0.9,
                                      opacity_add=0.05))
        ar.ar_debug_set_prefix(s.handle, shift)
        if limit:
            ar.ar_set_workspace_limit(s.handle, limit)
        out_lo = torch.empty((lo.shape[0], cam.height, cam.width, 3), device="cuda")
        out_hi = torch.empty_like(out_lo)
        s.render(cam, lo, hi, out_lo, out_hi, tile=16)
        torch.cuda.synchronize()
        res.append((out_lo.cpu().numpy(), out_hi.cpu().numpy()))
        s.close()
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])


def test_cull_before_decisions_is_bit_identical(arlib):
    """The cull of certain drops before the FP64 decision chain changes no
    record and no bound: a camera inside the scene (half the Gaussians behind
    the near plane, many outside the guard band) rendered with the cull always
    on, always off and chosen per workspace."""
    ar = arlib
    w = synth.unbounded750k(n=30_000, width=320, height=180, f=225.0, splits=(2, 1, 2, 1, 1, 1))
    outs = []
    for mode in (0, 1, -1):
        s = ar.Scene(w.scene)
        ar.ar_debug_set_cull(s.handle, mode)
        ar.ar_set_profiling(s.handle, True)
        out_lo = torch.full((w.n_cells, w.camera.height, w.camera.width, 3), -7.0, device="cuda")
        out_hi = torch.full_like(out_lo, -7.0)
        for _ in range(2):
            s.render(w.camera, w.cells_lo, w.cells_hi, out_lo, out_hi, tile=16)
        st = ar.ar_last_render_stats(s.handle)
        torch.cuda.synchronize()
        recs = s.debug_records(w.camera, w.cells_lo[0], w.cells_hi[0])
        outs.append((out_lo.cpu().numpy(), out_hi.cpu().numpy(), st, recs))
        s.close()
    assert outs[0][2]["n_records"] < 0.5 * 30_000 * w.n_cells   # most pairs reach no pixel
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
        assert o[2]["n_records"] == outs[0][2]["n_records"] and o[2]["n_entries"] == outs[0][2]["n_entries"]
        assert np.array_equal(o[3], outs[0][3])


def test_depth_prefix_and_cull_with_empty_cells(arlib, orc):
    """Cells that see nothing (the camera moved past the object) next to
    cells that do: every depth prefix, with the cull on and off, gives the
    bounds of one phase without the cull, the empty cells' bounds are 0, and
    a seen cell matches the oracle."""
    ar = arlib
    sc = synth.object_scene(2000, 21)
    cam = synth.look_camera(48, 40, 55.0, centre=(0, 0, -4))
    base_lo, base_hi = synth.cell_grid([0.03, 0.0, 0.03, 0.0, 0.01, 0.0], [2, 1, 1, 1, 2, 1])
    far = np.array([[0.0, 0.0, 8.0, 0.0, 0.0, 0.0]])     # 8 m forward: every Gaussian behind the camera
    lo = np.concatenate([base_lo[:2], far - 0.01, base_lo[2:]])
    hi = np.concatenate([base_hi[:2], far + 0.01, base_hi[2:]])
    res = {}
    for shift, cull in ((0, 0), (3, 0), (6, 1), (2, 1), (-1, -1)):
        s = ar.Scene(sc)
        ar.ar_debug_set_prefix(s.handle, shift)
        ar.ar_debug_set_cull(s.handle, cull)
        out_lo = torch.full((lo.shape[0], cam.height, cam.width, 3), -7.0, device="cuda")
        out_hi = torch.full_like(out_lo, -7.0)
        for _ in range(2):
            s.render(cam, lo, hi, out_lo, out_hi, tile=16)
        torch.cuda.synchronize()
        res[(shift, cull)] = (out_lo.double().cpu().numpy(), out_hi.double().cpu().numpy())
        s.close()
    ref_lo, ref_hi = res[(0, 0)]
    assert np.all(ref_lo[2] == 0) and np.all(ref_hi[2] == 0)
    for key, (o_lo, o_hi) in res.items():
        assert np.array_equal(o_lo, ref_lo) and np.array_equal(o_hi, ref_hi), key
    compare(orc, sc, cam, lo[1], hi[1], ref_lo[1], ref_hi[1], label="seen cell beside an empty one")


def test_cull_with_scene_boxes(arlib):
    """The cull reads the enclosures of the mean's box, as the FP64 chain
    reads the box: with scene-parameter boxes the records and bounds do not
    depend on it."""
    ar = arlib
    w = synth.unbounded750k(n=20_000, width=256, height=144, f=180.0, splits=(2, 1, 1, 1, 1, 1))
    boxes = synth.scene_boxes(w.scene, 4, frac=0.5, red_add=0.2, mean_d=(0.05, 0.02, 0.05), opacity_scale=0.9,
                              opacity_add=0.05)
    outs = []
    for cull in (0, 1):
        s = ar.Scene(w.scene)
        s.set_boxes(boxes)
        ar.ar_debug_set_cull(s.handle, cull)
        out_lo = torch.empty((w.n_cells, w.camera.height, w.camera.width, 3), device="cuda")
        out_hi = torch.empty_like(out_lo)
        s.render(w.camera, w.cells_lo, w.cells_hi, out_lo, out_hi, tile=16)
        torch.cuda.synchronize()
        outs.append((out_lo.cpu().numpy(), out_hi.cpu().numpy(),
                     s.debug_records(w.camera, w.cells_lo[0], w.cells_hi[0])))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])
