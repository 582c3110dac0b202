"""Seeded synthetic inputs: Gaussian-splat scenes, pinhole cameras and pose-cell grids.

This module only draws random numbers and lays out arrays.  It holds none of
the abstract-rendering arithmetic, so both the CUDA path and the CPU oracle can
be fed from it without sharing any of the method's code.

Scene records follow the paper's Gaussian tuple <uw, Mw, o, c> (Sec. 2.2): the
covariance factor Mw is carried as a log-scale vector and a unit quaternion
(w, x, y, z); colours are degree-0 RGB.  Cameras use the OpenCV frame (x right,
y down, z forward); a nominal pose is a world->camera rotation R_wc and the
camera centre t in world coordinates.  A pose cell is a box over
delta = (tx, ty, tz, rx, ry, rz): a world-frame translation of the camera
centre and XYZ Euler angles of a rotation applied in the camera frame.

The named workloads mirror the synthetic scenes the paper's trained scenes
(Table 3) are replaced by: a tiny 64-Gaussian check scene, a 10k-Gaussian
object, the same object at 300k Gaussians and 800x800, and a 750k-Gaussian
unbounded scene.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Scene:
    uw: np.ndarray        # (n, 3) float32 means, world frame
    logscale: np.ndarray  # (n, 3) float32 log of the per-axis scales
    quat: np.ndarray      # (n, 4) float32 unit quaternions (w, x, y, z)
    opacity: np.ndarray   # (n,)   float32 in (0, 1)
    rgb: np.ndarray       # (n, 3) float32 in [0, 1]

    @property
    def n(self) -> int:
        return int(self.uw.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.uw[idx].copy(), self.logscale[idx].copy(), self.quat[idx].copy(),
                     self.opacity[idx].copy(), self.rgb[idx].copy())


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    R_wc: np.ndarray      # (3, 3) float64 world -> camera rotation
    t: np.ndarray         # (3,) float64 camera centre in world coordinates


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    camera: Camera
    cells_lo: np.ndarray  # (n_cells, 6) float64
    cells_hi: np.ndarray  # (n_cells, 6) float64

    @property
    def n_cells(self) -> int:
        return int(self.cells_lo.shape[0])

    def pixel_cells(self) -> int:
        return self.camera.width * self.camera.height * self.n_cells


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def object_scene(n: int, seed: int, mean_sd: float = 0.5, logscale_mu: float = -4.0,
                 logscale_sd: float = 0.5, opacity_mu: float = 0.0) -> Scene:
    """Object-centred scene: means N(0, mean_sd^2 I), log-scales N(mu, sd), random
    rotations, opacity sigmoid(N(opacity_mu, 1)), RGB uniform [0, 1]."""
    rng = np.random.default_rng(seed)
    uw = rng.normal(scale=mean_sd, size=(n, 3))
    ls = rng.normal(loc=logscale_mu, scale=logscale_sd, size=(n, 3))
    q = _unit_quats(rng, n)
    o = _sigmoid(rng.normal(loc=opacity_mu, size=n))
    c = rng.uniform(size=(n, 3))
    return Scene(uw.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                 o.astype(np.float32), c.astype(np.float32))


def cube_scene(n: int, seed: int, half: float = 0.5, logscale_mu: float = -2.5,
               logscale_sd: float = 0.3) -> Scene:
    """Means uniform in [-half, half]^3 (the tiny check scene)."""
    rng = np.random.default_rng(seed)
    uw = rng.uniform(-half, half, size=(n, 3))
    ls = rng.normal(loc=logscale_mu, scale=logscale_sd, size=(n, 3))
    q = _unit_quats(rng, n)
    o = _sigmoid(rng.normal(size=n))
    c = rng.uniform(size=(n, 3))
    return Scene(uw.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                 o.astype(np.float32), c.astype(np.float32))


def box_scene(n: int, seed: int, extent=(20.0, 5.0, 20.0), logscale_mu: float = -3.0,
              logscale_sd: float = 0.7, opacity_mu: float = 0.5, clear_centre=None,
              clear_radius: float = 0.0) -> Scene:
    """Unbounded scene: means uniform in an axis box centred on the origin (y is up/down).
    Means closer than clear_radius to clear_centre are drawn again (a capture
    position has free space around it)."""
    rng = np.random.default_rng(seed)
    ext = np.asarray(extent, dtype=np.float64)
    uw = rng.uniform(-0.5, 0.5, size=(n, 3)) * ext
    if clear_radius > 0:
        c = np.asarray(clear_centre, dtype=np.float64)
        bad = np.linalg.norm(uw - c, axis=1) < clear_radius
        while bad.any():
            uw[bad] = rng.uniform(-0.5, 0.5, size=(int(bad.sum()), 3)) * ext
            bad = np.linalg.norm(uw - c, axis=1) < clear_radius
    ls = rng.normal(loc=logscale_mu, scale=logscale_sd, size=(n, 3))
    q = _unit_quats(rng, n)
    o = _sigmoid(rng.normal(loc=opacity_mu, size=n))
    c = rng.uniform(size=(n, 3))
    return Scene(uw.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                 o.astype(np.float32), c.astype(np.float32))


def scene_boxes(sc: Scene, seed: int, frac: float = 0.3, mean_d=(0.0, 0.0, 0.0), opacity_scale: float = 1.0,
                opacity_add: float = 0.0, red_add: float = 0.0) -> dict:
    """Scene-parameter boxes in the manner of the paper's Sec. 4.5 experiments,
    on a seeded fraction of the Gaussians: the mean moved by 0..mean_d (world
    frame), the opacity scaled by opacity_scale and raised by up to
    opacity_add (capped below 1), the red channel raised by up to red_add
    (capped at 1).  Returns float32 arrays uw_lo, uw_hi (n, 3), o_lo, o_hi
    (n,), c_lo, c_hi (n, 3); the other Gaussians keep lo = hi = nominal."""
    rng = np.random.default_rng(seed)
    sel = rng.uniform(size=sc.n) < frac
    d = np.asarray(mean_d, dtype=np.float64)
    uw = sc.uw.astype(np.float64)
    uw_lo = np.where(sel[:, None], uw + np.minimum(d, 0.0), uw)
    uw_hi = np.where(sel[:, None], uw + np.maximum(d, 0.0), uw)
    o = sc.opacity.astype(np.float64)
    o_lo = np.where(sel, np.minimum(o * opacity_scale, 0.99), o)
    o_hi = np.where(sel, np.minimum(o * opacity_scale + opacity_add, 0.99), o)
    c = sc.rgb.astype(np.float64)
    c_lo = c.copy()
    c_hi = c.copy()
    c_hi[:, 0] = np.where(sel, np.minimum(c[:, 0] + red_add, 1.0), c[:, 0])
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"uw_lo": f(uw_lo), "uw_hi": f(uw_hi), "o_lo": f(o_lo), "o_hi": f(o_hi), "c_lo": f(c_lo), "c_hi": f(c_hi)}


def look_camera(width: int, height: int, f: float, centre=(0.0, 0.0, -4.0), near: float = 0.2) -> Camera:
    """Pinhole camera with identity orientation (looking along +z) at `centre`.
    Intrinsics are rounded to float32 so every consumer sees the same values."""
    f32 = lambda v: float(np.float32(v))
    return Camera(width, height, f32(f), f32(f), f32(width / 2.0), f32(height / 2.0), f32(near),
                  np.eye(3, dtype=np.float64), np.asarray(centre, dtype=np.float64))


def cell_grid(halfwidth, splits) -> tuple[np.ndarray, np.ndarray]:
    """Uniform split of the box prod_k [-halfwidth_k, halfwidth_k] into prod_k splits_k cells.

    halfwidth and splits are length-6 sequences over (tx, ty, tz, rx, ry, rz);
    translations in metres, rotations in radians.  Cells are enumerated with
    the last dimension fastest."""
    hw = np.asarray(halfwidth, dtype=np.float64)
    sp = np.asarray(splits, dtype=np.int64)
    assert hw.shape == (6,) and sp.shape == (6,) and np.all(sp >= 1)
    edges = [np.linspace(-hw[k], hw[k], sp[k] + 1) for k in range(6)]
    idx = np.stack(np.meshgrid(*[np.arange(s) for s in sp], indexing="ij"), axis=-1).reshape(-1, 6)
    lo = np.empty(idx.shape, dtype=np.float64)
    hi = np.empty(idx.shape, dtype=np.float64)
    for k in range(6):
        lo[:, k] = edges[k][idx[:, k]]
        hi[:, k] = edges[k][idx[:, k] + 1]
    return lo, hi


def sample_poses(rng, lo, hi, n) -> np.ndarray:
    """n poses drawn uniformly from the cell [lo, hi] (shape (n, 6))."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.uniform(size=(n, 6))


DEG = math.pi / 180.0


def tiny64(seed: int = 0) -> Workload:
    """64 Gaussians in [-0.5, 0.5]^3, 32x32 image, f = 32, camera at z = -3,
    x-translation +-0.01 m as one cell."""
    sc = cube_scene(64, seed)
    cam = look_camera(32, 32, 32.0, centre=(0.0, 0.0, -3.0))
    lo, hi = cell_grid([0.01, 0, 0, 0, 0, 0], [1] * 6)
    return Workload("tiny64", sc, cam, lo, hi)


def object10k(seed: int = 0, n: int = 10_000, width: int = 200, height: int = 200,
              f: float = 220.0, splits=(2, 2, 2, 1, 2, 1)) -> Workload:
    """10k-Gaussian object, 200x200, f = 220, camera at distance 4; pose box
    +-5 cm translation x +-1 deg yaw split 2x2x2x2 = 16 cells."""
    sc = object_scene(n, seed)
    cam = look_camera(width, height, f, centre=(0.0, 0.0, -4.0))
    lo, hi = cell_grid([0.05, 0.05, 0.05, 0.0, 1.0 * DEG, 0.0], splits)
    return Workload("object10k", sc, cam, lo, hi)


def object300k(seed: int = 0, n: int = 300_000, width: int = 800, height: int = 800,
               f: float = 1100.0, splits=(2, 2, 2, 2, 2, 2)) -> Workload:
    """The object scene at 300k Gaussians, 800x800, f = 1100, camera at distance 4;
    full 6-DoF box +-2 cm / +-0.5 deg split 2^6 = 64 cells."""
    sc = object_scene(n, seed)
    cam = look_camera(width, height, f, centre=(0.0, 0.0, -4.0))
    lo, hi = cell_grid([0.02, 0.02, 0.02, 0.5 * DEG, 0.5 * DEG, 0.5 * DEG], splits)
    return Workload("object300k", sc, cam, lo, hi)


def unbounded750k(seed: int = 0, n: int = 750_000, width: int = 1280, height: int = 720,
                  f: float = 900.0, splits=(4, 2, 4, 2, 2, 2), clear_radius: float = 0.0) -> Workload:
    """750k Gaussians in a 20 x 5 x 20 m box, camera at the origin looking +z
    (inside the scene, so near-plane straddles occur), 1280x720, f = 900;
    +-10 cm / +-2 deg split into 256 cells.  clear_radius > 0 keeps Gaussians
    that far from the camera."""
    sc = box_scene(n, seed, clear_centre=(0.0, 0.0, 0.0), clear_radius=clear_radius)
    cam = look_camera(width, height, f, centre=(0.0, 0.0, 0.0))
    lo, hi = cell_grid([0.10, 0.10, 0.10, 2 * DEG, 2 * DEG, 2 * DEG], splits)
    return Workload("unbounded750k", sc, cam, lo, hi)


WORKLOADS = {
    "tiny64": tiny64,
    "object10k": object10k,
    "object300k": object300k,
    "unbounded750k": unbounded750k,
}


# ------------------------------------------------------------------ serving mix
SERVE_SCENES = {"object10k": lambda: object_scene(10_000, 0),
                "object300k": lambda: object_scene(300_000, 0),
                "unbounded750k": lambda: box_scene(750_000, 0)}

_SPLITS = {1: (1, 1, 1, 1, 1, 1), 4: (2, 1, 2, 1, 1, 1), 16: (2, 2, 2, 1, 2, 1), 64: (2, 2, 2, 2, 2, 2),
           256: (4, 2, 4, 2, 2, 2)}


@dataclasses.dataclass
class Request:
    scene: str            # key of SERVE_SCENES
    camera: Camera
    cells_lo: np.ndarray
    cells_hi: np.ndarray
    gap: float            # unit-mean exponential inter-arrival gap (scale by the mean interval)

    def pixel_cells(self) -> int:
        return self.cells_lo.shape[0] * self.camera.width * self.camera.height


def serving_mix(n_requests: int, seed: int = 0, max_out_bytes: float = 1.5e9) -> list[Request]:
    """A seeded stream of abstract-render requests over the resident 10k / 300k /
    750k scenes: resolutions 200x200 to 1280x720, 6-DoF pose boxes of 1 to 256
    cells, Poisson arrivals (unit-mean exponential gaps).  Cell counts are
    lowered (by 4x steps) until both bound images of a request fit in
    max_out_bytes."""
    rng = np.random.default_rng(seed)
    names = ["object10k", "object300k", "unbounded750k"]
    sizes = [(200, 200), (400, 300), (640, 480), (800, 800), (1280, 720)]
    counts = [1, 4, 16, 64, 256]
    out = []
    for _ in range(n_requests):
        name = names[int(rng.choice(3, p=[0.5, 0.3, 0.2]))]
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        nc = counts[int(rng.choice(5, p=[0.3, 0.3, 0.2, 0.15, 0.05]))]
        while nc > 1 and nc * w * h * 24 > max_out_bytes:
            nc //= 4
        if name == "unbounded750k":
            cam = look_camera(w, h, 0.703 * w, centre=(0.0, 0.0, 0.0))
            hw = [0.10, 0.10, 0.10, 2 * DEG, 2 * DEG, 2 * DEG]
        else:
            cam = look_camera(w, h, 1.1 * w if name == "object10k" else 1.375 * w, centre=(0.0, 0.0, -4.0))
            hw = [0.02, 0.02, 0.02, 0.5 * DEG, 0.5 * DEG, 0.5 * DEG]
        lo, hi = cell_grid(hw, _SPLITS[nc])
        out.append(Request(name, cam, lo, hi, float(rng.exponential())))
    return out
