"""FP64 CPU oracle for abstract rendering (test infrastructure only).

The arithmetic lives in oracle.c (plain C, double precision, straight loops in
the order of the paper's Algorithms 1-4).  This module compiles it with gcc and
marshals numpy arrays through ctypes.  Only the test-suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the CUDA library never
does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (OpenMP if available)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_render_concrete.argtypes = [P, P, P, P, P, I64, P, P, P, P, I, P]
        lib.orc_render_concrete.restype = I
        lib.orc_render_abstract.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I, I, I, I, P, P, P, P]
        lib.orc_render_abstract.restype = I
        lib.orc_render_abstract_tight.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I, I, I, I, P, P, P, P]
        lib.orc_render_abstract_tight.restype = I
        lib.orc_transmittance_chain.argtypes = [P, P, P, I, P, P]
        lib.orc_transmittance_chain.restype = I
        lib.orc_render_abstract_sort.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I, I, I, I, P, P]
        lib.orc_render_abstract_sort.restype = I
        lib.orc_records.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, P]
        lib.orc_records.restype = I
        lib.orc_matrixinv_interval.argtypes = [P, P, I, I, P, P, P]
        lib.orc_matrixinv_interval.restype = I
        lib.orc_matrixinv_cell.argtypes = [P, P, I, P, P, P]
        lib.orc_matrixinv_cell.restype = I
        lib.orc_relax_mul.argtypes = [P, P, P]
        lib.orc_relax_sq.argtypes = [P, P]
        lib.orc_relax_exp.argtypes = [P, P]
        lib.orc_alpha_from_m.argtypes = [P, D, D, D, D, I, P]
        lib.orc_pixel_alpha.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I64, I, I, P]
        lib.orc_pixel_alpha.restype = I
        lib.orc_rot_forms.argtypes = [P, P, P]
        lib.orc_concrete_alpha.argtypes = [P, P, P, D, P, P, P, P, D, D]
        lib.orc_concrete_alpha.restype = D
        lib.orc_check_samples.argtypes = [P, P, P, P, P, I64, P, P, P, P, I64, P, P, D, P]
        lib.orc_check_samples.restype = D
        lib.orc_empirical_bounds.argtypes = [P, P, P, P, P, I64, P, P, P, P, I64, P, P]
        lib.orc_pixel_detail.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I, I, P, I]
        lib.orc_pixel_detail.restype = I
        lib.orc_pixel_trace.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I64, I, I, P]
        lib.orc_pixel_trace.restype = I
        lib.orc_record_trace.argtypes = [P, P, P, P, P, I64, P, P, P, P, P, I64, P]
        lib.orc_record_trace.restype = I
        lib.orc_set_boxes.argtypes = [P, I64]
        lib.orc_set_boxes.restype = I
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = I
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the oracle's OpenMP thread count."""
    return int(_load().orc_set_threads(int(n)))


def _scene_args(scene):
    arrs = [_d(scene.uw), _d(scene.logscale), _d(scene.quat), _d(scene.opacity), _d(scene.rgb)]
    return arrs


def _cam_args(cam):
    intr = _d([cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.near])
    return intr, _d(cam.R_wc).reshape(9), _d(cam.t)


def render_concrete(scene, cam, delta, blend: str = "ind") -> np.ndarray:
    """GSplat (Algorithm 1) at one pose; blend 'sort' (Algorithm 2) or 'ind' (Algorithm 4)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    dl = _d(delta).reshape(6)
    out = np.zeros((cam.height, cam.width, 3), dtype=np.float64)
    st = lib.orc_render_concrete(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0), _p(dl),
                                 0 if blend == "sort" else 1, _p(out))
    if st:
        raise RuntimeError("oracle concrete render failed")
    return out


def set_boxes(boxes):
    """Scene-parameter boxes (Sec. 4.5) for the abstract calls that follow:
    an [n, 14] array per Gaussian (mean lo[3], hi[3]; opacity lo, hi; colour
    lo[3], hi[3]), or None to clear them."""
    lib = _load()
    if boxes is None:
        lib.orc_set_boxes(None, 0)
        return
    b = _d(boxes).reshape(-1, 14)
    if lib.orc_set_boxes(_p(b), b.shape[0]):
        raise MemoryError("oracle boxes")


def render_abstract(scene, cam, cell_lo, cell_hi, window=None, with_cond=False, tight=False):
    """AbstractSplat bounds of one pose cell.

    Returns (lo, hi, fragile) -- and cond if with_cond: lo/hi are [H, W, 3]
    float64 (only `window` = (px0, px1, py0, py1), inclusive, is filled; the
    rest stays NaN), fragile [H, W] uint8 marks pixels where a threshold
    decision that the single-precision path takes lies within its rounding
    band, and cond [H, W] estimates how far FP32 evaluation can move the
    bounds.  tight=True: the upper bound uses the relational transmittance
    of orc_render_abstract_tight (never above the interval one)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    lo = np.full((cam.height, cam.width, 3), np.nan)
    hi = np.full((cam.height, cam.width, 3), np.nan)
    frag = np.zeros((cam.height, cam.width), dtype=np.uint8)
    cond = np.zeros((cam.height, cam.width), dtype=np.float64)
    if window is None:
        window = (0, cam.width - 1, 0, cam.height - 1)
    px0, px1, py0, py1 = (int(v) for v in window)
    fn = lib.orc_render_abstract_tight if tight else lib.orc_render_abstract
    st = fn(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
            _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)),
            px0, px1, py0, py1, _p(lo), _p(hi), _p(frag), _p(cond))
    if st:
        raise RuntimeError("oracle abstract render failed")
    return (lo, hi, frag, cond) if with_cond else (lo, hi, frag)


def partition_cells(box_lo, box_hi, parts):
    """The pieces of a pose box cut into parts[k] equal pieces along dimension k
    (dimension 0 varying fastest): piece i of n is [lo + w i / n, lo + w (i+1) / n]
    with w = hi - lo, the last ending at hi.  Returns (lo [N, 6], hi [N, 6])."""
    box_lo = _d(box_lo).reshape(6)
    box_hi = _d(box_hi).reshape(6)
    parts = [int(p) for p in parts]
    n = int(np.prod(parts))
    lo = np.empty((n, 6))
    hi = np.empty((n, 6))
    for r0 in range(n):
        r = r0
        for k in range(6):
            P = parts[k]
            i = r % P
            r //= P
            w = box_hi[k] - box_lo[k]
            lo[r0, k] = box_lo[k] if i == 0 else box_lo[k] + w * float(i) / float(P)
            hi[r0, k] = box_hi[k] if i + 1 == P else box_lo[k] + w * float(i + 1) / float(P)
    return lo, hi


def render_abstract_partitioned(scene, cam, box_lo, box_hi, parts, window=None, tight=False):
    """Bounds of a pose box as the union of the bounds of its pieces (Sec. 5):
    the elementwise minimum of the pieces' lower bounds and maximum of their
    upper bounds.  Returns (lo, hi, fragile) like render_abstract; fragile marks
    a pixel fragile in any piece."""
    lo_c, hi_c = partition_cells(box_lo, box_hi, parts)
    lo = hi = frag = None
    for c in range(lo_c.shape[0]):
        a, b, f = render_abstract(scene, cam, lo_c[c], hi_c[c], window=window, tight=tight)
        lo = a if lo is None else np.minimum(lo, a)
        hi = b if hi is None else np.maximum(hi, b)
        frag = f if frag is None else np.maximum(frag, f)
    return lo, hi, frag


def transmittance_chain(L, alo, ahi):
    """Relational upper transmittance of a chain of factors (1 - a_j), taken
    in the given order: L [K, 7] lower opacity forms (six coefficients, then
    the constant), alo / ahi [K].  Returns (F [7], y_hi): F(p) >= prod (1 - a_j)
    for every p in [-1, 1]^6 and every a_j in [max(alo_j, L_j(p)), ahi_j]."""
    lib = _load()
    L = np.ascontiguousarray(L, dtype=np.float64).reshape(-1, 7)
    alo = np.ascontiguousarray(alo, dtype=np.float64).reshape(-1)
    ahi = np.ascontiguousarray(ahi, dtype=np.float64).reshape(-1)
    F = np.zeros(7)
    yhi = np.zeros(1)
    lib.orc_transmittance_chain(_p(L), _p(alo), _p(ahi), int(L.shape[0]), _p(F), _p(yhi))
    return F, float(yhi[0])


def render_abstract_sort(scene, cam, cell_lo, cell_hi, window=None):
    """Bounds of one pose cell with the abstract BlendSort of Example 2 (rank
    ranges from the depth-key intervals, interval hulls per rank) in place of
    BlendInd.  Returns (lo, hi), [H, W, 3] (NaN outside window)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    lo = np.full((cam.height, cam.width, 3), np.nan)
    hi = np.full((cam.height, cam.width, 3), np.nan)
    if window is None:
        window = (0, cam.width - 1, 0, cam.height - 1)
    px0, px1, py0, py1 = (int(v) for v in window)
    st = lib.orc_render_abstract_sort(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                                      _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)),
                                      px0, px1, py0, py1, _p(lo), _p(hi))
    if st:
        raise RuntimeError("oracle abstract render failed")
    return lo, hi


def records(scene, cam, cell_lo, cell_hi) -> dict:
    """Per-Gaussian summary of the abstract pipeline for one cell."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    out = np.zeros((scene.n, 13), dtype=np.float64)
    lib.orc_records(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                    _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)), _p(out))
    keys = ["valid", "straddle", "fallback", "klo", "khi", "px0", "px1", "py0", "py1", "rho",
            "pieces", "korder", "rho_margin"]
    return {k: out[:, i] for i, k in enumerate(keys)}


def concrete_alpha(uw, logscale, quat, opacity, cam, delta, ux, uy) -> float:
    lib = _load()
    intr, R0, t0 = _cam_args(cam)
    return float(lib.orc_concrete_alpha(_p(_d(uw)), _p(_d(logscale)), _p(_d(quat)), float(opacity),
                                        _p(intr), _p(R0), _p(t0), _p(_d(delta)), float(ux), float(uy)))


def matrixinv_interval(Xl, Xu, k: int = 8, symmetric: bool = False):
    """MatrixInv (Algorithm 3) on an interval 2x2 matrix whose entries are
    independent (symmetric=True: the off-diagonal entries are one variable).
    Returns (lower, upper, rho) as 2x2 arrays, or None if the assertion fails."""
    lib = _load()
    xl = _d(Xl).reshape(4)
    xu = _d(Xu).reshape(4)
    ol = np.zeros(4)
    ou = np.zeros(4)
    rho = np.zeros(1)
    st = lib.orc_matrixinv_interval(_p(xl), _p(xu), int(k), 1 if symmetric else 0, _p(ol), _p(ou), _p(rho))
    if st:
        return None
    return ol.reshape(2, 2), ou.reshape(2, 2), float(rho[0])


def matrixinv_cell(Xl, Xu, symmetric: bool = False):
    """The pipeline's MatrixInv on an interval 2x2 matrix (entries as in
    matrixinv_interval): adaptive Taylor order, and input splitting where the
    assertion fails on the whole box (Sec. 3.1, adjustments (2) and (3)).
    Returns (lower, upper, info) with info = {"pieces", "k", "rho"}, or None if
    even the split fails."""
    lib = _load()
    xl = _d(Xl).reshape(4)
    xu = _d(Xu).reshape(4)
    ol = np.zeros(4)
    ou = np.zeros(4)
    info = np.zeros(3)
    st = lib.orc_matrixinv_cell(_p(xl), _p(xu), 1 if symmetric else 0, _p(ol), _p(ou), _p(info))
    if st:
        return None
    return ol.reshape(2, 2), ou.reshape(2, 2), {"pieces": int(info[0]), "k": int(info[1]), "rho": float(info[2])}


def relax_mul(x, y) -> np.ndarray:
    """Mul relaxation on bounded scalars given as 14-vectors (lo form, hi form)."""
    lib = _load()
    out = np.zeros(14)
    lib.orc_relax_mul(_p(_d(x)), _p(_d(y)), _p(out))
    return out


def relax_sq(x) -> np.ndarray:
    lib = _load()
    out = np.zeros(14)
    lib.orc_relax_sq(_p(_d(x)), _p(out))
    return out


def relax_exp(x) -> np.ndarray:
    """Table 2's Exp relaxation on x <= 0 (x_hi clipped at 0): tangent at x_lo
    below, secant above.  x and the result are packed bounded scalars (14)."""
    out = np.zeros(14)
    _load().orc_relax_exp(_p(_d(x).reshape(14)), _p(out))
    return out


def alpha_from_m(m, o_lo, o_hi, tau_lo, tau_hi, straddle=False) -> dict:
    """The opacity stage a = o Exp(-m/2) with the clip to o and the cutoff
    ramps, from a packed bounded scalar m (14)."""
    out = np.zeros(19)
    _load().orc_alpha_from_m(_p(_d(m).reshape(14)), float(o_lo), float(o_hi), float(tau_lo), float(tau_hi),
                             int(bool(straddle)), _p(out))
    return {"L": out[0:7], "U": out[7:14], "alo": out[14], "ahi": out[15], "mlo": out[16], "mhi": out[17],
            "ramp": out[18]}


def pixel_alpha(scene, cam, cell_lo, cell_hi, gi, px, py):
    """The relaxed effective opacity of Gaussian gi at pixel (px, py) over one
    cell: its Mahalanobis term m (packed bounded scalar), the opacity forms L,
    U (7 each), alo, ahi, mlo, mhi, ramp and the record's opacity box and
    cutoff exponents.  None if the pair is not valid."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    out = np.zeros(39)
    st = lib.orc_pixel_alpha(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                             _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)), int(gi), int(px), int(py),
                             _p(out))
    if st:
        return None
    return {"m": out[0:14], "L": out[14:21], "U": out[21:28], "alo": out[28], "ahi": out[29], "mlo": out[30],
            "mhi": out[31], "ramp": out[32], "o_lo": out[33], "o_hi": out[34], "tau_lo": out[35],
            "tau_hi": out[36], "fallback": bool(out[37]), "straddle": bool(out[38])}


def rot_forms(lo, hi) -> np.ndarray:
    """Forms of the nine entries of R_delta over the cell: (9, 14)."""
    lib = _load()
    out = np.zeros((9, 14))
    lib.orc_rot_forms(_p(_d(lo)), _p(_d(hi)), _p(out))
    return out


def check_samples(scene, cam, poses, lo, hi, tol: float = 0.0):
    """Render at each pose (BlendSort) and compare with [lo, hi].
    Returns (largest violation, number of violating values)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    P = _d(poses).reshape(-1, 6)
    nv = np.zeros(1, dtype=np.int64)
    worst = lib.orc_check_samples(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0), _p(P), P.shape[0],
                                  _p(_d(lo)), _p(_d(hi)), float(tol), _p(nv))
    return float(worst), int(nv[0])


def empirical_bounds(scene, cam, poses):
    """Per-pixel min/max of the concrete renders over the given poses."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    P = _d(poses).reshape(-1, 6)
    lo = np.zeros((cam.height, cam.width, 3))
    hi = np.zeros((cam.height, cam.width, 3))
    lib.orc_empirical_bounds(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0), _p(P), P.shape[0],
                             _p(lo), _p(hi))
    return lo, hi


def pixel_detail(scene, cam, cell_lo, cell_hi, px, py, cap=4096):
    """Per-Gaussian relaxation details at one pixel (diagnosis): array (k, 12)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    out = np.zeros((cap, 12))
    k = lib.orc_pixel_detail(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                             _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)), int(px), int(py), _p(out), int(cap))
    return out[:k]


def pixel_trace(scene, cam, cell_lo, cell_hi, gi, px, py):
    """Intervals Dx, Dy, W[6], q[3], m of one Gaussian at one pixel (diagnosis)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    out = np.zeros(24)
    st = lib.orc_pixel_trace(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                             _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)), int(gi), int(px), int(py), _p(out))
    return None if st else out.reshape(12, 2)


def record_trace(scene, cam, cell_lo, cell_hi, gi):
    """X, E, Mp, conic intervals and rho of one (Gaussian, cell) pair (diagnosis)."""
    lib = _load()
    s = _scene_args(scene)
    intr, R0, t0 = _cam_args(cam)
    out = np.zeros(35)
    st = lib.orc_record_trace(*[_p(a) for a in s], scene.n, _p(intr), _p(R0), _p(t0),
                              _p(_d(cell_lo).reshape(6)), _p(_d(cell_hi).reshape(6)), int(gi), _p(out))
    return st, out
