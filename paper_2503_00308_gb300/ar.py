"""ctypes binding of libar (include/ar.h): same names, argument marshalling only.

Every computation runs in libar's CUDA kernels.  Loading fails loudly when the
library has not been built (there is no CPU fallback): run
``python -c "import __graft_entry__ as g; g.build()"`` first.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

AR_OK, AR_EINVAL, AR_ENOMEM, AR_EAGAIN, AR_ETIMEOUT, AR_EDEVICE, AR_ECANCELED = range(7)

c_int32, c_int64, c_float, c_double, c_void_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                 ctypes.c_double, ctypes.c_void_p)


class ar_intrinsics(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("near_plane", c_float)]


class ar_nominal_pose(ctypes.Structure):
    _fields_ = [("R_wc", c_double * 9), ("t", c_double * 3)]


class ar_pose_box(ctypes.Structure):
    _fields_ = [("lo", c_double * 6), ("hi", c_double * 6)]


class ar_render_stats(ctypes.Structure):
    _fields_ = [("n_records", c_int64), ("n_entries", c_int64), ("n_triples", c_int64),
                ("n_fallback", c_int64), ("n_launches", c_int32), ("tile", c_int32), ("m_vars", c_int32),
                ("ms_prep", c_float), ("ms_bin", c_float), ("ms_render", c_float), ("ms_total", c_float),
                ("n_evaluated", c_int64), ("n_reevaluated", c_int64), ("n_built", c_int64),
                ("n_restarted", c_int64), ("ms_build", c_float), ("n_split", c_int64),
                ("n_fp64", c_int64), ("n_fp64_segments", c_int64), ("n_graph_replays", c_int64),
                ("chunk", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ArError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libar error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """Load libar.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libar.so is not built (%s); call __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        P = c_void_p
        sig = {
            "ar_scene_create": ([P, P, P, P, P, c_int64, ctypes.c_int, P], ctypes.c_int),
            "ar_scene_destroy": ([P], ctypes.c_int),
            "ar_render_abstract": ([P, P, P, P, c_int32, c_int32, P, P, P], ctypes.c_int),
            "ar_render_abstract_host": ([P, P, P, P, c_int32, c_int32, P, P, P], ctypes.c_int),
            "ar_render_abstract_plain_fp64": ([P, P, P, P, c_int32, c_int32, P, P, P], ctypes.c_int),
            "ar_render_abstract_noalloc": ([P, P, P, P, c_int32, c_int32, P, P, P], ctypes.c_int),
            "ar_render_concrete": ([P, P, P, P, c_int32, P, P], ctypes.c_int),
            "ar_debug_records": ([P, P, P, P, P], ctypes.c_int),
            "ar_debug_alpha": ([P, P, P, P, c_int32, P, P, P, c_int32, P], ctypes.c_int),
            "ar_scene_set_boxes": ([P, P, P, P, P, P, P], ctypes.c_int),
            "ar_set_profiling": ([P, ctypes.c_int], ctypes.c_int),
            "ar_scene_set_blend": ([P, ctypes.c_int32], ctypes.c_int),
            "ar_scene_set_fp64_alpha": ([P, ctypes.c_float], ctypes.c_int),
            "ar_scene_set_graphs": ([P, ctypes.c_int32], ctypes.c_int),
            "ar_debug_set_chunk": ([P, ctypes.c_int32], ctypes.c_int),
            "ar_debug_set_entry_cap": ([P, c_int64], ctypes.c_int),
            "ar_debug_set_prefix": ([P, c_int32], ctypes.c_int),
            "ar_debug_set_cull": ([P, c_int32], ctypes.c_int),
            "ar_debug_learned_prefix": ([P, P, ctypes.c_uint64, ctypes.c_uint64, P], ctypes.c_int),
            "ar_debug_learned_window": ([P, P], ctypes.c_int),
            "ar_bounds_union": ([P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P], ctypes.c_int),
            "ar_partition_piece": ([P, P, c_int64, P], ctypes.c_int),
            "ar_render_abstract_refined": ([P, P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, P, ctypes.c_int32, P, P],
                                           ctypes.c_int),
            "ar_render_abstract_partitioned": ([P, P, P, P, P, ctypes.c_int32, P, P, P], ctypes.c_int),
            "ar_set_workspace_limit": ([P, c_int64], ctypes.c_int),
            "ar_last_render_stats": ([P, P], ctypes.c_int),
            "ar_serve_create": ([c_int64, c_int32, P], ctypes.c_int),
            "ar_serve_destroy": ([P], ctypes.c_int),
            "ar_serve_submit": ([P, P, P, P, P, c_int32, P, P, P], ctypes.c_int),
            "ar_serve_poll": ([P, ctypes.c_uint64, P, P], ctypes.c_int),
            "ar_serve_set_timeout": ([P, c_double], ctypes.c_int),
            "ar_serve_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
            "ar_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def check(code: int):
    if code != AR_OK:
        raise ArError(code, ar_last_error())
    return code


def ar_last_error() -> str:
    return lib().ar_last_error().decode()


# ------------------------------------------------------------- marshalling

def make_intrinsics(cam) -> ar_intrinsics:
    return ar_intrinsics(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx),
                         float(cam.cy), float(cam.near))


def make_pose(cam) -> ar_nominal_pose:
    p = ar_nominal_pose()
    R = np.asarray(cam.R_wc, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float64).reshape(3)
    for i in range(9):
        p.R_wc[i] = float(R[i])
    for i in range(3):
        p.t[i] = float(t[i])
    return p


def make_cells(lo, hi):
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 6)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 6)
    arr = (ar_pose_box * lo.shape[0])()
    for c in range(lo.shape[0]):
        for k in range(6):
            arr[c].lo[k] = float(lo[c, k])
            arr[c].hi[k] = float(hi[c, k])
    return arr


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def ar_scene_create(uw3, logscale3, quat4, opacity, rgb3, n: int, device_ptrs: int = 0):
    h = c_void_p()
    check(lib().ar_scene_create(_ptr(uw3), _ptr(logscale3), _ptr(quat4), _ptr(opacity), _ptr(rgb3),
                                int(n), int(device_ptrs), ctypes.byref(h)))
    return h


def ar_scene_destroy(scene):
    return check(lib().ar_scene_destroy(scene))


def ar_render_abstract(scene, intr, pose, cells, n_cells, tile, out_lower, out_upper, stream=0):
    return check(lib().ar_render_abstract(scene, ctypes.byref(intr), ctypes.byref(pose), cells, int(n_cells),
                                          int(tile), _ptr(out_lower), _ptr(out_upper), _ptr(stream)))


def ar_render_abstract_host(scene, intr, pose, cells, n_cells, tile, host_lower, host_upper, stream=0):
    return check(lib().ar_render_abstract_host(scene, ctypes.byref(intr), ctypes.byref(pose), cells,
                                               int(n_cells), int(tile), _ptr(host_lower), _ptr(host_upper),
                                               _ptr(stream)))


def ar_render_abstract_plain_fp64(scene, intr, pose, cells, n_cells, tile, out_lower, out_upper, stream=0):
    return check(lib().ar_render_abstract_plain_fp64(scene, ctypes.byref(intr), ctypes.byref(pose), cells,
                                                     int(n_cells), int(tile), _ptr(out_lower), _ptr(out_upper),
                                                     _ptr(stream)))


def ar_render_abstract_noalloc(scene, intr, pose, cells, n_cells, tile, out_lower, out_upper, stream=0):
    """The abstract render without any allocation (fixed 64 MiB scratch inside libar)."""
    return check(lib().ar_render_abstract_noalloc(scene, ctypes.byref(intr), ctypes.byref(pose), cells,
                                                  int(n_cells), int(tile), _ptr(out_lower), _ptr(out_upper),
                                                  _ptr(stream)))


def ar_bounds_union(in_lower, in_upper, n_cells, width, height, out_lower, out_upper, stream=0):
    """Elementwise min / max over cells of device bounds [n_cells, H, W, 3] into [H, W, 3]."""
    return check(lib().ar_bounds_union(_ptr(in_lower), _ptr(in_upper), int(n_cells), int(width), int(height),
                                       _ptr(out_lower), _ptr(out_upper), _ptr(stream)))


def ar_render_abstract_partitioned(scene, intr, pose, box, parts, tile, out_lower, out_upper, stream=0):
    """Bounds of one pose box (an ar_pose_box) from parts[k] pieces along each
    pose dimension, joined into device [H, W, 3] outputs."""
    p = (ctypes.c_int32 * 6)(*[int(v) for v in parts])
    return check(lib().ar_render_abstract_partitioned(scene, ctypes.byref(intr), ctypes.byref(pose), ctypes.byref(box),
                                                      p, int(tile), _ptr(out_lower), _ptr(out_upper), _ptr(stream)))


def ar_partition_piece(box, parts, index: int):
    """Piece `index` of the partition of an ar_pose_box into parts[k] pieces per
    dimension: returns (lo [6], hi [6]).  Host only."""
    p = (ctypes.c_int32 * 6)(*[int(v) for v in parts])
    out = ar_pose_box()
    check(lib().ar_partition_piece(ctypes.byref(box), p, int(index), ctypes.byref(out)))
    return np.array(list(out.lo)), np.array(list(out.hi))


def ar_render_abstract_refined(scene, intr, pose, box, rounds, tile, out_lower, out_upper, stream=0,
                               leaves_cap: int = 4096):
    """Bounds of one pose box (an ar_pose_box) from an adaptive partition
    into device [H, W, 3] outputs; returns the last round's pieces as
    (lo [n, 6], hi [n, 6]) arrays."""
    buf = (ar_pose_box * leaves_cap)()
    n = ctypes.c_int32(0)
    check(lib().ar_render_abstract_refined(scene, ctypes.byref(intr), ctypes.byref(pose), ctypes.byref(box),
                                           int(rounds), int(tile), _ptr(out_lower), _ptr(out_upper), buf,
                                           int(leaves_cap), ctypes.byref(n), _ptr(stream)))
    k = min(n.value, leaves_cap)
    lo = np.array([[buf[i].lo[j] for j in range(6)] for i in range(k)]).reshape(k, 6)
    hi = np.array([[buf[i].hi[j] for j in range(6)] for i in range(k)]).reshape(k, 6)
    return lo, hi


def ar_render_concrete(scene, intr, pose, deltas, n_poses, out, stream=0):
    d = np.ascontiguousarray(deltas, dtype=np.float64)
    return check(lib().ar_render_concrete(scene, ctypes.byref(intr), ctypes.byref(pose), d.ctypes.data,
                                          int(n_poses), _ptr(out), _ptr(stream)))


def ar_debug_records(scene, intr, pose, cell, n: int) -> np.ndarray:
    """Decision part of the records of one cell: [n, 10] (valid, straddle,
    k_lo, k_hi, px0, px1, py0, py1, mu_x, mu_y)."""
    out = np.zeros((n, 10), dtype=np.float64)
    check(lib().ar_debug_records(scene, ctypes.byref(intr), ctypes.byref(pose), ctypes.byref(cell), out.ctypes.data))
    return out


def ar_debug_alpha(scene, intr, pose, cell, gi, px, py, precision: int = 0) -> np.ndarray:
    gi = np.ascontiguousarray(gi, dtype=np.int64).reshape(-1)
    px = np.ascontiguousarray(px, dtype=np.int32).reshape(-1)
    py = np.ascontiguousarray(py, dtype=np.int32).reshape(-1)
    n = gi.size
    out = np.zeros((n, 40), dtype=np.float64)
    check(lib().ar_debug_alpha(scene, ctypes.byref(intr), ctypes.byref(pose), ctypes.byref(cell), n,
                               _ptr(gi), _ptr(px), _ptr(py), int(precision), _ptr(out)))
    return out


def ar_set_workspace_limit(scene, nbytes: int):
    return check(lib().ar_set_workspace_limit(scene, int(nbytes)))


def ar_set_profiling(scene, on: bool):
    return check(lib().ar_set_profiling(scene, 1 if on else 0))


AR_BLEND_INTERVAL, AR_BLEND_RELATIONAL = 0, 1


def ar_scene_set_blend(scene, mode: int):
    return check(lib().ar_scene_set_blend(scene, int(mode)))


def ar_scene_set_fp64_alpha(scene, threshold: float):
    return check(lib().ar_scene_set_fp64_alpha(scene, float(threshold)))


def ar_scene_set_graphs(scene, on: bool):
    return check(lib().ar_scene_set_graphs(scene, 1 if on else 0))


def ar_debug_set_chunk(scene, chunk: int):
    return check(lib().ar_debug_set_chunk(scene, int(chunk)))


def ar_debug_set_entry_cap(scene, cap: int):
    return check(lib().ar_debug_set_entry_cap(scene, int(cap)))


def ar_debug_set_prefix(scene, shift: int):
    return check(lib().ar_debug_set_prefix(scene, int(shift)))


def ar_debug_set_cull(scene, mode: int):
    return check(lib().ar_debug_set_cull(scene, int(mode)))


def ar_debug_learned_prefix(weights, counts, n_entries: int, n_events: int) -> int:
    """The depth-prefix shift learned from 64-bucket stop statistics (host only)."""
    w = np.ascontiguousarray(weights, dtype=np.uint64)
    c = np.ascontiguousarray(counts, dtype=np.uint32)
    if w.shape != (64,) or c.shape != (64,):
        raise ValueError("weights and counts must have 64 entries")
    out = c_int32()
    check(lib().ar_debug_learned_prefix(_ptr(w), _ptr(c), int(n_entries), int(n_events), ctypes.byref(out)))
    return out.value


def ar_debug_learned_window(hist) -> int:
    """The first round's record window learned from a 256-bucket sweep histogram (host only)."""
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    if h.shape != (256,):
        raise ValueError("hist must have 256 entries")
    out = ctypes.c_uint32()
    check(lib().ar_debug_learned_window(_ptr(h), ctypes.byref(out)))
    return out.value


def ar_last_render_stats(scene) -> dict:
    st = ar_render_stats()
    check(lib().ar_last_render_stats(scene, ctypes.byref(st)))
    return st.as_dict()


def ar_serve_create(hbm_budget_bytes: int, n_slots: int):
    h = c_void_p()
    check(lib().ar_serve_create(int(hbm_budget_bytes), int(n_slots), ctypes.byref(h)))
    return h


def ar_serve_destroy(server):
    return check(lib().ar_serve_destroy(server))


def ar_serve_submit(server, scene, intr, pose, cells, n_cells, out_lower, out_upper):
    """Returns the ticket, or None when admission is refused (AR_EAGAIN)."""
    t = ctypes.c_uint64()
    r = lib().ar_serve_submit(server, scene, ctypes.byref(intr), ctypes.byref(pose), cells, int(n_cells),
                              _ptr(out_lower), _ptr(out_upper), ctypes.byref(t))
    if r == AR_EAGAIN:
        return None
    check(r)
    return int(t.value)


def ar_serve_poll(server, ticket: int):
    """Returns (done, latency_ms)."""
    done = ctypes.c_int()
    lat = ctypes.c_double()
    check(lib().ar_serve_poll(server, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), float(lat.value)


def ar_serve_set_timeout(server, timeout_ms: float):
    return check(lib().ar_serve_set_timeout(server, float(timeout_ms)))


def ar_serve_cancel(server, ticket: int):
    return check(lib().ar_serve_cancel(server, ctypes.c_uint64(ticket)))


# ------------------------------------------------------------ conveniences

class Scene:
    """Owns an ar_scene handle created from a synth.Scene-like record (host arrays)."""

    def __init__(self, sc):
        self._arrays = [np.ascontiguousarray(a, dtype=np.float32) for a in
                        (sc.uw, sc.logscale, sc.quat, sc.opacity, sc.rgb)]
        self.n = int(self._arrays[0].shape[0])
        self.handle = ar_scene_create(*self._arrays, self.n, 0)

    def close(self):
        if self.handle is not None:
            ar_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cam, cells_lo, cells_hi, out_lower, out_upper, tile: int = 0, stream=0):
        cells = make_cells(cells_lo, cells_hi)
        ar_render_abstract(self.handle, make_intrinsics(cam), make_pose(cam), cells, len(cells), tile,
                           out_lower, out_upper, stream)

    def render_concrete(self, cam, deltas, out, stream=0):
        """Concrete renders at the poses deltas ([n][6]) into out ([n][H][W][3], device)."""
        d = np.ascontiguousarray(np.asarray(deltas, dtype=np.float64).reshape(-1, 6))
        ar_render_concrete(self.handle, make_intrinsics(cam), make_pose(cam), d, d.shape[0], out, stream)

    def set_boxes(self, boxes=None):
        """Scene-parameter boxes (a dict of float32 arrays uw_lo, uw_hi, o_lo,
        o_hi, c_lo, c_hi, any pair may be missing), or None for the nominal scene."""
        b = boxes or {}
        keep = []

        def arr(k):
            if k not in b:
                return None
            a = np.ascontiguousarray(b[k], dtype=np.float32)
            keep.append(a)
            return a.ctypes.data

        check(lib().ar_scene_set_boxes(self.handle, arr("uw_lo"), arr("uw_hi"), arr("o_lo"), arr("o_hi"),
                                       arr("c_lo"), arr("c_hi")))

    def debug_records(self, cam, cell_lo, cell_hi) -> np.ndarray:
        cells = make_cells(np.reshape(cell_lo, (1, 6)), np.reshape(cell_hi, (1, 6)))
        return ar_debug_records(self.handle, make_intrinsics(cam), make_pose(cam), cells[0], self.n)

    def debug_alpha(self, cam, cell_lo, cell_hi, gi, px, py, precision: int = 0) -> np.ndarray:
        cells = make_cells(np.reshape(cell_lo, (1, 6)), np.reshape(cell_hi, (1, 6)))
        return ar_debug_alpha(self.handle, make_intrinsics(cam), make_pose(cam), cells[0], gi, px, py, precision)

    def render_plain_fp64(self, cam, cells_lo, cells_hi, out_lower, out_upper, tile: int = 0, stream=0):
        cells = make_cells(cells_lo, cells_hi)
        ar_render_abstract_plain_fp64(self.handle, make_intrinsics(cam), make_pose(cam), cells, len(cells), tile,
                                      out_lower, out_upper, stream)


class Server:
    """Owns an ar_server handle (continuous batching over n_slots streams)."""

    def __init__(self, hbm_budget_bytes: int, n_slots: int):
        self.handle = ar_serve_create(hbm_budget_bytes, n_slots)

    def submit(self, scene: "Scene", cam, cells_lo, cells_hi, out_lower, out_upper):
        cells = make_cells(cells_lo, cells_hi)
        return ar_serve_submit(self.handle, scene.handle, make_intrinsics(cam), make_pose(cam), cells, len(cells),
                               out_lower, out_upper)

    def poll(self, ticket: int):
        return ar_serve_poll(self.handle, ticket)

    def set_timeout(self, timeout_ms: float):
        return ar_serve_set_timeout(self.handle, timeout_ms)

    def cancel(self, ticket: int):
        return ar_serve_cancel(self.handle, ticket)

    def close(self):
        if self.handle is not None:
            ar_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
