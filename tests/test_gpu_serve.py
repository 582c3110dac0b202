"""The request server (ar_serve_*): every request's bounds are the same when it
is served in a concurrent mix as when it is rendered alone (bit-identical:
the same kernels on the same inputs, each request on its own slot stream),
also under a memory budget that admits one request at a time, and the
argument checks of the serving calls."""
import time

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


def requests():
    """A mixed set: three scenes, several resolutions and cell counts."""
    rng = np.random.default_rng(21)
    scenes = [synth.object_scene(3000, 1), synth.object_scene(800, 2), synth.cube_scene(200, 3)]
    cams = [synth.look_camera(64, 48, 70.0, centre=(0, 0, -4)), synth.look_camera(40, 40, 44.0, centre=(0, 0, -4)),
            synth.look_camera(96, 54, 90.0, centre=(0, 0, -4))]
    boxes = [([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087], [1, 1, 1, 1, 1, 2]),
             ([0.05, 0.0, 0.05, 0.0, 0.0175, 0.0], [2, 1, 2, 1, 1, 1]),
             ([0.01, 0.0, 0.0, 0.0, 0.0, 0.0], [1, 1, 1, 1, 1, 1]),
             ([0.03, 0.03, 0.0, 0.0, 0.01, 0.0], [2, 2, 1, 1, 2, 1])]
    out = []
    for i in range(10):
        si = int(rng.integers(0, 3))
        ci = int(rng.integers(0, 3))
        hw, sp = boxes[int(rng.integers(0, 4))]
        lo, hi = synth.cell_grid(hw, sp)
        out.append((si, cams[ci], lo, hi))
    return scenes, out


def alloc(cam, nc):
    o = torch.full((nc, cam.height, cam.width, 3), -3.0, dtype=torch.float32, device="cuda")
    return o, torch.full_like(o, -3.0)


def alone(ar, handles, reqs):
    res = []
    for si, cam, lo, hi in reqs:
        a, b = alloc(cam, lo.shape[0])
        handles[si].render(cam, lo, hi, a, b)
        torch.cuda.synchronize()
        res.append((a.cpu(), b.cpu()))
    return res


def serve(ar, handles, reqs, budget, slots):
    srv = ar.Server(budget, slots)
    outs, tickets = [], []
    for si, cam, lo, hi in reqs:
        a, b = alloc(cam, lo.shape[0])
        outs.append((a, b))
        t = srv.submit(handles[si], cam, lo, hi, a, b)
        assert t is not None
        tickets.append(t)
    lat = {}
    t_end = time.time() + 120
    while len(lat) < len(tickets):
        assert time.time() < t_end, "requests did not complete"
        for t in tickets:
            if t not in lat:
                done, ms = srv.poll(t)
                if done:
                    lat[t] = ms
        time.sleep(0.002)
    srv.close()
    return [(a.cpu(), b.cpu()) for a, b in outs], [lat[t] for t in tickets]


def test_mix_equals_alone(arlib):
    scenes, reqs = requests()
    handles = [arlib.Scene(s) for s in scenes]
    ref = alone(arlib, handles, reqs)
    got, lat = serve(arlib, handles, reqs, budget=4 << 30, slots=4)
    for (ra, rb), (ga, gb) in zip(ref, got):
        assert torch.equal(ra, ga) and torch.equal(rb, gb)
    assert all(x >= 0 for x in lat)


def test_tight_budget_serialises(arlib):
    scenes, reqs = requests()
    handles = [arlib.Scene(s) for s in scenes]
    ref = alone(arlib, handles, reqs[:5])
    # 2 MiB: every request is capped at the whole budget, one runs at a time
    got, _ = serve(arlib, handles, reqs[:5], budget=2 << 20, slots=3)
    for (ra, rb), (ga, gb) in zip(ref, got):
        assert torch.equal(ra, ga) and torch.equal(rb, gb)


def test_serve_arguments(arlib):
    ar = arlib
    with pytest.raises(ar.ArError):
        ar.ar_serve_create(1 << 30, 0)
    with pytest.raises(ar.ArError):
        ar.ar_serve_create(100, 2)
    srv = ar.Server(1 << 30, 2)
    with pytest.raises(ar.ArError):
        srv.poll(12345)
    w = synth.tiny64()
    sc = ar.Scene(w.scene)
    a, b = alloc(w.camera, 1)
    bad_lo, bad_hi = w.cells_hi, w.cells_lo   # lo > hi
    with pytest.raises(ar.ArError):
        srv.submit(sc, w.camera, bad_lo, bad_hi, a, b)
    t = srv.submit(sc, w.camera, w.cells_lo, w.cells_hi, a, b)
    t_end = time.time() + 60
    while True:
        done, ms = srv.poll(t)
        if done:
            break
        assert time.time() < t_end
        time.sleep(0.001)
    assert ms >= 0
    with pytest.raises(ar.ArError):
        srv.poll(t)   # retired
    srv.close()
    sc.close()


def _wait(srv, t, limit_s=60):
    t_end = time.time() + limit_s
    while True:
        done, ms = srv.poll(t)
        if done:
            return ms
        assert time.time() < t_end, "request did not complete"
        time.sleep(0.001)


def test_cancel_queued_and_running(arlib):
    """One slot busy with a long request: a request cancelled while queued
    completes with AR_ECANCELED and its outputs are untouched; the long one,
    cancelled while running, completes with AR_ECANCELED too; the server then
    serves a new request normally."""
    ar = arlib
    big = ar.Scene(synth.object_scene(100_000, 4))
    cam = synth.look_camera(400, 400, 440.0, centre=(0, 0, -4))
    lo, hi = synth.cell_grid([0.02, 0.02, 0.02, 0.0087, 0.0087, 0.0087], [2, 2, 2, 1, 1, 2])   # 16 cells
    w = synth.tiny64()
    small = ar.Scene(w.scene)
    srv = ar.Server(8 << 30, 1)
    a, b = alloc(cam, lo.shape[0])
    t_big = srv.submit(big, cam, lo, hi, a, b)
    sa, sb = alloc(w.camera, 1)
    t_small = srv.submit(small, w.camera, w.cells_lo, w.cells_hi, sa, sb)
    srv.cancel(t_small)
    srv.cancel(t_big)
    for t in (t_small, t_big):
        with pytest.raises(ar.ArError) as e:
            _wait(srv, t)
        assert e.value.code == ar.AR_ECANCELED
    torch.cuda.synchronize()
    assert torch.all(sa == -3.0) and torch.all(sb == -3.0)
    ca, cb = alloc(w.camera, 1)
    t = srv.submit(small, w.camera, w.cells_lo, w.cells_hi, ca, cb)
    assert _wait(srv, t) >= 0
    ref_a, ref_b = alloc(w.camera, 1)
    small.render(w.camera, w.cells_lo, w.cells_hi, ref_a, ref_b)
    torch.cuda.synchronize()
    assert torch.equal(ca, ref_a) and torch.equal(cb, ref_b)
    with pytest.raises(ar.ArError):
        srv.cancel(t)            # retired by the poll
    srv.close()
    big.close()
    small.close()


def test_timeout(arlib):
    """With a timeout shorter than any request, every request completes with
    AR_ETIMEOUT (in the queue or by the watchdog); with the timeout off again
    the server serves requests normally."""
    ar = arlib
    scenes, reqs = requests()
    handles = [ar.Scene(s) for s in scenes]
    srv = ar.Server(4 << 30, 2)
    srv.set_timeout(1e-3)
    tickets = []
    for si, cam, lo, hi in reqs[:6]:
        a, b = alloc(cam, lo.shape[0])
        tickets.append((srv.submit(handles[si], cam, lo, hi, a, b), a, b))
    for t, _, _ in tickets:
        with pytest.raises(ar.ArError) as e:
            _wait(srv, t)
        assert e.value.code == ar.AR_ETIMEOUT
    srv.set_timeout(0.0)
    si, cam, lo, hi = reqs[0]
    a, b = alloc(cam, lo.shape[0])
    t = srv.submit(handles[si], cam, lo, hi, a, b)
    assert _wait(srv, t) >= 0
    ra, rb = alloc(cam, lo.shape[0])
    handles[si].render(cam, lo, hi, ra, rb)
    torch.cuda.synchronize()
    assert torch.equal(a, ra) and torch.equal(b, rb)
    with pytest.raises(ar.ArError):
        srv.set_timeout(-1.0)
    with pytest.raises(ar.ArError):
        srv.cancel(987654)
    srv.close()
