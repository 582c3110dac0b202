"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests re-types the oracle's formulas: each compares it with a
closed form worked by hand, an independent textbook formulation (EWA splatting
with scipy's rotations), a lemma of the paper (Lemma 1, Lemma 2, Theorem 1),
brute force over sampled or gridded poses, or a number printed in the paper
(Example 1, Sec. 4.5).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2503_00308_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _form(coeffs, k):
    f = np.zeros(7)
    f[: len(coeffs)] = coeffs
    f[6] = k
    return f


def _eval(f, p):
    return float(np.dot(f[:6], p) + f[6])


# --------------------------------------------------------------- relaxations

def test_mul_closed_form(orc):
    # x in [1, 3] = 2 + p0 ; y in [-2, 4] = 1 + 3 p1 (worked by hand):
    # lower plane x + 2y - 5, upper plane x + 2y + 1 (averaged McCormick planes)
    x = np.concatenate([_form([1], 2), _form([1], 2)])
    y = np.concatenate([_form([0, 3], 1), _form([0, 3], 1)])
    r = orc.relax_mul(x, y)
    np.testing.assert_allclose(r[:7], _form([1, 6], -1), atol=1e-14)
    np.testing.assert_allclose(r[7:], _form([1, 6], 5), atol=1e-14)


def test_square_closed_form(orc):
    # x in [1, 3] = 2 + p0: tangent at 2 -> 4x - 4 ; secant -> 4x - 3
    x = np.concatenate([_form([1], 2), _form([1], 2)])
    r = orc.relax_sq(x)
    np.testing.assert_allclose(r[:7], _form([4], 4), atol=1e-14)
    np.testing.assert_allclose(r[7:], _form([4], 5), atol=1e-14)
    # interval straddling zero: x in [-1, 3] = 1 + 2 p0: tangent at 1 -> 2x - 1 ; secant 2x + 3
    x = np.concatenate([_form([2], 1), _form([2], 1)])
    r = orc.relax_sq(x)
    np.testing.assert_allclose(r[:7], _form([4], 1), atol=1e-14)
    np.testing.assert_allclose(r[7:], _form([4], 5), atol=1e-14)


def _bs(lo, hi):
    return np.concatenate([lo, hi])


def test_exp_closed_form(orc):
    """Table 2's Exp: tangent at the lower end below, secant above (worked by hand)."""
    e2, e1, e3 = math.exp(-2), math.exp(-1), math.exp(-3)
    # x in [-2, 0] = -1 + p0: lower e^-2 (1 + x + 2) = e^-2 (p0 + 2);
    # upper e^-2 + s (x + 2) with s = (1 - e^-2) / 2, i.e. s p0 + (e^-2 + s)
    x = _bs(_form([1], -1), _form([1], -1))
    r = orc.relax_exp(x)
    s = (1 - e2) / 2
    np.testing.assert_allclose(r[:7], _form([e2], 2 * e2), rtol=0, atol=1e-15)
    np.testing.assert_allclose(r[7:], _form([s], e2 + s), rtol=0, atol=1e-15)
    # distinct lower and upper forms: x.lo = -2.5 + 0.5 p0 (min -3), x.hi = -1.5 + 0.5 p0 (max -1):
    # lower e^-3 (1 + x.lo + 3) = e^-3 (1.5 + 0.5 p0);
    # upper e^-3 + s (x.hi + 3) = e^-3 + s (1.5 + 0.5 p0), s = (e^-1 - e^-3) / 2
    x = _bs(_form([0.5], -2.5), _form([0.5], -1.5))
    r = orc.relax_exp(x)
    s = (e1 - e3) / 2
    np.testing.assert_allclose(r[:7], _form([0.5 * e3], 1.5 * e3), rtol=0, atol=1e-15)
    np.testing.assert_allclose(r[7:], _form([0.5 * s], e3 + 1.5 * s), rtol=0, atol=1e-15)
    # x in [-1, 1] = p0: the argument is -m/2 <= 0, so the secant ends at 0:
    # lower e^-1 (p0 + 2); upper e^-1 + (1 - e^-1)(p0 + 1)
    x = _bs(_form([1], 0), _form([1], 0))
    r = orc.relax_exp(x)
    np.testing.assert_allclose(r[:7], _form([e1], 2 * e1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(r[7:], _form([1 - e1], 1.0), rtol=0, atol=1e-15)
    # a point: both sides are the constant e^-0.7
    x = _bs(_form([], -0.7), _form([], -0.7))
    r = orc.relax_exp(x)
    np.testing.assert_allclose(r, _bs(_form([], math.exp(-0.7)), _form([], math.exp(-0.7))), rtol=0, atol=1e-15)


def test_exp_relaxation_sound_and_tight_at_ends(orc):
    """Soundness on random forms with x <= 0, and the closed form's own
    property: the lower form touches exp at the lower end of the interval,
    the upper one at both ends."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        c = rng.normal(size=6) * rng.uniform(0, 1, size=6)
        lo = _form(c, -np.sum(np.abs(c)) - rng.uniform(0, 4))
        hi = lo.copy()
        hi[6] += rng.uniform(0, 0.5)
        hi[6] = min(hi[6], -np.sum(np.abs(c)))          # x_hi <= 0 at every p
        r = orc.relax_exp(_bs(lo, hi))
        for _ in range(30):
            p = rng.uniform(-1, 1, size=6)
            xv = _eval(lo, p) + rng.uniform() * (_eval(hi, p) - _eval(lo, p))
            v = math.exp(xv)
            assert _eval(r[:7], p) <= v + 1e-12 and v <= _eval(r[7:], p) + 1e-12
        xl, xu = lo[6] - np.sum(np.abs(lo[:6])), hi[6] + np.sum(np.abs(hi[:6]))
        # concretised lower bound = exp(x_lo); upper bound = exp(x_hi)
        assert abs((r[6] - np.sum(np.abs(r[:6]))) - math.exp(xl)) < 1e-12
        assert abs((r[13] + np.sum(np.abs(r[7:13]))) - math.exp(xu)) < 1e-12


TAU = lambda o: 2 * math.log(255 * o)   # noqa: E731  (cutoff: o exp(-m/2) >= 1/255 iff m <= tau)


def test_alpha_stage_closed_form(orc):
    """a = o Exp(-m/2) with m in [2, 6] = 4 + 2 p0 and o = 0.8, far from the
    cutoff and the clip: x = -m/2 in [-3, -1], x.lo = x.hi = -2 - p0, so
    lower 0.8 e^-3 (1 + x + 3) = 0.8 e^-3 (2 - p0) and upper
    0.8 (e^-3 + s (x + 3)) = 0.8 (e^-3 + s (1 - p0)), s = (e^-1 - e^-3) / 2."""
    e1, e3 = math.exp(-1), math.exp(-3)
    s = (e1 - e3) / 2
    m = _bs(_form([2], 4), _form([2], 4))
    r = orc.alpha_from_m(m, 0.8, 0.8, TAU(0.8), TAU(0.8))
    np.testing.assert_allclose(r["L"], _form([-0.8 * e3], 1.6 * e3), rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["U"], _form([-0.8 * s], 0.8 * (e3 + s)), rtol=0, atol=1e-15)
    assert abs(r["alo"] - 0.8 * e3) < 1e-15 and abs(r["ahi"] - 0.8 * e1) < 1e-15
    assert r["ramp"] == 0.5
    # a near-plane straddle keeps the upper side and drops the lower one
    r = orc.alpha_from_m(m, 0.8, 0.8, TAU(0.8), TAU(0.8), straddle=True)
    np.testing.assert_allclose(r["L"], _form([], 0.0), rtol=0, atol=0)
    np.testing.assert_allclose(r["U"], _form([-0.8 * s], 0.8 * (e3 + s)), rtol=0, atol=1e-15)
    assert r["alo"] == 0.0


def test_alpha_lower_cutoff_ramp_closed_form(orc):
    """m in [8, 10.5] = 9.25 + 1.25 p0, o = 0.8, tau = 2 ln 204 = 10.636...:
    m_hi < tau, within the ramp of width 0.5 below it, so the lower form loses
    psi/255 with psi = (10.5 - tau + 0.5) / 0.5 = 2 (11 - tau); the upper form
    is untouched.  x.lo = x.hi = -4.625 - 0.625 p0, x in [-5.25, -4]."""
    tau = TAU(0.8)
    psi = 2 * (11 - tau)
    assert 0.7275 < psi < 0.7276
    e525, e4 = math.exp(-5.25), math.exp(-4)
    s = (e4 - e525) / 1.25
    m = _bs(_form([1.25], 9.25), _form([1.25], 9.25))
    r = orc.alpha_from_m(m, 0.8, 0.8, tau, tau)
    # lower: 0.8 e^-5.25 (1 + x + 5.25) - psi/255 = 0.8 e^-5.25 (1.625 - 0.625 p0) - psi/255 (> 0 on the cell)
    np.testing.assert_allclose(r["L"], _form([-0.5 * e525], 1.3 * e525 - psi / 255), rtol=0, atol=1e-15)
    assert abs(r["alo"] - (0.8 * e525 - psi / 255)) < 1e-15
    # upper: 0.8 (e^-5.25 + s (x + 5.25)) = 0.8 (e^-5.25 + s (0.625 - 0.625 p0))
    np.testing.assert_allclose(r["U"], _form([-0.5 * s], 0.8 * (e525 + 0.625 * s)), rtol=0, atol=1e-15)


def test_alpha_upper_cutoff_ramp_closed_form(orc):
    """m in [11, 12] = 11.5 + 0.5 p0, o = 0.8 (tau = 10.636...): m_lo > tau, so
    the upper form is scaled by 1 - psi2, psi2 = (11 - tau) / 0.5; m_hi > tau,
    so the lower form loses 1/255, and since 0.8 e^-6 (1 + x + 6) <= 1.2 e^-6
    < 1/255 on the cell, it is replaced by 0.  x = -5.75 - 0.25 p0."""
    tau = TAU(0.8)
    psi2 = 2 * (11 - tau)
    e6, e55 = math.exp(-6), math.exp(-5.5)
    s = (e55 - e6) / 0.5
    m = _bs(_form([0.5], 11.5), _form([0.5], 11.5))
    r = orc.alpha_from_m(m, 0.8, 0.8, tau, tau)
    keep = 1 - psi2
    # upper: keep * 0.8 (e^-6 + s (x + 6)) = keep * 0.8 (e^-6 + s (0.25 - 0.25 p0))
    np.testing.assert_allclose(r["U"], _form([-keep * 0.2 * s], keep * 0.8 * (e6 + 0.25 * s)), rtol=0, atol=1e-15)
    np.testing.assert_allclose(r["L"], _form([], 0.0), rtol=0, atol=0)
    assert r["alo"] == 0.0 and abs(r["ahi"] - keep * 0.8 * e55) < 1e-15


def test_alpha_clip_ramp_closed_form(orc):
    """A lower m form that dips below 0 (m.lo = 1 + 2 p0, min -1; m.hi = 5 + 2 p0,
    max 7) with o = 0.6: x_lo = -3.5 and the secant ends at x = 0, so the upper
    form 0.6 (e^-3.5 + s (x.hi + 3.5)), s = (1 - e^-3.5) / 3.5, x.hi = -0.5 - p0,
    peaks at 0.6 (e^-3.5 + 4 s) > 0.6.  It is blended toward the constant 0.6
    with lam = (1.25 - (e^-3.5 + 4 s)) / 0.25."""
    e35 = math.exp(-3.5)
    s = (1 - e35) / 3.5
    lam = (1.25 - (e35 + 4 * s)) / 0.25
    assert 0.44 < lam < 0.45
    m = _bs(_form([2], 1), _form([2], 5))
    r = orc.alpha_from_m(m, 0.6, 0.6, TAU(0.6), TAU(0.6))
    np.testing.assert_allclose(r["U"], _form([-0.6 * lam * s], lam * 0.6 * (e35 + 3 * s) + (1 - lam) * 0.6),
                               rtol=0, atol=1e-15)
    assert r["ahi"] == 0.6
    # lower: 0.6 e^-3.5 (1 + x.lo + 3.5), x.lo = -2.5 - p0, i.e. 0.6 e^-3.5 (2 - p0) (m_hi = 7 is far below tau)
    np.testing.assert_allclose(r["L"], _form([-0.6 * e35], 1.2 * e35), rtol=0, atol=1e-15)


def test_alpha_negative_lower_blend_closed_form(orc):
    """m in [7, 9] = 8 + p0 with o = 0.3 (tau = 2 ln 76.5 = 8.67...): m_hi > tau
    takes 1/255 off the lower form 0.3 e^-4.5 (1.5 - 0.5 p0), which then spans
    [0.3 e^-4.5 - 1/255, 0.6 e^-4.5 - 1/255] across 0, so it is scaled by
    mu = max / (max - min) = (0.6 e^-4.5 - 1/255) / (0.3 e^-4.5)."""
    e45 = math.exp(-4.5)
    lmax, lmin = 0.6 * e45 - 1 / 255, 0.3 * e45 - 1 / 255
    assert lmin < 0 < lmax
    mu = lmax / (lmax - lmin)
    m = _bs(_form([1], 8), _form([1], 8))
    r = orc.alpha_from_m(m, 0.3, 0.3, TAU(0.3), TAU(0.3))
    np.testing.assert_allclose(r["L"], _form([-0.15 * e45 * mu], mu * (0.45 * e45 - 1 / 255)), rtol=0, atol=1e-15)
    assert r["alo"] == 0.0


def test_pixel_alpha_closed_form_flat_gaussian(orc):
    """One Gaussian through the whole record chain with a Mahalanobis term
    known in closed form.  Camera at (0, 0, -3) looking down +z (R0 = I),
    fx = fy = 32, principal point (16, 16); the Gaussian at (a, b, 0) has
    identity rotation, scales (sx, sy, e^-30): flat along the view axis, so
    Mp = J Mc = diag(3 fx sx, 3 fy sy) up to terms of order e^-30, X and Conic
    are constant and W = diag(1 / (3 fx sx), 1 / (3 fy sy)).  On a cell
    tx = h p0, Delta_x = 9 (u - cx) - 3 fx (a - h p0) and Delta_y is constant,
    so q0 = alpha + beta p0 with alpha = (3 (ux - cx) - fx a) / (fx sx),
    beta = h / sx, and q1 = gamma = (3 (uy - cy) - fy b) / (fy sy).  The square
    relaxation then gives m.lo = alpha^2 + gamma^2 + 2 alpha beta p0 (tangent at
    alpha) and m.hi = m.lo + beta^2 (secant), and Table 2's Exp on
    x = -m/2 gives a's forms."""
    a, b, h, o = 0.05, -0.03, 0.01, 0.7
    ls = -2.5
    sc = synth.Scene(np.array([[a, b, 0.0]], np.float32), np.array([[ls, ls, -30.0]], np.float32),
                     np.array([[1, 0, 0, 0]], np.float32), np.array([o], np.float32),
                     np.array([[0.2, 0.5, 0.9]], np.float32))
    cam = synth.look_camera(32, 32, 32.0, centre=(0, 0, -3))
    assert np.array_equal(cam.R_wc, np.eye(3)) and cam.cx == 16 and cam.fx == 32
    a, b, o = float(sc.uw[0, 0]), float(sc.uw[0, 1]), float(sc.opacity[0])
    sx = math.exp(float(sc.logscale[0, 0]))
    lo = np.array([-h, 0, 0, 0, 0, 0])
    px, py = 16, 15
    r = orc.pixel_alpha(sc, cam, lo, -lo, 0, px, py)
    assert r is not None and not r["fallback"] and not r["straddle"]
    al = (3 * (px + 0.5 - 16) - 32 * a) / (32 * sx)
    be = h / sx
    ga = (3 * (py + 0.5 - 16) - 32 * b) / (32 * sx)
    mlo_form = _form([2 * al * be], al * al + ga * ga)
    mhi_form = _form([2 * al * be], al * al + be * be + ga * ga)
    np.testing.assert_allclose(r["m"], _bs(mlo_form, mhi_form), rtol=0, atol=1e-11)
    mlo = al * al + ga * ga - 2 * abs(al * be)
    mhi = al * al + be * be + ga * ga + 2 * abs(al * be)
    assert 0 < mlo < mhi < 0.1
    # x = -m/2 in [-mhi/2, -mlo/2]; lower o E (1 + x.lo - xl), upper o (E + s (x.hi - xl))
    xl, xu = -mhi / 2, -mlo / 2
    E = math.exp(xl)
    s = (math.exp(xu) - E) / (xu - xl)
    L = _form([-o * E * al * be], o * E * (1 - xl - (al * al + be * be + ga * ga) / 2))
    U = _form([-o * s * al * be], o * (E - s * xl - s * (al * al + ga * ga) / 2))
    np.testing.assert_allclose(r["L"], L, rtol=0, atol=1e-11)
    np.testing.assert_allclose(r["U"], U, rtol=0, atol=1e-11)
    assert abs(r["alo"] - o * math.exp(-mhi / 2)) < 1e-11 and abs(r["ahi"] - o * math.exp(-mlo / 2)) < 1e-11


def _random_bs(rng, scale=1.0):
    lo = _form(rng.normal(size=6) * scale * rng.uniform(0, 1, size=6), rng.normal() * 2 * scale)
    hi = lo.copy()
    hi[:6] += rng.normal(size=6) * 0.1 * scale
    hi[6] += np.sum(np.abs(hi[:6] - lo[:6])) + rng.uniform(0, 0.5) * scale
    return np.concatenate([lo, hi])


@pytest.mark.parametrize("op", ["mul", "sq"])
def test_relaxations_sound_random(orc, op):
    rng = np.random.default_rng(7)
    for _ in range(300):
        x = _random_bs(rng)
        y = _random_bs(rng)
        r = orc.relax_mul(x, y) if op == "mul" else orc.relax_sq(x)
        for _ in range(40):
            p = rng.uniform(-1, 1, size=6)
            xv = _eval(x[:7], p) + rng.uniform() * (_eval(x[7:], p) - _eval(x[:7], p))
            yv = _eval(y[:7], p) + rng.uniform() * (_eval(y[7:], p) - _eval(y[:7], p))
            v = xv * yv if op == "mul" else xv * xv
            assert _eval(r[:7], p) <= v + 1e-9 * (1 + abs(v))
            assert v <= _eval(r[7:], p) + 1e-9 * (1 + abs(v))


def test_mul_exact_when_one_operand_is_constant(orc):
    rng = np.random.default_rng(3)
    x = _random_bs(rng)
    c = np.concatenate([_form([], 2.5), _form([], 2.5)])
    r = orc.relax_mul(x, c)
    np.testing.assert_allclose(r, 2.5 * x, atol=1e-12)


def test_rotation_forms_contain_rotations(orc):
    rng = np.random.default_rng(11)
    for _ in range(20):
        ctr = rng.uniform(-0.3, 0.3, size=6)
        h = rng.uniform(0, 0.05, size=6)
        F = orc.rot_forms(ctr - h, ctr + h)
        for _ in range(50):
            p = rng.uniform(-1, 1, size=6)
            th = ctr[3:] + h[3:] * p[3:]
            R = Rotation.from_euler("XYZ", th).as_matrix()  # intrinsic X then Y then Z = Rx Ry Rz
            for e in range(9):
                v = R.flat[e]
                assert _eval(F[e, :7], p) <= v + 1e-12
                assert v <= _eval(F[e, 7:], p) + 1e-12
    # point cell: exact
    th = np.array([0, 0, 0, 0.1, -0.2, 0.3])
    F = orc.rot_forms(th, th)
    R = Rotation.from_euler("XYZ", th[3:]).as_matrix()
    np.testing.assert_allclose(F[:, 6], R.reshape(9), atol=1e-14)
    np.testing.assert_allclose(F[:, 13], R.reshape(9), atol=1e-14)


# ----------------------------------------------------------------- MatrixInv

def _inverse_hull(Xl, Xu, n=41, symmetric=False):
    Xl = np.asarray(Xl)
    Xu = np.asarray(Xu)
    g = [np.linspace(Xl.flat[e], Xu.flat[e], n) for e in range(4)]
    if symmetric:
        a, b, d = np.meshgrid(g[0], g[1], g[3], indexing="ij")
        M = np.stack([a, b, b, d], axis=-1).reshape(-1, 2, 2)
    else:
        a, b, c, d = np.meshgrid(*g, indexing="ij")
        M = np.stack([a, b, c, d], axis=-1).reshape(-1, 2, 2)
    inv = np.linalg.inv(M)
    return inv.min(axis=0), inv.max(axis=0)


def test_example1_matrixinv(orc):
    ex = json.load(open(os.path.join(GOLDEN, "matrixinv_example1.json")))
    Xl, Xu = np.array(ex["X_lower"]), np.array(ex["X_upper"])
    hl, hu = _inverse_hull(Xl, Xu)
    # the empirical width printed in Example 1 (reading -0.2 as -0.02)
    assert abs(np.linalg.norm(hu - hl) - ex["printed_width_empirical"]) < 0.01
    lo, hi, rho = orc.matrixinv_interval(Xl, Xu, k=8)
    assert rho < 1
    assert np.all(lo <= hl + 1e-12) and np.all(hi >= hu - 1e-12)     # Lemma 1 over the box
    width = np.linalg.norm(hi - lo)
    # tighter than the adjugate method's printed width, and near the printed MatrixInv width
    assert width < ex["printed_width_adjugate"]
    assert ex["printed_width_matrixinv"] - 0.05 < width < 0.85


def test_sec45_conic_contains_hull(orc):
    ex = json.load(open(os.path.join(GOLDEN, "conic_sec45.json")))
    Cl, Cu = np.array(ex["Cov_lower"]), np.array(ex["Cov_upper"])
    hl, hu = _inverse_hull(Cl, Cu, n=61, symmetric=True)
    lo, hi, rho = orc.matrixinv_interval(Cl, Cu, k=8, symmetric=True)
    assert np.all(lo <= hl + 1e-9) and np.all(hi >= hu - 1e-9)
    # the hull itself overlaps the printed conic box (same ballpark, same signs)
    pl, pu = np.array(ex["printed_conic_lower"]), np.array(ex["printed_conic_upper"])
    assert np.all(np.sign(pl) == np.sign(hl)) and np.all(np.sign(pu) == np.sign(hu))
    assert np.all(np.abs(hl - pl) < 5) and np.all(np.abs(hu - pu) < 5)


def test_lemma1_random_boxes(orc):
    rng = np.random.default_rng(5)
    done = 0
    while done < 40:
        A = rng.normal(size=(2, 2))
        C = A @ A.T + 0.5 * np.eye(2)
        W = np.abs(rng.normal(size=(2, 2))) * 0.03 * np.abs(C).max()
        Xl, Xu = C - W, C + W
        r = orc.matrixinv_interval(Xl, Xu, k=8)
        if r is None:
            continue
        lo, hi, rho = r
        M = Xl + (Xu - Xl) * rng.uniform(size=(500, 2, 2))
        inv = np.linalg.inv(M)
        assert np.all(inv >= lo - 1e-10) and np.all(inv <= hi + 1e-10)
        done += 1


def test_matrixinv_point_is_inverse(orc):
    X = np.array([[2.0, 0.3], [0.3, 1.5]])
    lo, hi, rho = orc.matrixinv_interval(X, X, k=8)
    np.testing.assert_allclose(lo, np.linalg.inv(X), atol=1e-13)
    np.testing.assert_allclose(hi, np.linalg.inv(X), atol=1e-13)


def test_matrixinv_rejects_wide_box(orc):
    # the assertion of Algorithm 3 fails when ||I - X X0|| >= 1
    assert orc.matrixinv_interval([[0.1, -1], [-1, 0.1]], [[2, 1], [1, 2]]) is None
    # the box holds singular matrices (x = y = 1, z = 1), so no piece of it
    # can pass the assertion either: input splitting fails too
    assert orc.matrixinv_cell([[0.1, -1], [-1, 0.1]], [[2, 1], [1, 2]], symmetric=True) is None


# ------------------------------------------ MatrixInv adjustments of Sec. 3.1

def test_matrixinv_adaptive_order_example1(orc):
    # adjustment (3): k grows from the default 8 until Eps <= 2^-24 ||X0||_F.
    # Worked by hand for Example 1 (rho = 0.2722): rho^(k+1) / (1 - rho) <=
    # 5.96e-8 needs k + 1 >= ln(4.34e-8) / ln(0.2722) = 13.03, so k = 13.
    ex = json.load(open(os.path.join(GOLDEN, "matrixinv_example1.json")))
    Xl, Xu = np.array(ex["X_lower"]), np.array(ex["X_upper"])
    lo, hi, info = orc.matrixinv_cell(Xl, Xu, symmetric=True)
    assert info["pieces"] == 0 and abs(info["rho"] - 0.2722) < 1e-4
    assert info["k"] == 13
    hl, hu = _inverse_hull(Xl, Xu, symmetric=True)
    assert np.all(lo <= hl + 1e-12) and np.all(hi >= hu - 1e-12)     # Lemma 1 over the box
    lo8, hi8, _ = orc.matrixinv_interval(Xl, Xu, k=8, symmetric=True)
    assert np.linalg.norm(hi - lo) <= np.linalg.norm(hi8 - lo8)       # a smaller remainder


def test_matrixinv_split_diagonal_box(orc):
    # X = diag(x, y) with x, y in [0.5, 4]: the centre is 2.25 I, so I - X X0
    # = diag(1 - x/2.25, 1 - y/2.25) with entries up to 1.75/2.25, and
    # rho = sqrt(2) 0.7778 = 1.0999 >= 1 (worked by hand): the assertion of
    # Algorithm 3 fails on the whole box and the input range is divided
    Xl = np.array([[0.5, 0.0], [0.0, 0.5]])
    Xu = np.array([[4.0, 0.0], [0.0, 4.0]])
    assert orc.matrixinv_interval(Xl, Xu, k=8, symmetric=True) is None
    lo, hi, info = orc.matrixinv_cell(Xl, Xu, symmetric=True)
    assert abs(info["rho"] - math.sqrt(2) * 1.75 / 2.25) < 1e-12
    assert 2 <= info["pieces"] <= 64
    # the exact hull of the inverse: diag([1/4, 2], [1/4, 2]) with a zero off-diagonal
    assert lo[0, 0] <= 0.25 and hi[0, 0] >= 2.0 and lo[1, 1] <= 0.25 and hi[1, 1] >= 2.0
    assert lo[0, 1] <= 0.0 <= hi[0, 1] and lo[1, 0] <= 0.0 <= hi[1, 0]


def test_matrixinv_split_brute_force(orc):
    # positive definite throughout (det >= 0.6^2 - 0.5^2 > 0) but too wide for
    # one expansion: x, y in [0.6, 5], z in [-0.5, 0.5] gives rho = 1.16
    Xl = np.array([[0.6, -0.5], [-0.5, 0.6]])
    Xu = np.array([[5.0, 0.5], [0.5, 5.0]])
    assert orc.matrixinv_interval(Xl, Xu, k=8, symmetric=True) is None
    lo, hi, info = orc.matrixinv_cell(Xl, Xu, symmetric=True)
    assert info["pieces"] >= 2
    hl, hu = _inverse_hull(Xl, Xu, n=41, symmetric=True)
    assert np.all(lo <= hl + 1e-12) and np.all(hi >= hu - 1e-12)
    rng = np.random.default_rng(8)
    a, d = rng.uniform(0.6, 5.0, size=(2, 20000))
    b = rng.uniform(-0.5, 0.5, size=20000)
    inv = np.linalg.inv(np.stack([a, b, b, d], axis=-1).reshape(-1, 2, 2))
    assert np.all(inv >= lo - 1e-12) and np.all(inv <= hi + 1e-12)


def test_matrixinv_split_scene_sound(orc):
    # Gaussians 0.9-1.5 m from the camera under a +-5 cm / +-2.5 deg cell:
    # MatrixInv fails on the whole cell for some pairs, input splitting
    # recovers some of them, and the render stays sound (Theorem 1) at
    # sampled poses
    sc = synth.cube_scene(60, 3, half=0.3)
    cam = synth.look_camera(32, 32, 28.0, centre=(0, 0, -1.2))
    clo = np.array([-0.05, -0.05, -0.05, -2.5 * synth.DEG, -2.5 * synth.DEG, -2.5 * synth.DEG])
    rec = orc.records(sc, cam, clo, -clo)
    v = rec["valid"] > 0
    split = v & (rec["pieces"] > 0)
    assert split.sum() >= 2
    assert np.all(rec["rho"][split] >= 1.0 - 1.0 / 1024.0)     # split only where the assertion failed
    assert np.all(rec["fallback"][split] == 0) and np.all(rec["pieces"][split] <= 64)
    assert np.all(rec["korder"][v & (rec["fallback"] == 0)] >= 8)
    lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    rng = np.random.default_rng(21)
    poses = np.concatenate([synth.sample_poses(rng, clo, -clo, 3000), _corners(clo, -clo)])
    worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst


# ------------------------------------------------------------ concrete render

def _ewa_alpha(uw, ls, q, o, cam, delta, ux, uy):
    """Textbook EWA splatting (mean projection + Jacobian-projected covariance)."""
    Rd = Rotation.from_euler("XYZ", delta[3:]).as_matrix()
    Rwc = Rd.T @ cam.R_wc
    t = cam.t + delta[:3]
    x, y, z = Rwc @ (uw - t)
    if z <= cam.near:
        return 0.0
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Cov = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
    Jst = np.array([[cam.fx / z, 0, -cam.fx * x / z**2], [0, cam.fy / z, -cam.fy * y / z**2]])
    S2 = Jst @ Rwc @ Cov @ Rwc.T @ Jst.T
    mu = np.array([cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy])
    dd = np.array([ux, uy]) - mu
    m = dd @ np.linalg.solve(S2, dd)
    if o * math.exp(-0.5 * m) < 1 / 255:
        return 0.0
    return o * math.exp(-0.5 * m)


def test_alpha_matches_textbook_ewa(orc):
    rng = np.random.default_rng(2)
    sc = synth.cube_scene(40, 9, logscale_mu=-1.8)
    cam = synth.look_camera(48, 40, 45.0, centre=(0.1, -0.05, -2.5))
    cam.R_wc = Rotation.from_euler("XYZ", [0.05, -0.04, 0.02]).as_matrix()
    n_nonzero = 0
    for i in range(sc.n):
        delta = np.concatenate([rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.05, 0.05, 3)])
        for _ in range(6):
            ux, uy = rng.uniform(0, 48), rng.uniform(0, 40)
            a = orc.concrete_alpha(sc.uw[i], sc.logscale[i], sc.quat[i], sc.opacity[i], cam, delta, ux, uy)
            b = _ewa_alpha(sc.uw[i].astype(float), sc.logscale[i].astype(float), sc.quat[i].astype(float),
                           float(sc.opacity[i]), cam, delta, ux, uy)
            assert abs(a - b) < 1e-9
            n_nonzero += a > 0
    assert n_nonzero > 20


def test_lemma2_blendsort_equals_blendind(orc):
    rng = np.random.default_rng(4)
    for seed in range(4):
        sc = synth.cube_scene(30, seed, logscale_mu=-2.0)
        cam = synth.look_camera(24, 20, 24.0, centre=(0, 0, -3))
        delta = rng.uniform(-0.05, 0.05, 6)
        a = orc.render_concrete(sc, cam, delta, "sort")
        b = orc.render_concrete(sc, cam, delta, "ind")
        assert np.abs(a - b).max() < 1e-12
        assert a.max() > 0.1


def test_blend_two_gaussians_closed_form(orc):
    sc = synth.cube_scene(2, 1, logscale_mu=-1.5)
    sc.uw[:] = [[0.0, 0.0, 0.3], [0.02, 0.0, -0.2]]   # Gaussian 1 is nearer the camera
    sc.rgb[:] = [[1, 0, 0], [0, 0, 1]]
    cam = synth.look_camera(16, 16, 16.0, centre=(0, 0, -3))
    img = orc.render_concrete(sc, cam, np.zeros(6), "ind")
    for (px, py) in [(8, 8), (7, 9), (10, 6)]:
        a0 = orc.concrete_alpha(sc.uw[0], sc.logscale[0], sc.quat[0], sc.opacity[0], cam, np.zeros(6), px + .5, py + .5)
        a1 = orc.concrete_alpha(sc.uw[1], sc.logscale[1], sc.quat[1], sc.opacity[1], cam, np.zeros(6), px + .5, py + .5)
        expect = a1 * np.array([0, 0, 1.0]) + (1 - a1) * a0 * np.array([1.0, 0, 0])
        np.testing.assert_allclose(img[py, px], expect, atol=1e-12)


# ------------------------------------------------------------ abstract render

def test_point_cell_equals_concrete(orc):
    w = synth.tiny64()
    rng = np.random.default_rng(8)
    for _ in range(3):
        d = np.concatenate([rng.uniform(-0.02, 0.02, 3), rng.uniform(-0.01, 0.01, 3)])
        lo, hi, frag = orc.render_abstract(w.scene, w.camera, d, d)
        img = orc.render_concrete(w.scene, w.camera, d, "sort")
        ok = frag == 0
        assert ok.mean() > 0.97
        assert np.abs(lo - img)[ok].max() < 1e-10
        assert np.abs(hi - img)[ok].max() < 1e-10
        # fragile pixels are still sound
        assert np.all(lo <= img + 1e-10) and np.all(img <= hi + 1e-10)


def _corners(lo, hi):
    idx = np.array(np.meshgrid(*[[0, 1]] * 6, indexing="ij")).reshape(6, -1).T
    return np.where(idx == 0, lo, hi)


def test_theorem1_tiny64_sampled_poses(orc):
    w = synth.tiny64()
    lo, hi, _ = orc.render_abstract(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0])
    rng = np.random.default_rng(0)
    poses = np.concatenate([synth.sample_poses(rng, w.cells_lo[0], w.cells_hi[0], 10_000),
                            _corners(w.cells_lo[0], w.cells_hi[0])])
    worst, nv = orc.check_samples(w.scene, w.camera, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst
    gap = np.linalg.norm(hi - lo, axis=2)
    assert gap.max() <= math.sqrt(3) + 1e-12          # XPG <= sqrt(3) (per-channel clip)
    assert 0 < gap.mean() < 0.2                        # tight for a 1 cm translation


@pytest.mark.parametrize("hw", [
    [0.02, 0.02, 0.02, 0.01, 0.01, 0.01],   # 6-DoF
    [0.0, 0.0, 0.0, 0.0, 0.0, 0.03],        # roll only
    [0.05, 0.0, 0.05, 0.0, 0.0, 0.0],       # translation only
])
def test_theorem1_object_cells(orc, hw):
    sc = synth.object_scene(400, 3, logscale_mu=-3.0)
    cam = synth.look_camera(40, 36, 48.0, centre=(0, 0, -3))
    clo, chi = synth.cell_grid(hw, [2 if h > 0 else 1 for h in hw])
    rng = np.random.default_rng(1)
    for c in range(0, clo.shape[0], max(1, clo.shape[0] // 3)):
        lo, hi, _ = orc.render_abstract(sc, cam, clo[c], chi[c])
        poses = np.concatenate([synth.sample_poses(rng, clo[c], chi[c], 1500), _corners(clo[c], chi[c])])
        worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
        assert nv == 0, worst
        assert np.all(lo <= hi)


def test_dense_grid_brute_force_tiny(orc):
    sc = synth.cube_scene(6, 21, half=0.3, logscale_mu=-1.7)
    cam = synth.look_camera(16, 16, 18.0, centre=(0, 0, -2.5))
    clo = np.array([-0.03, -0.02, -0.02, -0.02, -0.02, -0.02])
    chi = -clo
    lo, hi, _ = orc.render_abstract(sc, cam, clo, chi)
    g = np.linspace(0, 1, 4)
    grid = np.array(np.meshgrid(*[g] * 6, indexing="ij")).reshape(6, -1).T
    poses = clo + grid * (chi - clo)
    worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst
    # and the bounds are not vacuous: somewhere the lower bound is positive
    assert lo.max() > 0.05


def test_translation_only_keys_are_exact(orc):
    # the depth key subtracts the translation term shared by every Gaussian, so
    # a translation-only cell leaves key intervals of (almost) zero width
    w = synth.object10k(n=300, width=64, height=64, f=70.0)
    lo = np.array([-0.05, -0.05, -0.05, 0, 0, 0])
    rec = orc.records(w.scene, w.camera, lo, -lo)
    v = rec["valid"] > 0
    assert v.sum() > 100
    d_width = rec["khi"][v] - rec["klo"][v]
    assert d_width.max() < 1e-7
    # with a yaw interval the keys widen
    lo2 = np.array([0, 0, 0, 0, -0.02, 0])
    rec2 = orc.records(w.scene, w.camera, lo2, -lo2)
    assert (rec2["khi"] - rec2["klo"])[rec2["valid"] > 0].max() > 1e-4


def test_screen_box_is_sound(orc):
    # outside a Gaussian's pixel box its concrete alpha is zero at every pose of the cell
    sc = synth.object_scene(24, 5, logscale_mu=-2.6)
    cam = synth.look_camera(48, 48, 50.0, centre=(0, 0, -3))
    clo = np.array([-0.03, -0.03, -0.03, -0.02, -0.02, -0.02])
    rec = orc.records(sc, cam, clo, -clo)
    rng = np.random.default_rng(6)
    poses = synth.sample_poses(rng, clo, -clo, 200)
    for i in range(sc.n):
        if not rec["valid"][i]:
            continue
        px0, px1, py0, py1 = (int(rec[k][i]) for k in ["px0", "px1", "py0", "py1"])
        one = sc.subset([i])
        one.rgb[:] = 1.0
        lo = np.zeros((48, 48, 3))
        hi = np.zeros((48, 48, 3))
        hi[py0:py1 + 1, px0:px1 + 1] = 1.0
        worst, nv = orc.check_samples(one, cam, poses, lo, hi, tol=0.0)
        assert nv == 0, (i, worst)


def test_near_plane_straddle_sound(orc):
    # Gaussians close to the camera so that the near plane cuts through the depth range
    sc = synth.cube_scene(30, 2, half=0.25, logscale_mu=-2.5)
    sc.uw[:, 2] = np.linspace(-0.85, -0.65, 30).astype(np.float32)   # depth ~0.15..0.35 from z=-1
    cam = synth.look_camera(24, 24, 20.0, centre=(0, 0, -1.0))
    clo = np.array([-0.02, -0.02, -0.08, 0, 0, 0])
    rec = orc.records(sc, cam, clo, -clo)
    assert rec["straddle"].sum() > 0
    lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    rng = np.random.default_rng(12)
    poses = np.concatenate([synth.sample_poses(rng, clo, -clo, 2000), _corners(clo, -clo)])
    worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst


def test_bounds_contain_empirical_and_shrink_with_cell(orc):
    sc = synth.object_scene(300, 8, logscale_mu=-3.0)
    cam = synth.look_camera(32, 32, 40.0, centre=(0, 0, -3))
    gaps = []
    for hw in [0.04, 0.02, 0.01, 0.0]:
        clo = np.array([-hw, 0, 0, 0, 0, 0])
        lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
        gaps.append(np.linalg.norm(hi - lo, axis=2).mean())
    assert gaps[0] > gaps[1] > gaps[2] > gaps[3]
    assert gaps[3] < 1e-12


def _two_gaussian_scene(zA, zB, xA, xB, scale=-1.6, opac=0.95):
    sc = synth.cube_scene(2, 0)
    sc.uw[:] = [[xA, 0.0, zA], [xB, 0.0, zB]]
    sc.logscale[:] = scale
    sc.quat[:] = [1, 0, 0, 0]
    sc.opacity[:] = opac
    sc.rgb[:] = [[1, 0, 0], [0, 0, 1]]
    return sc


def test_uncertain_depth_order_is_sound(orc):
    # A yaw interval swaps the depth order of two laterally offset, overlapping,
    # nearly opaque Gaussians: the back one's lower bound must account for the
    # front one possibly occluding it (Ind uncertain -> factor 1 - a_hi).
    sc = _two_gaussian_scene(0.0, 0.0, -0.05, 0.05)
    cam = synth.look_camera(16, 16, 30.0, centre=(0, 0, -2))
    clo = np.array([0, 0, 0, 0, -0.01, 0])
    rec = orc.records(sc, cam, clo, -clo)
    assert rec["klo"][0] < rec["khi"][1] and rec["klo"][1] < rec["khi"][0]   # order uncertain
    lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    poses = synth.sample_poses(np.random.default_rng(0), clo, -clo, 400)
    worst, nv = orc.check_samples(sc, cam, np.concatenate([poses, _corners(clo, -clo)]), lo, hi, tol=1e-12)
    assert nv == 0, worst
    # at the centre both colours are visible for some pose but neither is guaranteed in full
    e_lo, e_hi = orc.empirical_bounds(sc, cam, poses)
    assert e_hi[8, 8, 0] - e_lo[8, 8, 0] > 0.3 and e_hi[8, 8, 2] - e_lo[8, 8, 2] > 0.3


def test_near_plane_drop_is_sound(orc):
    # One wide opaque Gaussian whose depth crosses the near plane inside the cell:
    # where d <= near it disappears, so its lower bound must be zero.
    sc = _two_gaussian_scene(-0.8, 5.0, 0.0, 3.0, scale=-3.0)
    cam = synth.look_camera(16, 16, 16.0, centre=(0, 0, -1.0))
    clo = np.array([0, 0, -0.05, 0, 0, 0])
    rec = orc.records(sc, cam, clo, -clo)
    assert rec["straddle"][0] == 1
    lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    poses = np.linspace(clo, -clo, 201)
    worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst
    assert hi[8, 8, 0] > 0.5 and lo[8, 8, 0] == 0.0


# ------------------------------------------------ frustum guard band (3DGS)
# A 16x16 image with f = 16 and cx = 8: the guard band keeps projected means
# with |u - 8| <= 0.65 * 16 = 10.4, i.e. u <= 18.4.  A wide opaque Gaussian at
# depth 1 and lateral offset x projects its mean to u = 8 + 16 x.

def _guard_scene(x):
    sc = synth.cube_scene(1, 0)
    sc.uw[:] = [[x, 0.0, 0.0]]
    sc.logscale[:] = -0.5          # sigma 0.61 m: about 10 px, reaching well into the image
    sc.quat[:] = [1, 0, 0, 0]
    sc.opacity[:] = 0.9
    sc.rgb[:] = [[1, 1, 1]]
    return sc


def test_guard_band_concrete(orc):
    cam = synth.look_camera(16, 16, 16.0, centre=(0, 0, -1.0))
    zero = np.zeros(6)
    inside = orc.render_concrete(_guard_scene(0.6), cam, zero, "sort")    # u = 17.6
    outside = orc.render_concrete(_guard_scene(0.7), cam, zero, "sort")   # u = 19.2
    assert inside[8, 15, 0] > 0.2 and inside[8, 8, 0] > 0.01
    assert np.all(outside == 0.0)


def test_guard_band_abstract_drop(orc):
    cam = synth.look_camera(16, 16, 16.0, centre=(0, 0, -1.0))
    clo = np.array([-0.001, 0, 0, 0, 0, 0])
    rec = orc.records(_guard_scene(0.7), cam, clo, -clo)
    assert rec["valid"][0] == 0
    lo, hi, _ = orc.render_abstract(_guard_scene(0.7), cam, clo, -clo)
    assert np.all(lo == 0.0) and np.all(hi == 0.0)


def test_guard_band_crossing_is_sound(orc):
    # the camera's x translation moves the mean across u = 18.4 inside the cell
    sc = _guard_scene(0.65)
    cam = synth.look_camera(16, 16, 16.0, centre=(0, 0, -1.0))
    clo = np.array([-0.05, 0, 0, 0, 0, 0])
    rec = orc.records(sc, cam, clo, -clo)
    assert rec["valid"][0] == 1 and rec["straddle"][0] == 1
    lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    poses = np.linspace(clo, -clo, 201)
    worst, nv = orc.check_samples(sc, cam, poses, lo, hi, tol=1e-12)
    assert nv == 0, worst
    assert np.all(lo == 0.0) and hi[8, 15, 0] > 0.2


# ------------------------------------------------ scene-parameter boxes (Sec. 4.5)

def _box_array(b):
    return np.concatenate([b["uw_lo"], b["uw_hi"], b["o_lo"][:, None], b["o_hi"][:, None], b["c_lo"], b["c_hi"]],
                          axis=1).astype(np.float64)


def _sample_scene(sc, b, rng):
    u = lambda shape: rng.uniform(size=shape)
    lo, hi = b["uw_lo"].astype(np.float64), b["uw_hi"].astype(np.float64)
    uw = lo + (hi - lo) * u(lo.shape)
    o = b["o_lo"] + (b["o_hi"].astype(np.float64) - b["o_lo"]) * u(sc.n)
    c = b["c_lo"] + (b["c_hi"].astype(np.float64) - b["c_lo"]) * u((sc.n, 3))
    return synth.Scene(uw, sc.logscale.astype(np.float64), sc.quat.astype(np.float64), o, c)


def test_boxes_point_cell_closed_form(orc):
    # one Gaussian seen from a fixed pose, with opacity in [o/2, o] and red in
    # [c - 0.2, c]: at a pixel where no opacity of the box is cut, a = o e^-m/2
    # is exact at a point cell and T = 1, so the bounds are c_lo o_lo e and
    # c_hi o_hi e (e from the textbook EWA formula)
    sc = synth.object_scene(1, 7, mean_sd=0.0, logscale_mu=-1.6)
    sc.opacity[:] = 0.9
    sc.rgb[:] = np.array([0.7, 0.4, 0.2], dtype=np.float32)
    cam = synth.look_camera(24, 24, 30.0, centre=(0, 0, -3))
    b = {"uw_lo": sc.uw.copy(), "uw_hi": sc.uw.copy(), "o_lo": np.float32([0.45]), "o_hi": np.float32([0.9]),
         "c_lo": np.float32([[0.5, 0.4, 0.2]]), "c_hi": np.float32([[0.7, 0.4, 0.2]])}
    d = np.zeros(6)
    orc.set_boxes(_box_array(b))
    try:
        lo, hi, _ = orc.render_abstract(sc, cam, d, d)
    finally:
        orc.set_boxes(None)
    n_checked = 0
    for py in range(8, 16):
        for px in range(8, 16):
            e = _ewa_alpha(sc.uw[0].astype(np.float64), sc.logscale[0].astype(np.float64),
                           sc.quat[0].astype(np.float64), 1.0, cam, d, px + 0.5, py + 0.5)
            if 0.45 * e < 1.5 / 255:
                continue
            # (the box ends are float32 values)
            exp_lo = b["c_lo"][0].astype(np.float64) * float(b["o_lo"][0]) * e
            exp_hi = b["c_hi"][0].astype(np.float64) * float(b["o_hi"][0]) * e
            np.testing.assert_allclose(lo[py, px], exp_lo, rtol=1e-9, atol=1e-12)
            np.testing.assert_allclose(hi[py, px], exp_hi, rtol=1e-9, atol=1e-12)
            n_checked += 1
    assert n_checked > 20


def test_boxes_equal_to_nominal_change_nothing(orc):
    w = synth.tiny64()
    b = synth.scene_boxes(w.scene, 3, frac=0.0)
    lo0, hi0, _ = orc.render_abstract(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0])
    orc.set_boxes(_box_array(b))
    try:
        lo1, hi1, _ = orc.render_abstract(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0])
    finally:
        orc.set_boxes(None)
    assert np.array_equal(lo0, lo1) and np.array_equal(hi0, hi1)


@pytest.mark.parametrize("kind", ["colour", "mean", "opacity", "all"])
def test_boxes_sound_sampled(orc, kind):
    # Theorem 1 over the product of the pose cell and the parameter boxes:
    # concrete renders at sampled (pose, scene) pairs lie inside the bounds
    sc = synth.object_scene(300, 11, logscale_mu=-3.0)
    cam = synth.look_camera(36, 32, 44.0, centre=(0, 0, -3))
    clo = np.array([-0.01, -0.01, -0.01, 0.0, -0.003, 0.0])
    args = {"colour": dict(red_add=0.5), "mean": dict(mean_d=(0.0, 0.08, 0.0)),
            "opacity": dict(opacity_scale=0.5, opacity_add=0.1),
            "all": dict(red_add=0.3, mean_d=(0.03, 0.03, 0.0), opacity_scale=0.8, opacity_add=0.1)}[kind]
    b = synth.scene_boxes(sc, 5, frac=0.4, **args)
    orc.set_boxes(_box_array(b))
    try:
        lo, hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    finally:
        orc.set_boxes(None)
    base_lo, base_hi, _ = orc.render_abstract(sc, cam, clo, -clo)
    assert np.all(lo <= hi)
    if kind in ("colour", "mean"):
        # boxes that hold the nominal scene widen the bounds
        assert (hi - lo).sum() > (base_hi - base_lo).sum()
    rng = np.random.default_rng(2)
    corners = _corners(clo, -clo)
    for k in range(60):
        s2 = _sample_scene(sc, b, rng)
        pose = corners[k] if k < 8 else synth.sample_poses(rng, clo, -clo, 1)[0]
        img = orc.render_concrete(s2, cam, pose, "ind")
        assert np.all(img >= lo - 1e-12) and np.all(img <= hi + 1e-12), (kind, k)


# ------------------------------------------------ abstract BlendSort (Example 2)

def _three_gaussians():
    # three Gaussians (red, green, blue) at increasing depths in front of a
    # camera at the origin, in the manner of Example 2 (its scene is not printed)
    uw = np.array([[-0.35, 0.1, 3.0], [0.0, -0.1, 3.6], [0.35, 0.05, 4.2]], dtype=np.float32)
    ls = np.log(np.array([[0.45, 0.35, 0.3], [0.4, 0.5, 0.3], [0.5, 0.4, 0.35]], dtype=np.float32))
    q = np.array([[1, 0, 0, 0], [0.96, 0.2, 0.1, 0.1], [0.9, -0.1, 0.3, 0.2]], dtype=np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sc = synth.Scene(uw, ls, q, np.array([0.8, 0.75, 0.85], dtype=np.float32), np.eye(3, dtype=np.float32))
    return sc, synth.look_camera(20, 20, 16.0, centre=(0, 0, 0))


def test_abstract_blendsort_point_cell_is_concrete(orc):
    # at a point cell every rank is exact and every opacity interval a point:
    # the abstract BlendSort is Algorithm 2 itself
    sc, cam = _three_gaussians()
    d = np.array([0.02, -0.01, 0.05, 0.0, 0.0, 0.0])
    lo, hi = orc.render_abstract_sort(sc, cam, d, d)
    img = orc.render_concrete(sc, cam, d, "sort")
    assert np.abs(lo - img).max() < 1e-10 and np.abs(hi - img).max() < 1e-10


@pytest.mark.parametrize("h", [0.1, 0.3])
def test_abstract_blendsort_sound(orc, h):
    sc, cam = _three_gaussians()
    clo = np.array([-h, -h, -h, 0.0, 0.0, 0.0])
    lo, hi = orc.render_abstract_sort(sc, cam, clo, -clo)
    rng = np.random.default_rng(4)
    poses = np.concatenate([synth.sample_poses(rng, clo, -clo, 400), _corners(clo, -clo)])
    for p in poses:
        img = orc.render_concrete(sc, cam, p, "sort")
        assert np.all(img >= lo - 1e-12) and np.all(img <= hi + 1e-12)
    # the same cell with BlendInd is sound too, and both are wider than the samples
    li, hi2, _ = orc.render_abstract(sc, cam, clo, -clo)
    assert np.all(li >= 0) and np.all(hi2 <= 1)
    w = synth.tiny64()
    slo, shi = orc.render_abstract_sort(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0])
    worst, nv = orc.check_samples(w.scene, w.camera, synth.sample_poses(rng, w.cells_lo[0], w.cells_hi[0], 2000),
                                  slo, shi, tol=1e-12)
    assert nv == 0, worst


# ------------------------------------- relational upper transmittance (tight)

def test_transmittance_chain_closed_forms(orc):
    # one factor: F = 1 - L where a_lo > 0, else the constant 1
    F, y = orc.transmittance_chain([_form([0.1], 0.3)], [0.2], [0.4])
    assert np.allclose(F, _form([-0.1], 0.7), atol=1e-15) and y == pytest.approx(0.8)
    F, y = orc.transmittance_chain([_form([0.3], 0.1)], [0.0], [0.4])
    assert np.allclose(F, _form([], 1.0), atol=1e-15) and y == 1.0
    # two factors, worked by hand: L1 = 0.1 p0 + 0.3 on [0.2, 0.4],
    # L2 = -0.05 p1 + 0.5 on [0.45, 0.6].  After the first, F = 0.7 - 0.1 p0 and
    # y = 0.8; then F = 0.8 (0.5 + 0.05 p1) + 0.4 (0.7 - 0.1 p0 - 0.8)
    #                = 0.36 - 0.04 p0 + 0.04 p1, y = 0.8 * 0.55 = 0.44
    F, y = orc.transmittance_chain([_form([0.1], 0.3), _form([0, -0.05], 0.5)], [0.2, 0.45], [0.4, 0.6])
    assert np.allclose(F, _form([-0.04, 0.04], 0.36), atol=1e-15) and y == pytest.approx(0.44)
    # at p = (1, -1) the product is at most 0.6 * 0.45 = 0.27: F gives 0.28,
    # the interval product 0.44
    assert _eval(F, np.array([1, -1, 0, 0, 0, 0])) == pytest.approx(0.28)


def test_transmittance_chain_point_forms_are_the_interval_product(orc):
    # constant forms (a point cell): the chain is the interval product
    rng = np.random.default_rng(11)
    a = rng.uniform(0.05, 0.6, 8)
    L = np.stack([_form([], v) for v in a])
    F, y = orc.transmittance_chain(L, a, a)
    assert np.allclose(F[:6], 0.0) and F[6] == pytest.approx(np.prod(1 - a), rel=1e-12)
    assert y == pytest.approx(np.prod(1 - a), rel=1e-12)


def test_transmittance_chain_sound_and_below_interval_product(orc):
    # brute force: random chains of lower forms over three active variables;
    # the product is largest where every a_j takes its least consistent value
    rng = np.random.default_rng(12)
    for trial in range(40):
        K = int(rng.integers(1, 9))
        L, alo, ahi = [], [], []
        for _ in range(K):
            c = rng.uniform(-0.08, 0.08, 3)
            k = rng.uniform(0.0, 0.5)
            lo_v = k - np.abs(c).sum()
            L.append(_form(c, k))
            alo.append(max(0.0, lo_v))
            ahi.append(min(0.95, k + np.abs(c).sum() + rng.uniform(0, 0.2)))
        F, y = orc.transmittance_chain(np.stack(L), alo, ahi)
        assert F[6] + np.abs(F[:6]).sum() <= y + 1e-12          # never above the interval product
        P = rng.uniform(-1, 1, (300, 6))
        P[:, 3:] = 0.0
        P[:8, :3] = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
        for p in P:
            amin = np.array([max(alo[j], _eval(L[j], p)) for j in range(K)])
            assert np.prod(1 - amin) <= _eval(F, p) + 1e-12


def test_tight_blend_never_looser_and_sound(orc):
    # the relational upper transmittance only lowers the upper bound, and the
    # bounds stay sound at sampled poses
    w = synth.tiny64()
    lo, hi, _ = orc.render_abstract(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0])
    tlo, thi, _ = orc.render_abstract(w.scene, w.camera, w.cells_lo[0], w.cells_hi[0], tight=True)
    assert np.array_equal(lo, tlo)
    assert np.all(thi <= hi + 1e-12)
    assert (thi - tlo).mean() < 0.9 * (hi - lo).mean()
    rng = np.random.default_rng(13)
    worst, nv = orc.check_samples(w.scene, w.camera, synth.sample_poses(rng, w.cells_lo[0], w.cells_hi[0], 2000),
                                  tlo, thi, tol=1e-12)
    assert nv == 0, worst
    # a point cell: every form is constant and both blends agree
    d = np.array([0.004, -0.003, 0.01, 0.002, -0.004, 0.003])
    lo, hi, _ = orc.render_abstract(w.scene, w.camera, d, d)
    tlo, thi, _ = orc.render_abstract(w.scene, w.camera, d, d, tight=True)
    assert np.array_equal(lo, tlo) and np.abs(hi - thi).max() < 1e-12


# ------------------------------------------------------- partition and union

def test_partition_pieces_cover_the_box(orc):
    box_lo = np.array([-0.03, 0.0, -0.01, 0.0, -0.02, 0.0])
    box_hi = np.array([0.03, 0.0, 0.05, 0.0, 0.02, 0.0])
    lo, hi = orc.partition_cells(box_lo, box_hi, [3, 1, 2, 1, 4, 1])
    assert lo.shape == (24, 6)
    # per dimension the pieces tile [lo, hi] end to end, with equal widths
    for k, P in enumerate([3, 1, 2, 1, 4, 1]):
        edges = sorted(set(lo[:, k]) | set(hi[:, k]))
        assert len(edges) == P + 1 or box_lo[k] == box_hi[k]
        assert edges[0] == box_lo[k] and edges[-1] == box_hi[k]
        assert np.allclose(np.diff(edges), (box_hi[k] - box_lo[k]) / P)
    # dimension 0 varies fastest
    assert lo[1, 0] > lo[0, 0] and lo[1, 2] == lo[0, 2]


def test_partition_union_is_sound_and_tighter(orc):
    # Sec. 5: bounds of the pieces, joined, bound the whole box, and finer
    # partitions tighten them
    w = synth.tiny64()
    blo, bhi = w.cells_lo[0], w.cells_hi[0]
    act = [int(v) for v in (bhi > blo)]
    parts = [2 if a else 1 for a in act]
    lo1, hi1, _ = orc.render_abstract(w.scene, w.camera, blo, bhi)
    lo2, hi2, _ = orc.render_abstract_partitioned(w.scene, w.camera, blo, bhi, parts)
    assert (hi2 - lo2).mean() < 0.9 * (hi1 - lo1).mean()
    rng = np.random.default_rng(31)
    worst, nv = orc.check_samples(w.scene, w.camera, synth.sample_poses(rng, blo, bhi, 2000), lo2, hi2, tol=1e-12)
    assert nv == 0, worst
    # one piece is the box itself
    lo3, hi3, _ = orc.render_abstract_partitioned(w.scene, w.camera, blo, bhi, [1] * 6)
    assert np.array_equal(lo3, lo1) and np.array_equal(hi3, hi1)
