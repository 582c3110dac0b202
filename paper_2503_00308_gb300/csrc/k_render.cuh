// k_render.cuh -- per-pixel effective-opacity relaxation and BlendInd blend.
//
// One CTA per (cell, tile), one thread per pixel.  The tile's bin holds the
// two depth-key endpoints of every (Gaussian, cell) pair whose pixel box meets
// the tile, sorted by key.  Each pixel sweeps that list once:
//
//   lower endpoint of i : effective-opacity bounds of i at this pixel
//                         (Algorithm 1 lines 9-10 relaxed: Delta = S u - P,
//                         q = Delta^T W, m = q q^T, a = o Exp(-m/2) with the
//                         tangent/secant of Table 2 and the 1/255 cutoff);
//                         T_hi(i) = prod over j certainly in front of i of
//                         (1 - a_lo(j)), i.e. keys with khi(j) < klo(i);
//                         the upper colour form gains T_hi(i) c_i U_i.
//   upper endpoint of i : T_lo(i) = prod over j != i that may be in front of
//                         i of (1 - a_hi(j)), i.e. klo(j) < khi(i); the lower
//                         colour form gains T_lo(i) c_i L_i.
//
// This is BlendInd (Algorithm 4) with Ind(d_i - d_j) three-valued from the
// depth-key intervals and Prod bounded by interval products (REL = true adds
// the relational upper transmittance of RelT below).  Products over
// keys strictly below a value are running products over the sorted list;
// endpoints with equal keys are handled as a group (queries before
// absorptions) so strictness matches the pairwise definition.
#pragma once
#include "ar_common.cuh"

namespace ar {

template <int M, class R = float> struct AlphaOut {
    LF<M, R> L, U;  // lower / upper forms of the effective opacity
    R rL, rU;       // their coefficient radii
    R alo, ahi;     // scalar enclosure of a over the cell
    R dev;          // estimate of how far single precision moves alo, ahi (see pixel_alpha)
};

// n elements (a multiple of 4, 16-byte aligned) copied with 16-byte loads
template <int n>
__device__ __forceinline__ void load_vec(const float *src, float *dst)
{
#pragma unroll
    for (int q = 0; q < n / 4; ++q) reinterpret_cast<float4 *>(dst)[q] = reinterpret_cast<const float4 *>(src)[q];
}
template <int n>
__device__ __forceinline__ void load_vec(const double *src, double *dst)
{
#pragma unroll
    for (int q = 0; q < n / 2; ++q) reinterpret_cast<double2 *>(dst)[q] = reinterpret_cast<const double2 *>(src)[q];
}

// c[M], -klo, khi, r (S and R entries; vlo, vhi are not needed).  The record
// element type RE may be narrower than the arithmetic type R (an FP32 record
// evaluated in FP64): the conversion is exact.
template <int M, class R, class RE>
__device__ __forceinline__ void load_sb(const RE *src, SB<M, R> &b)
{
    RE v[Rec<M>::SBW];
    load_vec<Rec<M>::SBW>(src, v);
#pragma unroll
    for (int j = 0; j < M; ++j) b.c[j] = (R)v[j];
    b.klo = -(R)v[M];
    b.khi = (R)v[M + 1];
    b.r = (R)v[M + 2];
}

// c[M], -klo, khi, -vlo, vhi, r, mid (W entries); returns sb_mid(b), read
// from the record where it was computed in the same precision, else computed
template <int M, class R, class RE>
__device__ __forceinline__ R load_sbw(const RE *src, SB<M, R> &b)
{
    RE v[Rec<M>::WS];
    load_vec<Rec<M>::WS>(src, v);
#pragma unroll
    for (int j = 0; j < M; ++j) b.c[j] = (R)v[j];
    b.klo = -(R)v[M];
    b.khi = (R)v[M + 1];
    b.vlo = -(R)v[M + 2];
    b.vhi = (R)v[M + 3];
    b.r = (R)v[M + 4];
    if constexpr (sizeof(R) == sizeof(RE)) return v[M + 5];
    else return sb_mid(b);
}

__device__ __forceinline__ float clamp01(float x) { return fminf(1.f, fmaxf(0.f, x)); }
__device__ __forceinline__ double clamp01(double x) { return fmin(1.0, fmax(0.0, x)); }

// flags word of a record: the bit pattern of a float, or the value of a double
__device__ __forceinline__ uint32_t rec_flags(const float *r, int at) { return __float_as_uint(r[at]); }
__device__ __forceinline__ uint32_t rec_flags(const double *r, int at) { return (uint32_t)r[at]; }

// The bounded m of a record at pixel (ux, uy) (Algorithm 1 line 10 relaxed):
// Delta = S u - P, held as (u - mu) S + R (see Rec): the lower form takes
// S.lo and R.lo whatever the sign of u - mu (the pair is u S.lo - P.hi
// exactly); where u - mu < 0 the conversion gap of S is covered.  Then
// q = Delta^T W by McCormick products and m = sum_c q_c^2.
template <int M, class R, class RE>
__device__ __forceinline__ SB<M, R> m_form(const RE *__restrict__ r, R ux, R uy)
{
    using RL = Rec<M>;
    using N = Num<R>;
    typedef SB<M, R> B;
    B Dx, Dy;
    {
        B S, Rr;
        load_sb<M, R, RE>(r + RL::S, S);
        const R dx = ux - r[RL::MU_X], dy = uy - r[RL::MU_Y];  // exact: both are half-integers
        const R gap = r[RL::GAP_S];
        SAcc<M, R> a;
        load_sb<M, R, RE>(r + RL::RX, Rr);
        a.init(0, 0);
        a.term_same_side(dx, S);
        a.term((R)1, Rr);
        if (dx < (R)0) a.add_slack(N::mul_ru(-dx, gap));
        Dx = a.result();
        load_sb<M, R, RE>(r + RL::RY, Rr);
        a.init(0, 0);
        a.term_same_side(dy, S);
        a.term((R)1, Rr);
        if (dy < (R)0) a.add_slack(N::mul_ru(-dy, gap));
        Dy = a.result();
    }
    // m = sum_c (Delta_x W_0c + Delta_y W_1c)^2
    SAcc<M, R> pm;
    pm.init(0, 0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B w0, w1;
        const R m0 = load_sbw<M, R, RE>(r + RL::W0 + c * RL::WS, w0);
        const R m1 = load_sbw<M, R, RE>(r + RL::W0 + (3 + c) * RL::WS, w1);
        SAcc<M, R> pq;
        pq.init(0, 0);
        pq.mul_ym(Dx, w0, m0);
        pq.mul_ym(Dy, w1, m1);
        const B q = pq.result();
        pm.sqr(q);
    }
    return pm.result();
}

// ---------------------------------------------------------------------------
// The same chain in FP32 with the lower and upper constants of every pair
// held together as the float2 (-lo, hi).  Directed rounding is symmetric
// under negation, RD(x) = -RU(-x) for every operation (signed zeros
// included), so both ends move in one packed operation rounded up
// (__ffma2_ru, __fadd2_ru, __fmul2_ru), and each end gets the bits of the
// scalar SAcc operation it stands for; m_form_packed returns m_form's value.
template <int M> struct PSB {
    float c[M];
    float2 k;  // (-klo, khi)
    float r;
    float2 v;  // (-vlo, vhi)
};

// S and R entries: c[M], -klo, khi, r
template <int M>
__device__ __forceinline__ void load_psb(const float *src, PSB<M> &b)
{
    float v[Rec<M>::SBW];
    load_vec<Rec<M>::SBW>(src, v);
#pragma unroll
    for (int j = 0; j < M; ++j) b.c[j] = v[j];
    b.k = make_float2(v[M], v[M + 1]);
    b.r = v[M + 2];
}
// W entries: c[M], -klo, khi, -vlo, vhi, r; returns the stored midpoint
template <int M>
__device__ __forceinline__ float load_psbw(const float *src, PSB<M> &b)
{
    float v[Rec<M>::WS];
    load_vec<Rec<M>::WS>(src, v);
#pragma unroll
    for (int j = 0; j < M; ++j) b.c[j] = v[j];
    b.k = make_float2(v[M], v[M + 1]);
    b.v = make_float2(v[M + 2], v[M + 3]);
    b.r = v[M + 4];
    return v[M + 5];
}

// SAcc<M, float> with packed constants
template <int M> struct PSAcc {
    float c[M];
    float2 k;  // (-klo, khi)
    float rs, ex;
    int n;

    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int j = 0; j < M; ++j) c[j] = 0.f;
        k = make_float2(-0.f, 0.f);  // the negation of +0, and +0
        rs = 0.f;
        ex = 0.f;
        n = 0;
    }
    // SAcc::term_same_side
    __device__ __forceinline__ void term_same_side(float a, const PSB<M> &x)
    {
        axpy_rn<M>(a, x.c, c);
        k = __ffma2_ru(make_float2(a, a), x.k, k);
        rs = __fmaf_ru(fabsf(a), x.r, rs);
        ++n;
    }
    // SAcc::term: for a < 0 the lower end takes (-a) x.hi, the upper one
    // (-a) (-x.lo)
    __device__ __forceinline__ void term(float a, const PSB<M> &x)
    {
        axpy_rn<M>(a, x.c, c);
        const bool pos = a >= 0.f;
        const float b = pos ? a : -a;
        const float2 p = pos ? x.k : make_float2(x.k.y, x.k.x);
        k = __ffma2_ru(make_float2(b, b), p, k);
        rs = __fmaf_ru(fabsf(a), x.r, rs);
        ++n;
    }
    // SAcc::mul_ym.  The constants (-dlo, dhi) are
    //   (RU(RU(xl yl + RU(xh yh)) / 2), RU(RU(xh (-yl) + RU((-xl) yh)) / 2)),
    // the second being -RD(RD(xh yl + RD(xl yh)) / 2).
    __device__ __forceinline__ void mul_ym(const PSB<M> &x, const PSB<M> &y, float ym)
    {
        const float nxl = x.v.x, xh = x.v.y, nyl = y.v.x, yh = y.v.y;
        const float xm = __fmul_rn(xh - nxl, 0.5f);  // sb_mid(x)
        term(ym, x);
        term(xm, y);
        const float2 q = __ffma2_ru(x.v, make_float2(nyl, nyl), make_float2(__fmul_ru(xh, yh), __fmul_ru(nxl, yh)));
        k = __fadd2_ru(k, __fmul2_ru(q, make_float2(0.5f, 0.5f)));
        const float xa = fmaxf(fabsf(nxl), fabsf(xh)), ya = fmaxf(fabsf(nyl), fabsf(yh));
        ex = __fadd_ru(ex, __fmul_ru(__fmaf_ru(fabsf(ym), xa, __fmul_ru(fabsf(xm), ya)), Num<float>::U * 1.001f));
    }
    // SAcc::sqr: the constants (-dlo, dhi) are
    //   (RU(cm cm), max(RU(xl xl + RU(-s xl)), RU(xh xh + RU(-s xh))))
    __device__ __forceinline__ void sqr(const PSB<M> &x)
    {
        const float nxl = x.v.x, xh = x.v.y;
        const float s = xh - nxl;
        const float cm = __fmul_rn(s, 0.5f);
        term(s, x);
        const float2 e = __ffma2_ru(x.v, x.v, __fmul2_ru(make_float2(s, -s), x.v));
        k = __fadd2_ru(k, make_float2(__fmul_ru(cm, cm), fmaxf(e.x, e.y)));
    }
    // SAcc::result with sb_finish
    __device__ __forceinline__ PSB<M> result() const
    {
        const float sl = __fadd_ru(__fmaf_ru(gamma_n<float>(n), rs, ex), Num<float>::TINY);
        PSB<M> b;
#pragma unroll
        for (int j = 0; j < M; ++j) b.c[j] = c[j];
        b.k = __fadd2_ru(k, make_float2(sl, sl));
        float r = 0.f;
#pragma unroll
        for (int j = 0; j < M; ++j) r = __fadd_ru(r, fabsf(c[j]));
        b.r = r;
        b.v = __fadd2_ru(b.k, make_float2(r, r));
        return b;
    }
};

template <int M>
__device__ __forceinline__ SB<M, float> m_form_packed(const float *__restrict__ r, float ux, float uy)
{
    using RL = Rec<M>;
    PSB<M> Dx, Dy;
    {
        PSB<M> S, Rr;
        load_psb<M>(r + RL::S, S);
        const float dx = ux - r[RL::MU_X], dy = uy - r[RL::MU_Y];
        const float gap = r[RL::GAP_S];
        PSAcc<M> a;
        load_psb<M>(r + RL::RX, Rr);
        a.init();
        a.term_same_side(dx, S);
        a.term(1.f, Rr);
        if (dx < 0.f) a.ex = __fadd_ru(a.ex, __fmul_ru(-dx, gap));
        Dx = a.result();
        load_psb<M>(r + RL::RY, Rr);
        a.init();
        a.term_same_side(dy, S);
        a.term(1.f, Rr);
        if (dy < 0.f) a.ex = __fadd_ru(a.ex, __fmul_ru(-dy, gap));
        Dy = a.result();
    }
    PSAcc<M> pm;
    pm.init();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        PSB<M> w0, w1;
        const float m0 = load_psbw<M>(r + RL::W0 + c * RL::WS, w0);
        const float m1 = load_psbw<M>(r + RL::W0 + (3 + c) * RL::WS, w1);
        PSAcc<M> pq;
        pq.init();
        pq.mul_ym(Dx, w0, m0);
        pq.mul_ym(Dy, w1, m1);
        pm.sqr(pq.result());
    }
    const PSB<M> p = pm.result();
    SB<M, float> m;
#pragma unroll
    for (int j = 0; j < M; ++j) m.c[j] = p.c[j];
    m.klo = -p.k.x;
    m.khi = p.k.y;
    m.r = p.r;
    m.vlo = -p.v.x;
    m.vhi = p.v.y;
    return m;
}

// Effective-opacity bounds of one (Gaussian, cell) record at pixel (ux, uy),
// in the arithmetic of R from a record of element type RE.
//
// out.dev estimates how far evaluating in R's precision moves alo and ahi: m
// is a small difference of terms of magnitude about |m_lo| + |m_hi|, so its
// ends move by about 32 u (|m_lo| + |m_hi|), and a = o e^(-m/2) moves by half
// of that times a (a_hi only while m_lo > 0: below that the secant ends at
// x = 0 and a_hi = o).  The FP32 renderer evaluates the pair again in FP64
// where this estimate exceeds its threshold (pixel_alpha_fp64).
//
// upper_c = false leaves the upper form's coefficients out (they are zero in
// out.U): its constant, radius and out.ahi do not depend on them, and a sweep
// whose upper sums are final uses no more than those.  SCALAR = true takes the
// FP32 chain to m with the scalar SAcc steps in place of the packed ones (the
// same bits; a test hook checks that they are).
template <int M, class R = float, class RE = R, bool SCALAR = false>
__device__ __forceinline__ void pixel_alpha(const RE *__restrict__ r, R ux, R uy, AlphaOut<M, R> &out,
                                            R *m_out = nullptr, bool upper_c = true)
{
    using RL = Rec<M>;
    using N = Num<R>;
    // opacity box [o_lo, o]: o_lo scales the lower forms, o the upper ones
    const R o = r[RL::O], o_lo = r[RL::O_LO];
    const uint32_t flags = rec_flags(r, RL::FLAGS);
    out.dev = 0;
    if (flags & F_FALLBACK) {
#pragma unroll
        for (int j = 0; j < M; ++j) { out.L.c[j] = 0; out.U.c[j] = 0; }
        out.L.k = 0; out.U.k = o; out.rL = 0; out.rU = 0;
        out.alo = 0; out.ahi = o;
        return;
    }
    typedef SB<M, R> B;
    B m;
    if constexpr (!SCALAR && sizeof(R) == sizeof(float) && sizeof(RE) == sizeof(float)) m = m_form_packed<M>(r, ux, uy);
    else m = m_form<M, R, RE>(r, ux, uy);
    const R mlo = m.vlo, mhi = m.vhi;
    if (m_out) {
        m_out[0] = mlo;
        m_out[1] = mhi;
    }
    // Exp on x = -m/2 in [xl, xu], xu clipped at 0 because m >= 0
    const R xl = R(-0.5) * mhi;
    R xu = N::min(R(-0.5) * mlo, R(0));
    if (!(xu >= xl)) xu = xl;
    const R el_dn = N::exp_dn(xl), el_up = N::exp_up(xl), eu_up = N::exp_up(xu);
    // lower: o e(xl) (1 + x - xl) with x >= -m.hi/2
    Acc<M, R, true> la;
    const R e1 = N::mul_rd(o_lo, el_dn);
    la.init(N::mul_rd(e1, N::sub_rd(R(1), xl)));
    la.term_ck(R(-0.5) * e1, m.c, m.khi, m.r);
    LF<M, R> La = la.result();
    // upper: o (e(xl) + s (x - xl)) with x <= -m.lo/2
    const R w = N::sub_rd(xu, xl);
    R s = (w > R(0)) ? N::div_pos_up(N::sub_ru(eu_up, el_up), w) : eu_up;
    s = N::min(N::max(s, R(0)), N::BIG);
    const R e2 = N::mul_ru(o, el_up), s2 = N::mul_ru(o, s);
    Acc<M, R, false> ua;
    ua.init(N::fma_ru(-s2, xl, e2));
    ua.term_ck(R(-0.5) * s2, m.c, m.klo, m.r, upper_c);
    LF<M, R> Ua = ua.result();
    const R rUa = ua.radius_bound();
    const R amax = N::add_ru(Ua.k, rUa);
    // blend the upper form toward the constant o where its maximum exceeds o
    // The blend weights lam, psi2 (where m_lo > tau), psi (where m_hi <= tau)
    // and mu keep the bounds sound at any value in [0, 1], so they are divided
    // to a few ulp and clamped (a non-finite quotient clamps into [0, 1] too).
    const R lam = clamp01(N::div_weight(o * (R(1) + R(CLIP_RAMP)) - amax, o * R(CLIP_RAMP)));
    // cutoff ramps (width shrinks with the m interval)
    R ramp = N::min(R(CUT_RAMP), mhi - mlo);
    if (!(ramp > R(0))) ramp = 0;
    const R tdn = r[RL::TAU_DN], tup = r[RL::TAU_UP];
    const R psi2 = (mlo <= tup) ? R(0) : (ramp > R(0) ? clamp01(N::div_weight(mlo - tup, ramp)) : R(1));
    const R psi = (mhi > tdn) ? R(1) : (ramp > R(0) ? clamp01(N::div_weight(mhi - tdn + ramp, ramp)) : R(0));
    {
        Acc<M, R, false> u1;
        const R keep = R(1) - psi2;
        u1.init(N::mul_ru(keep, N::mul_ru(N::sub_ru(R(1), lam), o)));
        u1.term(keep * lam, Ua, rUa, upper_c);
        out.U = u1.result();
        out.rU = u1.radius_bound();
    }
    out.ahi = N::min(o, N::add_ru(out.U.k, out.rU));
    // lower: subtract psi/255, then blend toward 0 where the form dips below 0
    La.k = N::sub_rd(La.k, N::mul_ru(psi, R(ALPHA_MIN_UP)));
    const R rLa = la.radius_bound();
    const R l2min = N::sub_rd(La.k, rLa), l2max = La.k + rLa;
    const R mu = (l2min >= R(0)) ? R(1) : ((l2max <= R(0)) ? R(0) : clamp01(N::div_weight(l2max, l2max - l2min)));
    if ((flags & F_STRADDLE) || mu == R(0)) {
#pragma unroll
        for (int j = 0; j < M; ++j) out.L.c[j] = 0;
        out.L.k = 0;
        out.rL = 0;
        out.alo = 0;
    } else if (mu == R(1)) {
        out.L = La;
        out.rL = rLa;
        out.alo = N::max(R(0), l2min);
    } else {
        Acc<M, R, true> l1;
        l1.init(0);
        l1.term(mu, La, rLa);
        out.L = l1.result();
        out.rL = l1.radius_bound();
        out.alo = N::max(R(0), N::sub_rd(out.L.k, out.rL));
    }
    out.dev = R(0.5 * 32) * N::U * (N::abs(mlo) + N::abs(mhi)) * ((mlo > R(0) ? out.ahi : R(0)) + out.alo);
}

// The same evaluation in FP64 arithmetic from the FP32 record, narrowed back
// to FP32 forms soundly: each coefficient is rounded to nearest and the
// rounding errors, summed (|p_j| <= 1), move the constant outward; radii,
// constants and the scalar enclosure round outward.  This takes the Exp
// stage's tangent and secant points (the ends of the m interval) in FP64 for
// the pairs whose m interval is so wide that FP32 cannot carry its ends to
// the bounds' tolerance.  Kept out of line: it runs for few evaluations, and
// the FP32 sweep keeps its registers.
template <int M>
__device__ __noinline__ AlphaOut<M, float> pixel_alpha_fp64(const float *r, float ux, float uy,
                                                           double *m_out = nullptr)
{
    AlphaOut<M, float> out;
    AlphaOut<M, double> d;
    pixel_alpha<M, double, float>(r, (double)ux, (double)uy, d, m_out);
    double eL = 0.0, eU = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        out.L.c[j] = __double2float_rn(d.L.c[j]);
        out.U.c[j] = __double2float_rn(d.U.c[j]);
        eL = __dadd_ru(eL, fabs(__dsub_rn(d.L.c[j], (double)out.L.c[j])));
        eU = __dadd_ru(eU, fabs(__dsub_rn(d.U.c[j], (double)out.U.c[j])));
    }
    out.L.k = __double2float_rd(__dsub_rd(d.L.k, eL));
    out.U.k = __double2float_ru(__dadd_ru(d.U.k, eU));
    out.rL = __double2float_ru(__dadd_ru(d.rL, eL));
    out.rU = __double2float_ru(__dadd_ru(d.rU, eU));
    out.alo = __double2float_rd(d.alo);
    out.ahi = __double2float_ru(d.ahi);
    out.dev = 0.f;
    return out;
}

// Colour accumulator: sum_i w_i F_i per channel, with the rounding error of
// the round-to-nearest coefficient sums bounded step by step:
//   each step's error <= min(u * sum_j |acc_j|, w * r_F), and
//   sum_j |acc_j| <= Q = sum of w * r_F so far (times 1.01 for the error
//   already accumulated, valid below 10^5 steps in FP32).
// Colours lie in [0, 1], so every channel's weight w = T c is at most T and
// one pair Q, err computed with T in place of w bounds all three channels.
template <int M, bool DN, class R = float> struct ColourAcc {
    using N = Num<R>;
    R c[3][M];
    R k[3];
    R q, err;
    int steps;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
            for (int j = 0; j < M; ++j) c[ch][j] = 0;
            k[ch] = 0;
        }
        q = 0;
        err = 0;
        steps = 0;
    }
    __device__ __forceinline__ void add(R T, const R *col, const LF<M, R> &F, R rF)
    {
        const R u = N::U * R(1.01);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const R w = DN ? N::mul_rd(T, col[ch]) : N::mul_ru(T, col[ch]);
            axpy_rn<M>(w, F.c, c[ch]);
            k[ch] = DN ? N::fma_rd(w, F.k, k[ch]) : N::fma_ru(w, F.k, k[ch]);
        }
        const R t = N::mul_ru(T, rF);
        q = N::add_ru(q, t);
        err = N::add_ru(err, N::min(N::mul_ru(q, u), t));
        ++steps;
    }
    __device__ __forceinline__ R radius(int ch) const
    {
        R r = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) r = N::add_ru(r, N::abs(c[ch][j]));
        return N::add_ru(N::add_ru(r, err), N::mul_ru((R)steps, N::TINY));
    }
    // the outward concretisation of the accumulated form
    __device__ __forceinline__ R bound(int ch) const
    {
        const R r = radius(ch);
        return DN ? N::sub_rd(k[ch], r) : N::add_ru(k[ch], r);
    }
    // constant minus radius rounded up: at least the computed lower bound
    __device__ __forceinline__ R upper_min(int ch) const
    {
        R r = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) r = N::add_rd(r, N::abs(c[ch][j]));
        return N::sub_ru(k[ch], N::add_rd(r, err));
    }
};

// Relational upper transmittance (the AR_BLEND_RELATIONAL mode; a tighter
// blend than the interval Prod of Algorithm 4).  F is an affine upper form of
// the running product over the Gaussians already certainly in front, y its
// interval bound (rounded up).  Each factor x = 1 - a_j, with x >= x_lo =
// 1 - a_hi(j) and x <= X(p) (X = 1 - L_j where a_lo(j) > 0, so that X stays
// below 1 - a_lo(j); else the constant 1), enters through the McCormick plane
//   (y - prod)(x - x_lo) >= 0  =>  prod x <= y X + x_lo (F - y),
// which is sound because y >= 0 and x_lo >= 0 weight upper bounds; step by
// step F <= y at every pose of the cell.  The coefficients are rounded to
// nearest: each is within 2u (1 + u) of |y L_j.c| + |x_lo F.c| (plus an
// underflow term), so 2.01 u r2 + TINY bounds their total error, which the
// constant takes; rF bounds sum |F.c|.
template <int M> struct RelT {
    LF<M, float> F;
    float rF, y;
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int j = 0; j < M; ++j) F.c[j] = 0.f;
        F.k = 1.f;
        rF = 0.f;
        y = 1.f;
    }
    __device__ __forceinline__ void absorb(const LF<M, float> &L, float rL, float alo, float ahi)
    {
        const float xlo = __fsub_rd(1.f, ahi);
        float k2 = __fmul_ru(xlo, __fsub_ru(F.k, y));
        float r2 = __fmul_ru(xlo, rF);
        if (alo > 0.f) {
#pragma unroll
            for (int j = 0; j < M; ++j) F.c[j] = __fmaf_rn(-y, L.c[j], __fmul_rn(xlo, F.c[j]));
            k2 = __fadd_ru(k2, __fmul_ru(y, __fsub_ru(1.f, L.k)));
            r2 = __fadd_ru(r2, __fmul_ru(y, rL));
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) F.c[j] = __fmul_rn(xlo, F.c[j]);
            k2 = __fadd_ru(k2, y);
        }
        const float e = __fmaf_ru(r2, 2.01f * Num<float>::U, Num<float>::TINY);
        F.k = __fadd_ru(k2, e);
        rF = __fadd_ru(r2, e);
        y = __fmul_ru(y, __fsub_ru(1.f, alo));
    }
};

struct EvInfo {
    uint32_t rec;   // record index within the cell
    uint32_t bits;  // bit 0: upper endpoint, bit 1: key equals the previous entry's key
};

// Early exit.  Write PA, PB for the running transmittance products and
// "open" for the Gaussians of this pixel whose lower endpoint has been swept
// but not yet their upper one (n_open of them).  Every depth-key interval is open (klo < khi:
// the keys are padded), so the lower endpoint of a Gaussian that has not yet
// started precedes, with a strictly smaller key, the upper endpoint of every
// Gaussian behind it.
//  - upper: a later term T_hi c U has U >= a >= 0 at every pose of the cell,
//    so the constant of its U form is >= 0 and the upward-rounded constant of
//    the upper sum only grows; its final bound is at least that constant, so
//    once the constant is >= 1 in every channel the clipped bound is 1.
//    Otherwise the remaining terms add at most Eh = (events left) 1.1 PB to
//    the maximum over the cell (T_hi <= PB, max U <= 1.0625 o).
//  - lower: a later term T_lo c L has |L| <= a_hi over the cell.  For the
//    Gaussians not yet started, taken in the order of their upper endpoints,
//    T_lo(i_k) <= PA prod_{l<k} (1 - a_hi(i_l)) (the division by 1 - a_hi at
//    the upper endpoint removes i_k's own factor), so their terms telescope
//    to at most PA; an open Gaussian i adds at most T_lo(i) a_hi(i) <=
//    PA a_hi(i) / (1 - a_hi(i)).  open_w is the sum of these ratios over the
//    open Gaussians, each rounded up and kept with upward-rounded additions
//    and subtractions (so it is never below the exact sum); n_open / (1 -
//    o_max) bounds it too.  So the remaining terms move the minimum over the
//    cell by at most El = PA (1 + min(open_w, n_open / (1 - o_max))) (times
//    1.01 for the rounding of PA), and once (constant - radius) + El <= 0 in
//    every channel the clipped bound is 0.
// Otherwise a side also stops once its E is below EXIT_EPS; its bound is then
// widened by E, which keeps it sound and within EXIT_EPS of the full sweep.
// EXIT_EPS is a tenth of the 1e-4 to which the bounds match a full FP64
// sweep: it leaves 9e-5 to the single-precision arithmetic, and it saves a
// fifth of the opacity evaluations against 5e-8.
// A pixel stops when both sides have; a tile stops when all its pixels have.
constexpr float EXIT_EPS = 1e-5f;
// an incomplete list (a depth prefix) of a segment with at most this many
// entries in full is not swept but deferred to the next round
constexpr uint32_t SHORT_DEFER = 256;

// a / (1 - a) rounded up, for 0 <= a < 1 (__fdividef is within 2 ulp here;
// the factor 1 + 2^-21 covers that)
__device__ __forceinline__ float open_ratio_up(float a)
{
    const float den = __fsub_rd(1.f, a);
    return den > 0.f ? __fmul_ru(__fdividef(a, den), 1.000000477f) : 3.0e38f;
}

// Shared-memory layout of the render kernel (dynamic; about 70 KB at six
// pose variables, tile 16, chunks of 16 and a ring of 4, so two CTAs fit on an SM):
//   two buffers (one in the FP64 instance), each with the records staged for
//   a chunk of CH events, their event info and pixel boxes (the next chunk is
//   copied in while the current one is swept),
//   and a per-thread ring of the last RING opacity evaluations made at lower
//   endpoints (record id + alo, ahi, rL, L, the latter as 16-byte vectors),
//   stored column-per-thread so that every access is bank-conflict free.  The ring lets the upper endpoint of
//   a Gaussian reuse the evaluation made at its lower endpoint; an upper
//   endpoint whose evaluation has left the ring evaluates again.
// NTH: threads per CTA (the tile's pixels, or one warp for the FP64 instance);
// NBUF: chunk buffers (two, or one for the FP64 instance, whose one-warp CTAs
// then fit fourteen to an SM instead of nine)
template <int M, int TS, int CH, int RING, int NTH = TS * TS, int NBUF = 2> struct RenderSmem {
    static constexpr int NT = NTH;
    static constexpr int PAY = M + 4;  // alo, ahi, rL, L.k, L.c[M]
    static constexpr int PV = (PAY + 3) / 4;  // ... as 16-byte vectors (the last one padded)
    static constexpr size_t REC = NBUF * sizeof(float) * CH * Rec<M>::WIDTH;  // chunk buffers
    static constexpr size_t EV = NBUF * sizeof(EvInfo) * CH;
    static constexpr size_t BOX = NBUF * sizeof(PixBox) * CH;
    static constexpr size_t RID = sizeof(uint32_t) * RING * NT;
    static constexpr size_t RPAY = sizeof(float4) * RING * PV * NT;
    static constexpr size_t BYTES = REC + EV + BOX + RID + RPAY + 16;
};

// element i of an array of float4 (i a compile-time constant after unrolling)
template <int N>
__device__ __forceinline__ float f4_at(const float4 (&v)[N], int i)
{
    const float4 &t = v[i >> 2];
    return (i & 3) == 0 ? t.x : (i & 3) == 1 ? t.y : (i & 3) == 2 ? t.z : t.w;
}

// 16-byte asynchronous global -> shared copies (completed by cp_async_wait_all)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Two 256-thread CTAs share an SM (16 warps: the sweep is latency-bound, and
// 128 registers per thread cost it a few spills but double the warps that hide
// the FMA latency); 64-thread CTAs are not limited.
template <int TS> struct RenderOcc {
    static constexpr int MIN_BLOCKS = TS * TS >= 256 ? 2 : 1;
};
// The FP64 instance runs one warp per CTA, sixteen CTAs per SM (the same
// registers per thread as two 256-thread CTAs)
template <int TS, bool F64> struct RenderShape {
    static constexpr int NTH = F64 ? 32 : TS * TS;
    static constexpr int NBUF = F64 ? 1 : 2;  // chunk buffers (see RenderSmem)
    static constexpr int MIN_BLOCKS = F64 ? 16 : RenderOcc<TS>::MIN_BLOCKS;
    static constexpr int MASKW = TS * TS / 32 + 1;  // words per listed segment: pixel mask, abandon flag
};

// Persistent grid: each CTA takes (cell, tile) segments from the active list
// (longest first in the first round) through an atomic counter until none
// are left; block = TS*TS threads.
//
// Windowed rounds: only the records of the pairs whose lower endpoints lie in
// the first `window` entries of an active segment have been built.  A
// segment that would stage an entry beyond its window before all its pixels
// have stopped is abandoned (no output written) and appended to next_active;
// the next round builds the records of a wider window and sweeps it again
// from its start.  The sweep is deterministic, so the restarted segment
// gives the same bounds it would have given in one pass.
//
// Precision (F64): the opacity evaluations whose weighted FP32 deviation
// estimate exceeds fp64_dev are taken in FP64 (pixel_alpha_fp64).  The FP32
// sweep (F64 = false) keeps that out-of-line call out of its code: it sweeps
// every segment in FP32, writes the bounds of the pixels that met no such
// evaluation, and appends a segment where some pixel did to precise_list,
// with the mask of those pixels (one word per warp) in precise_mask.  The
// F64 = true instance sweeps the listed segments again from their start for
// the masked pixels alone (the others start as stopped and write nothing).
// The decision is per pixel, taken from the pixel's own sweep, so every pixel
// gets the bounds one FP64-capable sweep would give it.  The FP64 instance
// runs one warp per CTA: each work item is a listed segment and a group of up
// to 32 of its listed pixels, so that many segments are in flight at once.
template <int M, int TS, int CH, int RING, bool REL, bool F64>
__global__ void __launch_bounds__(RenderShape<TS, F64>::NTH, RenderShape<TS, F64>::MIN_BLOCKS) render_kernel(
    const float *__restrict__ recs, const PixBox *__restrict__ boxes, const uint32_t *__restrict__ seg_start,
    const uint32_t *__restrict__ seg_end, const uint32_t *__restrict__ seg_total,
    const uint32_t *__restrict__ cell_ev, const uint32_t *__restrict__ active, const uint32_t *__restrict__ n_active,
    uint32_t window, uint32_t *__restrict__ next_active, uint32_t *__restrict__ n_next,
    uint32_t *__restrict__ precise_list, uint32_t *__restrict__ n_precise, uint32_t *__restrict__ precise_mask,
    uint32_t *__restrict__ sweep_hist,
    const uint32_t *__restrict__ entry_ev, const uint32_t *__restrict__ ev_val,
    const uint64_t *__restrict__ ev_key, int W, int H, int ntx, int n_tiles, int64_t n_gauss,
    float k_open, float fp64_dev, float *__restrict__ out_lo, float *__restrict__ out_hi,
    unsigned long long *__restrict__ counters, unsigned int *__restrict__ work, int direct)
{
    using RL = Rec<M>;
    using SH = RenderShape<TS, F64>;
    using SM = RenderSmem<M, TS, CH, RING, SH::NTH, SH::NBUF>;
    constexpr int NT = SH::NTH;      // threads
    constexpr int NPIX = TS * TS;    // pixels of a tile
    constexpr int GROUPS = F64 ? NPIX / 32 : 1;  // work items per listed segment
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float(*s_rec2)[RL::WIDTH] = reinterpret_cast<float(*)[RL::WIDTH]>(smem_raw);        // [2 * CH]
    EvInfo *s_ev2 = reinterpret_cast<EvInfo *>(smem_raw + SM::REC);                    // [2 * CH]
    PixBox *s_box2 = reinterpret_cast<PixBox *>(smem_raw + SM::REC + SM::EV);          // [2 * CH]
    uint32_t *s_rid = reinterpret_cast<uint32_t *>(smem_raw + SM::REC + SM::EV + SM::BOX);
    float4 *s_pay = reinterpret_cast<float4 *>(smem_raw + SM::REC + SM::EV + SM::BOX + SM::RID);
    uint32_t *s_next = reinterpret_cast<uint32_t *>(smem_raw + SM::REC + SM::EV + SM::BOX + SM::RID + SM::RPAY);
    const int tid = threadIdx.x;
    uint32_t evals = 0, recomp = 0, wide = 0;
    const uint32_t n_seg = *n_active;

    // direct: one CTA per active segment (the grid covers them all), so that
    // CTAs finish one by one and a higher-priority stream's work can take
    // their SMs; else persistent CTAs take segments from the work counter
    for (uint32_t round = 0;; ++round) {
        if (tid == 0) *s_next = direct ? (round == 0 ? blockIdx.x : 0xffffffffu) : atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t item = *s_next;
        __syncthreads();
        const uint32_t wk = item / GROUPS, grp = item % GROUPS;
        if (wk >= n_seg) break;
        const uint32_t seg = active[wk];
        const int cell = (int)(seg / (uint32_t)n_tiles);
        const int tile = (int)(seg - (uint32_t)cell * (uint32_t)n_tiles);
        const int tx = tile % ntx, ty = tile / ntx;
        // each warp covers an 8 x 4 block of the tile, so that the pixel boxes
        // of small Gaussians cut fewer warps and warps finish together
        const int wb = tid >> 5, ln = tid & 31;
        // the pixel this thread sweeps, by its thread index in the FP32
        // sweep's layout; the FP64 instance takes the listed pixels of rank
        // 32 grp + tid among the mask's set bits
        int pid = tid;
        bool active = true;
        if (F64) {
            const uint32_t *pm = precise_mask + (size_t)wk * SH::MASKW;
            int rem = (int)grp * 32 + tid;
            pid = -1;
#pragma unroll
            for (int w = 0; w < NPIX / 32; ++w) {
                uint32_t m = pm[w];
                const int c = __popc(m);
                if (pid < 0 && rem < c) {
                    for (int k = 0; k < rem; ++k) m &= m - 1u;
                    pid = w * 32 + __ffs(m) - 1;
                } else if (pid < 0) {
                    rem -= c;
                }
            }
            active = pid >= 0;
            if (!active) pid = 0;  // a position of the tile; the thread sweeps nothing
            if (!__syncthreads_or(active)) continue;  // a group past the segment's listed pixels
        }
        const int pwb = pid >> 5, pln = pid & 31;
        const int px = tx * TS + (pwb % (TS / 8)) * 8 + (pln & 7);
        const int py = ty * TS + (pwb / (TS / 8)) * 4 + (pln >> 3);
        const bool inside = px < W && py < H;
        const float ux = px + 0.5f, uy = py + 0.5f;
        const uint32_t b0 = seg_start[seg], b1 = seg_end[seg];
        // entries of the segment's full list; the list at hand may be a
        // prefix of it (the first binning phase)
        const uint32_t total = seg_total ? seg_total[seg] : b1 - b0;
        const bool incomplete = total > b1 - b0;
        const float *rec_cell = recs + (size_t)cell * n_gauss * RL::WIDTH;
        const PixBox *box_cell = boxes + (size_t)cell * n_gauss;

        ColourAcc<M, true> lo;
        ColourAcc<M, false> hi;
        lo.init();
        hi.init();
        float PA = 1.f, PB = 1.f, PAp = 1.f, PBp = 1.f;
        // relational mode: F of the Gaussians absorbed so far; rel_tie once
        // one has been absorbed in the current group of equal keys (a query
        // later in that group takes the interval term: the group's absorptions
        // are not certainly in front of it)
        RelT<M> rel;
        bool rel_tie = false;
        // relational mode: the constants of the interval terms alone (the
        // upper sum of the interval blend); where they reach 1 in every
        // channel the upper bound is taken as 1, as the interval blend's is
        float hk[3] = {0.f, 0.f, 0.f};
        if (REL) rel.init();
        int n_open = 0;      // Gaussians of this pixel between their two endpoints
        float open_w = 0.f;  // sum over them of a_hi / (1 - a_hi), rounded up
        uint32_t c_rec = 0xffffffffu;  // register copy of the latest evaluation
        AlphaOut<M> cache;
#pragma unroll
        for (int k = 0; k < RING; ++k) s_rid[k * NT + tid] = 0xffffffffu;
        uint32_t head = 0;
        // the FP64 instance sweeps only the pixels the FP32 sweep listed
        bool done = !inside || !active;
        float lo_adj = 0.f, hi_adj = 0.f;  // -1: decided 0 / 1; >= 0: widening for skipped events
        // the upper sums' constants have reached 1 in every channel (interval
        // blend): final, because they only grow, so the upper bounds are 1
        // and the sweep stops adding to them
        bool hi_fix = false;
        bool abandoned = false;
        uint32_t swept = b1 - b0;  // entries swept before the tile stopped
        uint32_t seg_evals = 0, seg_recomp = 0, seg_wide = 0;
        bool wide_hit = false;  // F64 = false: an evaluation needed FP64

        // Copy the chunk starting at entry sb into buffer bf: warp w takes
        // events EPW w .. EPW w + EPW - 1, its first EPW lanes read their event
        // info, and the whole warp copies their record rows asynchronously.
        constexpr int NWARP = NT / 32, EPW = CH / NWARP, ROW4 = RL::WIDTH / 4;
        static_assert(CH % NWARP == 0 && EPW <= 32, "chunk must split evenly over the warps");
        auto stage = [&](int bf, uint32_t sb) {
            const int k0 = wb * EPW;
            uint32_t rec = 0;
            const bool have_ev = ln < EPW && sb + (uint32_t)(k0 + ln) < b1;
            if (have_ev) {
                const uint32_t i = sb + (uint32_t)(k0 + ln);
                const uint32_t e = entry_ev[i];
                const uint32_t v = ev_val[e];
                uint32_t bits = v & 1u;
                if (i > b0 && ev_key[entry_ev[i - 1]] == ev_key[e]) bits |= 2u;
                rec = (v >> 1) - (uint32_t)(cell * n_gauss);
                s_ev2[bf * CH + k0 + ln] = EvInfo{rec, bits};
                s_box2[bf * CH + k0 + ln] = box_cell[rec];
            }
            const uint32_t nv = __ballot_sync(0xffffffffu, have_ev);
            for (int q0 = 0; q0 < EPW * ROW4; q0 += 32) {
                const int q = q0 + ln;
                const int k = min(q / ROW4, EPW - 1);
                const uint32_t rk = __shfl_sync(0xffffffffu, rec, k);
                if (q < EPW * ROW4 && ((nv >> k) & 1u)) {
                    const int part = q - k * ROW4;
                    cp_async16(&s_rec2[bf * CH + k0 + k][4 * part], rec_cell + (size_t)rk * RL::WIDTH + 4 * part);
                }
            }
        };
        int buf = 0;
        // a short list held only in part is deferred to the next round, which
        // has it in full: the segments that outrun their depth prefix are
        // mostly short (sparse tiles), and a sweep of their prefix would be
        // done twice
        if (incomplete && total <= SHORT_DEFER) abandoned = true;
        if (b0 < b1 && !abandoned) stage(0, b0);
        // a complete list ends the sweep when it runs out; a prefix only when
        // every pixel has stopped, or by abandoning the segment at the first
        // chunk it does not hold in full (the next binning phase gives the
        // segment its full list, and the sweep starts again: the exit tests
        // fall at the same entries, so the bounds are those of one sweep)
        for (uint32_t base = b0; !abandoned && (base < b1 || incomplete); base += CH, buf = (buf + 1) % SH::NBUF) {
            if (!done) {
                const float left = (float)(total - (base - b0));
                // PA is rounded down; 1.01 covers its relative error for < 10^5 factors
                const float ow = fminf(open_w, __fmul_ru((float)n_open, k_open));
                const float elo2 = __fmul_ru(__fmul_ru(PA, 1.01f), __fadd_ru(ow, 1.f));
                const float ehi2 = __fmul_ru(1.1f, __fmul_ru(left, PB));
                bool lo_zero = true, hi_one = true;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    lo_zero = lo_zero && __fadd_ru(lo.upper_min(ch), elo2) <= 0.f;
                    hi_one = hi_one && (REL ? hk[ch] : hi.k[ch]) >= 1.f;
                }
                if (!REL) hi_fix = hi_one;
                const bool lo_dec = lo_zero || elo2 <= EXIT_EPS;
                const bool hi_dec = hi_one || ehi2 <= EXIT_EPS;
                if (lo_dec && hi_dec) {
                    done = true;
                    lo_adj = lo_zero ? -1.f : elo2;
                    hi_adj = hi_one ? -1.f : ehi2;
                }
            }
            // one buffer: the chunk is copied in once every thread has swept
            // the previous one
            if (SH::NBUF == 1 && base != b0) {
                __syncthreads();
                stage(0, base);
            }
            cp_async_wait_all();  // this thread's copies of the current chunk
            if (__syncthreads_and(done)) {  // ... and everyone's, now visible
                swept = base - b0;
                break;
            }
            if (incomplete && base + CH > b1) {  // the chunk reaches beyond the prefix
                abandoned = true;
                break;
            }
            const int cnt = (int)min((uint32_t)CH, b1 - base);
            if (base + (uint32_t)cnt - b0 > window) {  // records beyond the window are not built
                abandoned = true;
                break;
            }
            // the next chunk streams in while this one is swept; the buffer it
            // overwrites was swept by every thread before the barrier above
            if (SH::NBUF == 2 && base + CH < b1) stage(buf ^ 1, base + CH);
            const EvInfo *s_ev = s_ev2 + buf * CH;
            const PixBox *s_box = s_box2 + buf * CH;
            float(*s_rec)[RL::WIDTH] = s_rec2 + buf * CH;
            if (done) continue;
            for (int e = 0; e < cnt; ++e) {
                const EvInfo ev = s_ev[e];
                if (!(ev.bits & 2u)) {
                    PA = __fmul_rd(PA, PAp);
                    PB = __fmul_ru(PB, PBp);
                    PAp = 1.f;
                    PBp = 1.f;
                    rel_tie = false;
                }
                const PixBox bx = s_box[e];
                if (px < bx.x0 || px > bx.x1 || py < bx.y0 || py > bx.y1) continue;
                const float *r = s_rec[e];
                const bool lower = !(ev.bits & 1u);
                n_open += lower ? 1 : -1;
                bool have = !lower && c_rec == ev.rec;
                if (!lower && !have) {
                    int hit = -1;
#pragma unroll
                    for (int k = 0; k < RING; ++k)
                        if (s_rid[k * NT + tid] == ev.rec) hit = k;
                    if (hit >= 0) {
                        const float4 *pp = s_pay + (size_t)hit * SM::PV * NT + tid;
                        float4 v[SM::PV];
#pragma unroll
                        for (int q = 0; q < SM::PV; ++q) v[q] = pp[q * NT];
                        cache.alo = v[0].x;
                        cache.ahi = v[0].y;
                        cache.rL = v[0].z;
                        cache.L.k = v[0].w;
#pragma unroll
                        for (int j = 0; j < M; ++j) cache.L.c[j] = f4_at(v, 4 + j);
                        have = true;
                    }
                }
                if (!have) {
                    pixel_alpha<M>(r, ux, uy, cache, (float *)nullptr, lower && !hi_fix);
                    // a wide m interval: the Exp stage's points in FP64 where
                    // the FP32 deviation, weighted by how much this pixel's
                    // bounds can still move with it, exceeds the threshold.
                    // The upper bound moves by at most T_hi = PB times it,
                    // and not at all once its constant has reached 1 in every
                    // channel (final: the constant only grows); the lower one
                    // by at most T_lo (PA here, or PA / (1 - a_hi) at an
                    // upper endpoint whose evaluation left the ring), and not
                    // at all once the early exit's test decides it 0 on the
                    // state before this event (final as well).  The weight is
                    // at most 2, so smaller deviations skip it.
                    if (cache.dev > 0.5f * fp64_dev) {
                        bool sat = true, dead = true;
                        const int nb = n_open + (lower ? -1 : 1);  // before this event
                        const float ow = fminf(open_w, __fmul_ru((float)nb, k_open));
                        const float elo = __fmul_ru(__fmul_ru(PA, 1.01f), __fadd_ru(ow, 1.f));
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            sat = sat && (REL ? hk[ch] : hi.k[ch]) >= 1.f;
                            dead = dead && __fadd_ru(lo.upper_min(ch), elo) <= 0.f;
                        }
                        const float tlo = dead ? 0.f
                                               : (lower ? PA : fminf(1.f, __fdividef(PA, fmaxf(1.f - cache.ahi, 1e-6f))));
                        if (cache.dev * ((sat ? 0.f : PB) + tlo) > fp64_dev) {
                            if (F64) {
                                cache = pixel_alpha_fp64<M>(r, ux, uy);
                                ++seg_wide;
                            } else {
                                wide_hit = true;
                            }
                        }
                    }
                    // a MatrixInv fallback is a constant [0, o]: not an evaluation
                    if (!(__float_as_uint(r[RL::FLAGS]) & F_FALLBACK)) {
                        if (lower) ++seg_evals; else ++seg_recomp;
                    }
                }
                c_rec = ev.rec;
                // colour box: c_lo in the lower sum, c_hi in the upper one
                const float col[3] = {r[RL::COL], r[RL::COL + 1], r[RL::COL + 2]};
                const float colh[3] = {r[RL::COL_HI], r[RL::COL_HI + 1], r[RL::COL_HI + 2]};
                if (lower) {
                    if (!hi_fix) hi.add(PB, colh, cache.U, cache.rU);
                    if (REL) {
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) hk[ch] = __fmaf_ru(__fmul_ru(PB, colh[ch]), cache.U.k, hk[ch]);
                    }
                    if (REL && !rel_tie && cache.alo > 0.f) {
                        // McCormick plane of T a: PB U + a_lo (F - PB), F <= PB
                        LF<M, float> D = rel.F;
                        D.k = __fsub_ru(rel.F.k, PB);
                        hi.add(cache.alo, colh, D, rel.rF);
                    }
                    PAp = __fmul_rd(PAp, __fsub_rd(1.f, cache.ahi));
                    open_w = __fadd_ru(open_w, open_ratio_up(cache.ahi));
                    const int k = (int)(head % RING);
                    ++head;
                    s_rid[k * NT + tid] = ev.rec;
                    float4 *pp = s_pay + (size_t)k * SM::PV * NT + tid;
                    auto pay = [&](int i) { return i < 4 ? (i == 0 ? cache.alo : i == 1 ? cache.ahi : i == 2 ? cache.rL : cache.L.k)
                                                         : (i < 4 + M ? cache.L.c[i < 4 + M ? i - 4 : 0] : 0.f); };
#pragma unroll
                    for (int q = 0; q < SM::PV; ++q) pp[q * NT] = make_float4(pay(4 * q), pay(4 * q + 1), pay(4 * q + 2), pay(4 * q + 3));
                } else {
                    open_w = fmaxf(0.f, __fsub_ru(open_w, open_ratio_up(cache.ahi)));
                    const uint32_t flags = __float_as_uint(r[RL::FLAGS]);
                    float T = PA;
                    if (flags & F_OPEN) {
                        const float den = __fsub_ru(1.f, cache.ahi);
                        T = (den > 0.f) ? Num<float>::div_pos_dn(PA, den) : 0.f;
                    }
                    lo.add(T, col, cache.L, cache.rL);
                    PBp = __fmul_ru(PBp, __fsub_ru(1.f, cache.alo));
                    if (REL) {
                        rel.absorb(cache.L, cache.rL, cache.alo, cache.ahi);
                        rel_tie = true;
                    }
                }
            }
        }
        if (abandoned) {
            // (the FP64 instance's groups of one segment list it once)
            if (tid == 0 && (!F64 || atomicOr(&precise_mask[(size_t)wk * SH::MASKW + NPIX / 32], 1u) == 0u)) {
                next_active[atomicAdd(n_next, 1u)] = seg;
                if (counters) atomicAdd(&counters[5], 1ull);
            }
            continue;
        }
        if (!F64 && __syncthreads_or(wide_hit)) {
            // list the segment with the mask of its pixels that need FP64
            // (the slot goes through s_next[1]: s_next[0], the work index, is
            // rewritten at the next segment's start while others may read this)
            if (tid == 0) {
                const uint32_t slot = atomicAdd(n_precise, 1u);
                precise_list[slot] = seg;
                precise_mask[(size_t)slot * SH::MASKW + NPIX / 32] = 0u;  // the FP64 instance's abandon flag
                s_next[1] = slot;
                if (counters) atomicAdd(&counters[7], 1ull);
            }
            __syncthreads();
            const uint32_t m = __ballot_sync(0xffffffffu, wide_hit);
            if ((tid & 31) == 0) precise_mask[(size_t)s_next[1] * SH::MASKW + (tid >> 5)] = m;
        }
        if (!F64 && sweep_hist && tid == 0) atomicAdd(&sweep_hist[min(swept / 32u, 255u)], 1u);
        // where in its cell's depth order the segment stopped (64 buckets of
        // the cell's sorted events), weighted by its full length and counted:
        // the host sizes the next render's depth prefix from them
        if (!F64 && sweep_hist && cell_ev && tid == 0 && b1 > b0) {
            const uint32_t c0 = cell_ev[cell], ec = cell_ev[cell + 1] - c0;
            const uint32_t stop = entry_ev[b0 + (swept ? swept : 1u) - 1u];
            const uint32_t bkt = ec ? (uint32_t)min((uint64_t)(stop - c0) * 64u / ec, (uint64_t)63) : 0u;
            atomicAdd(reinterpret_cast<unsigned long long *>(sweep_hist + 256) + bkt, (unsigned long long)total);
            atomicAdd(sweep_hist + 384 + bkt, 1u);
        }
        evals += seg_evals;
        recomp += seg_recomp;
        wide += seg_wide;
        if (REL && hk[0] >= 1.f && hk[1] >= 1.f && hk[2] >= 1.f) hi_adj = -1.f;
        // pixels listed for the FP64 sweep, and in it the pixels not listed,
        // leave their outputs to the other instance
        if (inside && active && (F64 || !wide_hit)) {
            const size_t o = ((size_t)cell * H * W + (size_t)py * W + px) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                out_lo[o + ch] = lo_adj < 0.f ? 0.f : clamp01(__fsub_rd(lo.bound(ch), lo_adj));
                out_hi[o + ch] = hi_adj < 0.f ? 1.f : clamp01(__fadd_ru(hi.bound(ch), hi_adj));
            }
        }
    }
    if (counters) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, evals);
        const uint32_t b = __reduce_add_sync(0xffffffffu, recomp);
        const uint32_t c = __reduce_add_sync(0xffffffffu, wide);
        if ((tid & 31) == 0) {
            if (a) atomicAdd(&counters[0], (unsigned long long)a);
            if (b) atomicAdd(&counters[1], (unsigned long long)b);
            if (c) atomicAdd(&counters[6], (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// Plain FP64 renderer: the comparison path for the batched FP32 renderer.
// One CTA per (cell, tile) segment, one thread per pixel; FP64 records and
// FP64 arithmetic (outward rounded), every event of the segment swept (no
// early exit), and the opacity bounds evaluated again at each upper endpoint
// (no cache).  The host drives it one cell per launch sequence.
template <int M, int TS, int CH>
__global__ void __launch_bounds__(TS *TS) render_plain_kernel(
    const double *__restrict__ recs, const PixBox *__restrict__ boxes, const uint32_t *__restrict__ seg_start,
    const uint32_t *__restrict__ seg_end, const uint32_t *__restrict__ entry_ev, const uint32_t *__restrict__ ev_val,
    const uint64_t *__restrict__ ev_key, int W, int H, int ntx, int n_tiles, int64_t n_gauss,
    float *__restrict__ out_lo, float *__restrict__ out_hi)
{
    using RL = Rec<M>;
    using N = Num<double>;
    __shared__ __align__(16) double s_rec[CH][RL::WIDTH];
    __shared__ EvInfo s_ev[CH];
    __shared__ PixBox s_box[CH];
    const int tid = threadIdx.x;
    const uint32_t seg = blockIdx.x;
    const int cell = (int)(seg / (uint32_t)n_tiles);
    const int tile = (int)(seg - (uint32_t)cell * (uint32_t)n_tiles);
    const int px = (tile % ntx) * TS + (tid % TS);
    const int py = (tile / ntx) * TS + (tid / TS);
    const bool inside = px < W && py < H;
    const double ux = px + 0.5, uy = py + 0.5;
    const uint32_t b0 = seg_start[seg], b1 = seg_end[seg];
    const double *rec_cell = recs + (size_t)cell * n_gauss * RL::WIDTH;
    const PixBox *box_cell = boxes + (size_t)cell * n_gauss;

    ColourAcc<M, true, double> lo;
    ColourAcc<M, false, double> hi;
    lo.init();
    hi.init();
    double PA = 1, PB = 1, PAp = 1, PBp = 1;
    AlphaOut<M, double> a;
    for (uint32_t base = b0; base < b1; base += CH) {
        const int cnt = (int)min((uint32_t)CH, b1 - base);
        if (tid < cnt) {
            const uint32_t i = base + tid;
            const uint32_t e = entry_ev[i];
            const uint32_t v = ev_val[e];
            uint32_t bits = v & 1u;
            if (i > b0 && ev_key[entry_ev[i - 1]] == ev_key[e]) bits |= 2u;
            const uint32_t rec = (v >> 1) - (uint32_t)(cell * n_gauss);
            s_ev[tid] = EvInfo{rec, bits};
            s_box[tid] = box_cell[rec];
        }
        __syncthreads();
        for (int t = tid; t < cnt * (RL::WIDTH / 2); t += TS * TS) {
            const int e = t / (RL::WIDTH / 2), q = t - e * (RL::WIDTH / 2);
            const double2 *src = reinterpret_cast<const double2 *>(rec_cell + (size_t)s_ev[e].rec * RL::WIDTH);
            reinterpret_cast<double2 *>(s_rec[e])[q] = src[q];
        }
        __syncthreads();
        if (inside) {
            for (int e = 0; e < cnt; ++e) {
                const EvInfo ev = s_ev[e];
                if (!(ev.bits & 2u)) {
                    PA = N::mul_rd(PA, PAp);
                    PB = N::mul_ru(PB, PBp);
                    PAp = 1;
                    PBp = 1;
                }
                const PixBox bx = s_box[e];
                if (px < bx.x0 || px > bx.x1 || py < bx.y0 || py > bx.y1) continue;
                const double *r = s_rec[e];
                pixel_alpha<M, double>(r, ux, uy, a);
                const double col[3] = {r[RL::COL], r[RL::COL + 1], r[RL::COL + 2]};
                const double colh[3] = {r[RL::COL_HI], r[RL::COL_HI + 1], r[RL::COL_HI + 2]};
                if (!(ev.bits & 1u)) {
                    hi.add(PB, colh, a.U, a.rU);
                    PAp = N::mul_rd(PAp, N::sub_rd(1.0, a.ahi));
                } else {
                    double T = PA;
                    if ((uint32_t)r[RL::FLAGS] & F_OPEN) {
                        const double den = N::sub_ru(1.0, a.ahi);
                        T = (den > 0.0) ? N::div_rd(PA, den) : 0.0;
                    }
                    lo.add(T, col, a.L, a.rL);
                    PBp = N::mul_ru(PBp, N::sub_ru(1.0, a.alo));
                }
            }
        }
        __syncthreads();
    }
    if (inside) {
        const size_t o = ((size_t)cell * H * W + (size_t)py * W + px) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            out_lo[o + ch] = __double2float_rd(clamp01(lo.bound(ch)));
            out_hi[o + ch] = __double2float_ru(clamp01(hi.bound(ch)));
        }
    }
}

// Test and diagnosis hook: the opacity relaxation of listed (record, pixel)
// triples, in FP32 (precision 0) or FP32 then FP64 where the renderer would
// take FP64 (precision 1: the threshold fp64_dev) or always (precision 2).
// Per triple DEBUG_ALPHA_W doubles: L.c[6 slots], L.k, U.c[6 slots], U.k,
// rL, rU, alo, ahi, dev, mlo, mhi, W[6] as (vlo, vhi), S, Rx, Ry as their
// concretised (lo, hi), flags, whether FP64 was taken.
constexpr int DEBUG_ALPHA_W = 42;
template <int M>
__global__ void debug_alpha_kernel(const float *__restrict__ recs, int n, const int64_t *__restrict__ gi,
                                   const int32_t *__restrict__ px, const int32_t *__restrict__ py, int precision,
                                   float fp64_dev, double *__restrict__ out)
{
    using RL = Rec<M>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float *r = recs + (size_t)gi[t] * RL::WIDTH;
    const float ux = px[t] + 0.5f, uy = py[t] + 0.5f;
    AlphaOut<M, float> a;
    float m32[2] = {0.f, 0.f};
    double m64[2] = {0.0, 0.0};
    if (precision == 3) pixel_alpha<M, float, float, true>(r, ux, uy, a, m32);
    else pixel_alpha<M>(r, ux, uy, a, m32);
    double mlo = m32[0], mhi = m32[1];
    int took = 0;
    if (precision == 2 || (precision == 1 && a.dev > fp64_dev)) {
        const float dev = a.dev;
        a = pixel_alpha_fp64<M>(r, ux, uy, m64);
        a.dev = dev;
        mlo = m64[0];
        mhi = m64[1];
        took = 1;
    }
    double *o = out + (size_t)t * DEBUG_ALPHA_W;
    for (int k = 0; k < DEBUG_ALPHA_W; ++k) o[k] = 0.0;
    for (int j = 0; j < M; ++j) { o[j] = a.L.c[j]; o[7 + j] = a.U.c[j]; }
    o[6] = a.L.k; o[13] = a.U.k;
    o[14] = a.rL; o[15] = a.rU; o[16] = a.alo; o[17] = a.ahi; o[18] = a.dev; o[19] = mlo; o[20] = mhi;
    for (int e = 0; e < 6; ++e) {
        o[21 + 2 * e] = -r[RL::W0 + e * RL::WS + M + 2];
        o[22 + 2 * e] = r[RL::W0 + e * RL::WS + M + 3];
    }
    const int sb[3] = {RL::S, RL::RX, RL::RY};
    for (int q = 0; q < 3; ++q) {
        o[33 + 2 * q] = -(double)r[sb[q] + M] - (double)r[sb[q] + M + 2];
        o[34 + 2 * q] = (double)r[sb[q] + M + 1] + (double)r[sb[q] + M + 2];
    }
    o[39] = (double)__float_as_uint(r[RL::FLAGS]);
    o[40] = took;
}

}  // namespace ar
