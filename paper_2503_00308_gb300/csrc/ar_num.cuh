// ar_num.cuh -- sound linear bounds over a pose cell, in directed rounding.
//
// A pose cell is a box; every pose variable is normalised to p in [-1, 1]^M.
// A bounded scalar holds two affine forms lo(p) <= v <= hi(p) (the
// piecewise-linear relations of Sec. 2.1 with one piece) plus their
// concretisation over the box.  Here the two forms share their coefficients
// (SB below); LF is a single form.
//
// Soundness in floating point: coefficients are computed round-to-nearest and
// the worst-case rounding error of every coefficient, summed over the box
// (|p_j| <= 1), is moved into the constant term, which itself is computed in
// the outward rounding direction (down for lower forms, up for upper forms).
// For a sum of n products a_t * F_t accumulated by a chain of n FMAs, the error
// of each coefficient is at most n u (1 + u)^n sum_t |a_t F_tj| (u = unit
// roundoff), so the constant moves by gamma_n * sum_t |a_t| r_t with r_t the
// radius of F_t.  A tiny absolute term covers subnormal rounding.
//
// The relaxations are the ones the abstract-rendering construction uses:
//   Mul x*y : averaged McCormick planes, y_m x + x_m y - (x_lo y_lo + x_hi y_hi)/2
//             below and y_m x + x_m y - (x_hi y_lo + x_lo y_hi)/2 above;
//   Sqr x^2 : tangent at the midpoint below, secant above;
//   Exp     : tangent at the lower end below, secant above (Table 2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ar {

template <class R> struct Num;

template <> struct Num<float> {
    static constexpr float U = 5.9604644775390625e-8f;  // 2^-24
    static constexpr float TINY = 1e-36f;
    static constexpr float BIG = 3.0e38f;
    __device__ static __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
    __device__ static __forceinline__ float add_ru(float a, float b) { return __fadd_ru(a, b); }
    __device__ static __forceinline__ float sub_rd(float a, float b) { return __fsub_rd(a, b); }
    __device__ static __forceinline__ float sub_ru(float a, float b) { return __fsub_ru(a, b); }
    __device__ static __forceinline__ float mul_rd(float a, float b) { return __fmul_rd(a, b); }
    __device__ static __forceinline__ float mul_ru(float a, float b) { return __fmul_ru(a, b); }
    __device__ static __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
    __device__ static __forceinline__ float fma_rd(float a, float b, float c) { return __fmaf_rd(a, b, c); }
    __device__ static __forceinline__ float fma_ru(float a, float b, float c) { return __fmaf_ru(a, b, c); }
    __device__ static __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    __device__ static __forceinline__ float div_rd(float a, float b) { return __fdiv_rd(a, b); }
    __device__ static __forceinline__ float div_ru(float a, float b) { return __fdiv_ru(a, b); }
    __device__ static __forceinline__ float sqrt_ru(float a) { return __fsqrt_ru(a); }
    // a / b to a few ulp, for weights where any value in [0, 1] is sound
    __device__ static __forceinline__ float div_weight(float a, float b) { return __fdividef(a, b); }
    // a / b rounded up (div_pos_up) or down (div_pos_dn) for a >= 0, b > 0.
    // CUDA documents __fdividef as within 2 ulp for b in [2^-126, 2^126]; with
    // a >= 2^-100 and b in [2^-120, 2^20] the quotient is normal, so its
    // relative error is at most 2^-22 and a directed product with 1 +- 2^-21
    // moves it past the exact value.  Other operands take the correctly
    // rounded division.
    __device__ static __forceinline__ bool fast_div_ok(float a, float b)
    {
        return a >= 0x1p-100f && b >= 0x1p-120f && b <= 0x1p20f;
    }
    __device__ static __forceinline__ float div_pos_up(float a, float b)
    {
        return fast_div_ok(a, b) ? __fmul_ru(__fdividef(a, b), 1.f + 4.76837158203125e-7f) : __fdiv_ru(a, b);
    }
    __device__ static __forceinline__ float div_pos_dn(float a, float b)
    {
        return fast_div_ok(a, b) ? __fmul_rd(__fdividef(a, b), 1.f - 4.76837158203125e-7f) : __fdiv_rd(a, b);
    }
    __device__ static __forceinline__ float abs(float a) { return fabsf(a); }
    __device__ static __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
    __device__ static __forceinline__ float min(float a, float b) { return fminf(a, b); }
    // exp with its error bound: CUDA documents expf as within 2 ulp over its
    // full range; 4 ulp (2^-21 relative) plus a subnormal floor is used here.
    __device__ static __forceinline__ float exp_dn(float x)
    {
        float e = expf(x);
        return fmaxf(0.f, __fsub_rd(__fmul_rd(e, 1.f - 4.76837158203125e-7f), 1e-44f));
    }
    __device__ static __forceinline__ float exp_up(float x)
    {
        float e = expf(x);
        return __fadd_ru(__fmul_ru(e, 1.f + 4.76837158203125e-7f), 1e-44f);
    }
};

template <> struct Num<double> {
    static constexpr double U = 1.1102230246251565e-16;  // 2^-53
    static constexpr double TINY = 1e-300;
    static constexpr double BIG = 1.0e300;
    __device__ static __forceinline__ double add_rd(double a, double b) { return __dadd_rd(a, b); }
    __device__ static __forceinline__ double add_ru(double a, double b) { return __dadd_ru(a, b); }
    __device__ static __forceinline__ double sub_rd(double a, double b) { return __dsub_rd(a, b); }
    __device__ static __forceinline__ double sub_ru(double a, double b) { return __dsub_ru(a, b); }
    __device__ static __forceinline__ double mul_rd(double a, double b) { return __dmul_rd(a, b); }
    __device__ static __forceinline__ double mul_ru(double a, double b) { return __dmul_ru(a, b); }
    __device__ static __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ double fma_rd(double a, double b, double c) { return __fma_rd(a, b, c); }
    __device__ static __forceinline__ double fma_ru(double a, double b, double c) { return __fma_ru(a, b, c); }
    __device__ static __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
    __device__ static __forceinline__ double div_rd(double a, double b) { return __ddiv_rd(a, b); }
    __device__ static __forceinline__ double div_ru(double a, double b) { return __ddiv_ru(a, b); }
    __device__ static __forceinline__ double sqrt_ru(double a) { return __dsqrt_ru(a); }
    __device__ static __forceinline__ double div_weight(double a, double b) { return a / b; }
    __device__ static __forceinline__ double div_pos_up(double a, double b) { return __ddiv_ru(a, b); }
    __device__ static __forceinline__ double div_pos_dn(double a, double b) { return __ddiv_rd(a, b); }
    __device__ static __forceinline__ double abs(double a) { return fabs(a); }
    __device__ static __forceinline__ double max(double a, double b) { return fmax(a, b); }
    __device__ static __forceinline__ double min(double a, double b) { return fmin(a, b); }
    // CUDA documents exp (double) as within 1 ulp; 4 ulp are allowed here.
    __device__ static __forceinline__ double exp_dn(double x)
    {
        double e = exp(x);
        return fmax(0.0, __dsub_rd(__dmul_rd(e, 1.0 - 8.881784197001252e-16), 1e-320));
    }
    __device__ static __forceinline__ double exp_up(double x)
    {
        double e = exp(x);
        return __dadd_ru(__dmul_ru(e, 1.0 + 8.881784197001252e-16), 1e-320);
    }
};

template <int M, class R> struct LF {
    R c[M];
    R k;
};

// c[j] = fma_rn(a, x[j], c[j]) for j < M.  For float, pairs of coefficients
// go through the packed FMA of sm_100 and later (__ffma2_rn: per element the
// same result as __fmaf_rn, two elements per instruction), which halves the
// issue slots of the coefficient updates without changing a bit.
template <int M, class R>
__device__ __forceinline__ void axpy_rn(R a, const R *x, R *c)
{
#pragma unroll
    for (int j = 0; j < M; ++j) c[j] = Num<R>::fma_rn(a, x[j], c[j]);
}
template <int M>
__device__ __forceinline__ void axpy_rn(float a, const float *x, float *c)
{
    const float2 aa = make_float2(a, a);
#pragma unroll
    for (int j = 0; j + 1 < M; j += 2) {
        const float2 r = __ffma2_rn(aa, make_float2(x[j], x[j + 1]), make_float2(c[j], c[j + 1]));
        c[j] = r.x;
        c[j + 1] = r.y;
    }
    if (M & 1) c[M - 1] = __fmaf_rn(a, x[M - 1], c[M - 1]);
}

// gamma_n = n u (1 + 2^-12), which covers (1 + u)^n - 1 for n < 2^10.  The
// product is exact (n (1 + 2^-12) has at most 24 significant bits for
// n < 2^11, and u is a power of two), so it is written in round-to-nearest:
// the value is the directed product's, and it folds to a constant where n is
// known at compile time.
template <class R>
__device__ __forceinline__ R gamma_n(int n)
{
    return (R)n * (Num<R>::U * (R)1.000244140625);
}
// 1 + gamma_n rounded up, exactly.  The numbers just above 1 are spaced 2u
// apart, and gamma_n / (2u) = n/2 + n 2^-13 lies strictly between floor(n/2)
// and floor(n/2) + 1 for 1 <= n < 2^12, so the rounded-up sum is
// 1 + (floor(n/2) + 1) 2u, a sum without rounding.
template <class R>
__device__ __forceinline__ R one_plus_gamma_ru(int n)
{
    return n > 0 ? (R)1 + (R)(n / 2 + 1) * ((R)2 * Num<R>::U) : (R)1;
}

// Accumulator of a sound form  sum_t a_t F_t + b  (one side).  DN = true for
// a lower form (constant rounded down, slack subtracted), false for upper.
// The coefficient updates of term / term_ck can be left out (cf = false)
// where only the constant and the radius of the result are used: they do not
// depend on the coefficients.
template <int M, class R, bool DN> struct Acc {
    LF<M, R> f;
    R rs;   // sum_t |a_t| r_t  (to be scaled by gamma_n)
    R ex;   // extra absolute slack
    int n;  // number of terms

    __device__ __forceinline__ void init(R b)
    {
#pragma unroll
        for (int j = 0; j < M; ++j) f.c[j] = 0;
        f.k = b; rs = 0; ex = 0; n = 0;
    }
    __device__ __forceinline__ void add_const(R b)
    {
        using N = Num<R>;
        f.k = DN ? N::add_rd(f.k, b) : N::add_ru(f.k, b);
    }
    __device__ __forceinline__ void add_slack(R s) { ex = Num<R>::add_ru(ex, s); }
    // add a * (Fc . p + Fk) where the form has radius r (the caller has
    // chosen the side of the form)
    __device__ __forceinline__ void term_ck(R a, const R *Fc, R Fk, R r, bool cf = true)
    {
        using N = Num<R>;
        if (cf) axpy_rn<M>(a, Fc, f.c);
        f.k = DN ? N::fma_rd(a, Fk, f.k) : N::fma_ru(a, Fk, f.k);
        rs = N::fma_ru(N::abs(a), r, rs);
        ++n;
    }
    // add a * F where F has radius r (the caller has chosen the side of F)
    __device__ __forceinline__ void term(R a, const LF<M, R> &F, R r, bool cf = true)
    {
        using N = Num<R>;
        if (cf) axpy_rn<M>(a, F.c, f.c);
        f.k = DN ? N::fma_rd(a, F.k, f.k) : N::fma_ru(a, F.k, f.k);
        rs = N::fma_ru(N::abs(a), r, rs);
        ++n;
    }
    // An upper bound on sum_j |c_j| of the result without summing it: each
    // coefficient is a chain of n rounded FMAs, so sum_j |c_j| <= (1 + gamma_n)
    // sum_t |a_t| r_t, plus a floor for subnormal rounding.  Tight where the
    // terms cannot cancel (one term).
    __device__ __forceinline__ R radius_bound() const
    {
        using N = Num<R>;
        return N::fma_ru(rs, one_plus_gamma_ru<R>(n), N::TINY);
    }
    __device__ __forceinline__ LF<M, R> result() const
    {
        using N = Num<R>;
        R s = N::add_ru(N::fma_ru(gamma_n<R>(n), rs, ex), N::TINY);
        LF<M, R> out = f;
        out.k = DN ? N::sub_rd(f.k, s) : N::add_ru(f.k, s);
        return out;
    }
};

// ---------------------------------------------------------------------------
// Bounded scalars with shared coefficients.  Every operation of the value
// chain gives the lower and the upper form the same coefficients: the pose
// forms differ only in their constants (Taylor remainder), the McCormick
// planes of a product share their slopes (y_m x + x_m y), the tangent and
// secant of a square share the slope x_lo + x_hi, and linear maps act on both
// alike.  So the pair is held as lo(p) = c.p + klo, hi(p) = c.p + khi with one
// coefficient vector, computed once; r = sum |c| (rounded up), and the
// concretisation is vlo = klo - r, vhi = khi + r.
template <int M, class R> struct SB {
    R c[M];
    R klo, khi;
    R r;
    R vlo, vhi;
};

template <int M, class R>
__device__ __forceinline__ void sb_finish(SB<M, R> &b)
{
    using N = Num<R>;
    R r = N::abs(b.c[0]);  // = RU(0 + |c_0|)
#pragma unroll
    for (int j = 1; j < M; ++j) r = N::add_ru(r, N::abs(b.c[j]));
    b.r = r;
    b.vlo = N::sub_rd(b.klo, r);
    b.vhi = N::add_ru(b.khi, r);
}

// midpoint of the concretisation, rounded to nearest: the slope a product
// takes for the other factor
template <int M, class R>
__device__ __forceinline__ R sb_mid(const SB<M, R> &b)
{
    return Num<R>::mul_rn(b.vlo + b.vhi, (R)0.5);
}

template <int M, class R>
__device__ __forceinline__ SB<M, R> sb_cst(R lo, R hi)
{
    SB<M, R> b;
#pragma unroll
    for (int j = 0; j < M; ++j) b.c[j] = 0;
    b.klo = lo; b.khi = hi; b.r = 0; b.vlo = lo; b.vhi = hi;
    return b;
}

// Accumulator of sum_t a_t X_t + b for both sides at once.  Coefficients are
// summed round-to-nearest; their worst-case error summed over the box,
// gamma_n sum_t |a_t| r_t, and any extra slack move into the constants, which
// are themselves rounded outward (see Acc).
template <int M, class R> struct SAcc {
    R c[M];
    R klo, khi;
    R rs;   // sum_t |a_t| r_t
    R ex;   // extra absolute slack
    int n;

    __device__ __forceinline__ void init(R blo, R bhi)
    {
#pragma unroll
        for (int j = 0; j < M; ++j) c[j] = 0;
        klo = blo; khi = bhi; rs = 0; ex = 0; n = 0;
    }
    __device__ __forceinline__ void add_const(R dlo, R dhi)
    {
        using N = Num<R>;
        klo = N::add_rd(klo, dlo);
        khi = N::add_ru(khi, dhi);
    }
    __device__ __forceinline__ void add_slack(R s) { ex = Num<R>::add_ru(ex, s); }
    // + a x, the side of x chosen by the sign of a
    __device__ __forceinline__ void term(R a, const SB<M, R> &x)
    {
        using N = Num<R>;
        axpy_rn<M>(a, x.c, c);
        if (a >= 0) {
            klo = N::fma_rd(a, x.klo, klo);
            khi = N::fma_ru(a, x.khi, khi);
        } else {
            klo = N::fma_rd(a, x.khi, klo);
            khi = N::fma_ru(a, x.klo, khi);
        }
        rs = N::fma_ru(N::abs(a), x.r, rs);
        ++n;
    }
    // + a x with x's lower form in the lower sum and its upper form in the
    // upper sum whatever the sign of a (only where an exact identity with
    // another term makes the pair sound, e.g. (u - mu) S + (mu S - P))
    __device__ __forceinline__ void term_same_side(R a, const SB<M, R> &x)
    {
        using N = Num<R>;
        axpy_rn<M>(a, x.c, c);
        klo = N::fma_rd(a, x.klo, klo);
        khi = N::fma_ru(a, x.khi, khi);
        rs = N::fma_ru(N::abs(a), x.r, rs);
        ++n;
    }
    // + x * y  (averaged McCormick planes)
    __device__ __forceinline__ void mul(const SB<M, R> &x, const SB<M, R> &y)
    {
        mul_ym(x, y, sb_mid(y));
    }
    // the same with y's midpoint given (a value of sb_mid(y) computed before)
    __device__ __forceinline__ void mul_ym(const SB<M, R> &x, const SB<M, R> &y, R ym)
    {
        using N = Num<R>;
        const R xl = x.vlo, xh = x.vhi, yl = y.vlo, yh = y.vhi;
        const R xm = sb_mid(x);
        term(ym, x);
        term(xm, y);
        // constants: -(xl yl + xh yh)/2 below, -(xh yl + xl yh)/2 above
        add_const(-N::mul_ru(N::fma_ru(xl, yl, N::mul_ru(xh, yh)), (R)0.5),
                  -N::mul_rd(N::fma_rd(xh, yl, N::mul_rd(xl, yh)), (R)0.5));
        // the slopes are the rounded midpoints: cover |ym - y_mid| max|x| + ...
        const R xa = N::max(N::abs(xl), N::abs(xh)), ya = N::max(N::abs(yl), N::abs(yh));
        add_slack(N::mul_ru(N::fma_ru(N::abs(ym), xa, N::mul_ru(N::abs(xm), ya)), N::U * (R)1.001));  // (an exact product)
    }
    // + x^2  (tangent at the midpoint c below, secant above; both have slope
    // x_lo + x_hi = 2c)
    __device__ __forceinline__ void sqr(const SB<M, R> &x)
    {
        using N = Num<R>;
        const R xl = x.vlo, xh = x.vhi;
        const R s = xl + xh;
        const R c = N::mul_rn(s, (R)0.5);
        term(s, x);
        add_const(-N::mul_ru(c, c), N::max(N::fma_ru(xl, xl, N::mul_ru(-s, xl)), N::fma_ru(xh, xh, N::mul_ru(-s, xh))));
    }
    __device__ __forceinline__ SB<M, R> result() const
    {
        using N = Num<R>;
        const R sl = N::add_ru(N::fma_ru(gamma_n<R>(n), rs, ex), N::TINY);
        SB<M, R> b;
#pragma unroll
        for (int j = 0; j < M; ++j) b.c[j] = c[j];
        b.klo = N::sub_rd(klo, sl);
        b.khi = N::add_ru(khi, sl);
        sb_finish(b);
        return b;
    }
};

template <int M, class R>
__device__ __forceinline__ SB<M, R> sb_mul(const SB<M, R> &x, const SB<M, R> &y)
{
    SAcc<M, R> p; p.init(0, 0); p.mul(x, y); return p.result();
}
template <int M, class R>
__device__ __forceinline__ SB<M, R> sb_sqr(const SB<M, R> &x)
{
    SAcc<M, R> p; p.init(0, 0); p.sqr(x); return p.result();
}
template <int M, class R>
__device__ __forceinline__ SB<M, R> sb_add(const SB<M, R> &x, const SB<M, R> &y)
{
    SAcc<M, R> p; p.init(0, 0); p.term((R)1, x); p.term((R)1, y); return p.result();
}

}  // namespace ar
