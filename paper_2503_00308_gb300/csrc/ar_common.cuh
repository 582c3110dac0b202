// ar_common.cuh -- data layout shared by the abstract-rendering kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ar_num.cuh"

namespace ar {

// Algorithm constants (the relaxation choices of the abstract renderer).
constexpr int KTAYLOR = 8;                       // MatrixInv order, k = 8 (Sec. 3.3 footnote)
constexpr int KMAX = 24;                         // adaptive order: k grows from KTAYLOR up to KMAX (Sec. 3.1 (3))
constexpr double EPS_TOL = 5.9604644775390625e-8;  // 2^-24: k grows until Eps <= EPS_TOL ||X0||_F
constexpr int SPLIT_DEPTH = 6;                   // input splitting: at most 6 bisections of a cell (Sec. 3.1 (2))
constexpr double RHO_MAX = 1.0 - 1.0 / 1024.0;   // MatrixInv used while ||I - X X0|| < RHO_MAX
constexpr float CUT_RAMP = 0.5f;                 // widest cutoff ramp (units of m)
constexpr float CLIP_RAMP = 0.25f;               // upper-alpha blend toward o
constexpr double KEY_SLACK = 1e-9;               // relative widening of depth keys
constexpr double BOX_SLACK = 1e-9;               // relative widening of screen boxes
constexpr double GUARD = 0.65;                   // frustum guard band: 1.3 x the half-extent (fraction of W, H)
constexpr float ALPHA_MIN_UP = 0.003921568859368563f;  // 1/255 rounded up to float

constexpr int MAXV = 6;  // pose variables tx ty tz rx ry rz

// Per-call pose-cell data produced by the cell kernel.
//   FP64 part (decision chain): forms over the M active variables, computed
//   round-to-nearest in the order the CPU reference uses.
//   FP64 value-chain copies: the same forms widened to be sound in FP64.
template <int M> struct CellData {
    double rd_lo[9][M + 1], rd_hi[9][M + 1];  // R_delta entries (coefficients, then constant)
    double s[3][M + 1];                       // s = R_wc * delta_t (exact)
    double g[M];                              // depth-key offset (translation part of d)
    double rd_int[9][2];                      // concretised R_delta entries
    double s_int[3][2];                       // concretised s
    // FP32 enclosures of FP64 constants of the screen-box filter
    float rd_int32[9][2][2];                  // of rd_int[e][end]: [lo, hi]
    float s_int32[3][2][2];                   // of s_int[a][end]
    float guard32[4][2];                      // of cx + gx, cx - gx, cy + gy, cy - gy
    float slack32[2];                         // of BOX_SLACK
    // per-cell parts of the depth chain d = sum_b R_delta[b][2] (v_b - s_b):
    // the interval [lo, hi] of each R_delta[b][2] and its midpoint, the
    // translation-slot coefficients of d and of the depth-key form, and the
    // slot ranges (translation slots [0, n_t), rotation slots [n_t, n_a))
    double dx[3][3];
    double dd_t[M], kd_t[M];
    int n_t, n_a;
    // FP32 enclosures ([lo, hi]) of the depth chain's per-cell values, for
    // the early certain drops of the decision part
    float dx32[3][3][2];       // of dx[b][k]
    float s32[3][M + 1][2];    // of s[b][j]
    float rdd32[3][2][M + 1][2];  // of rd_lo[3 b + 2][j] (0) and rd_hi[3 b + 2][j] (1)
    float ddt32[M][2];         // of dd_t[j]
    SB<M, double> rd64[9];  // the same forms widened by a relative 1e-14 (sound in FP64)
    SB<M, double> s64[3];
};

// Per-(Gaussian, cell) record read by the per-pixel kernel, in elements of
// the record precision (float for the batched renderer, double for the plain
// one).  A bounded scalar with shared coefficients is stored as c[M], -klo,
// khi, r (SB), the W entries also with their concretisation -vlo, vhi and the
// midpoint of [vlo, vhi].  The lower ends are stored negated: the FP32 pixel
// stage holds each (lower, upper) pair as (-lo, hi) and updates both ends in
// one packed operation rounded up.
//
// Delta = S u - P (Algorithm 1 line 9 with S = d^2, P = d up) is stored as
//   Delta.lo = (u - mu) S.lo + R.lo,  R.lo = mu S.lo - P.hi,
//   Delta.hi = (u - mu) S.hi + R.hi,  R.hi = mu S.hi - P.lo,
// with mu a pixel centre near the projected mean: algebraically the same
// forms as u S.lo - P.hi and u S.hi - P.lo (sound because u > 0), but the
// large, nearly cancelling terms S u and P are combined once in FP64 instead
// of per pixel.  GAP_S bounds, over the cell, how far the stored S forms lie
// outside the FP64 ones R was formed from (their outward conversion); where
// u - mu < 0 the pixel stage widens Delta by |u - mu| GAP_S.
// Every entry starts on a multiple of 4 elements, so that the pixel stage reads
// it with 16-byte vector loads.
template <int M> struct Rec {
    static constexpr int SBW = (M + 3 + 3) / 4 * 4;  // c[M], -klo, khi, r (padded)
    static constexpr int S = 0, RX = SBW, RY = 2 * SBW;
    static constexpr int WS = (M + 5 + 3) / 4 * 4;   // c[M], -klo, khi, -vlo, vhi, r, mid (padded)
    static constexpr int W0 = 3 * SBW;               // W_rc at W0 + (3 r + c) WS
    // scalars: o_hi, tau_dn, tau_up, c_lo[3], flags, mu_x, mu_y, gap_s, o_lo, c_hi[3]
    // (the opacity and colour boxes of the scene parameters; lo = hi without boxes)
    static constexpr int SC = W0 + 6 * WS;
    static constexpr int O = SC, TAU_DN = SC + 1, TAU_UP = SC + 2, COL = SC + 3, FLAGS = SC + 6;
    static constexpr int MU_X = SC + 7, MU_Y = SC + 8, GAP_S = SC + 9, O_LO = SC + 10, COL_HI = SC + 11;
    static constexpr int SCW = 16;
    static constexpr int WIDTH = SC + SCW;            // a multiple of 4 elements
};

// record flags
constexpr uint32_t F_FALLBACK = 1u;  // MatrixInv failed, even on split pieces: a in [0, o]
constexpr uint32_t F_STRADDLE = 2u;  // depth may cross the near plane: lower alpha is 0
constexpr uint32_t F_OPEN = 4u;      // depth-key interval has positive width
constexpr uint32_t F_SPLIT = 8u;     // MatrixInv held only after splitting the cell (constant Conic)
constexpr uint32_t F_SPLIT_PENDING = 16u;  // returned by a deferred record build, never stored
constexpr uint32_t F_KHIGH_PENDING = 32u;  // likewise, for a Taylor order above the default

// doubles per Gaussian of the per-call array vN: v = R_wc (uw - t) as an
// interval over the mean's box (lower ends 3, upper ends 3), then N = R_wc Mw
// (9), then, in the storage of VN_ENC_DOUBLES doubles, 30 floats: the FP32
// enclosures (lo, hi) of those 15 values, for the screen-box filter
constexpr int VN_ENC = 15, VN_ENC_DOUBLES = 15;
constexpr int VN_STRIDE = VN_ENC + VN_ENC_DOUBLES;

// Per-Gaussian scene parameters of the abstract render as boxes (Sec. 4.5):
// opacity o in [o_lo, o_hi], the cutoff exponent tau = 2 ln(255 o) at both
// ends (-inf below 1/255), and each colour channel in [c_lo, c_hi]; lo = hi
// without boxes.  (The mean's box enters through v; see pose_prep_kernel.)
struct GParam {
    double tau_lo, tau_hi;
    float o_lo, o_hi;
    float c_lo[3], c_hi[3];
};

// Pixel box of a (Gaussian, cell) pair: x0 < 0 marks "contributes nowhere".
struct PixBox {
    int x0, x1, y0, y1;
};

// ---------------------------------------------------------------------------
// Plain FP64 forms for the decision chain (round-to-nearest, no contraction).
template <int M> struct DF {
    double c[M];
    double k;
};

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

template <int M> __device__ __forceinline__ double df_min(const DF<M> &f)
{
    double s = f.k;
#pragma unroll
    for (int j = 0; j < M; ++j) s = dsub(s, fabs(f.c[j]));
    return s;
}
template <int M> __device__ __forceinline__ double df_max(const DF<M> &f)
{
    double s = f.k;
#pragma unroll
    for (int j = 0; j < M; ++j) s = dadd(s, fabs(f.c[j]));
    return s;
}
// intervals for the screen box
struct DI {
    double l, u;
};
__device__ __forceinline__ DI di_mul(DI a, DI b)
{
    double p0 = dmul(a.l, b.l), p1 = dmul(a.l, b.u), p2 = dmul(a.u, b.l), p3 = dmul(a.u, b.u);
    DI r = {p0, p0};
    r.l = fmin(r.l, p1); r.u = fmax(r.u, p1);
    r.l = fmin(r.l, p2); r.u = fmax(r.u, p2);
    r.l = fmin(r.l, p3); r.u = fmax(r.u, p3);
    return r;
}
// di_mul for a > 0 (a.l > 0): the extreme products are picked by the sign of
// b's ends, so the result is the same pair of IEEE products di_mul selects
__device__ __forceinline__ DI di_mul_pos(DI a, DI b)
{
    return DI{b.l >= 0 ? dmul(a.l, b.l) : dmul(a.u, b.l), b.u >= 0 ? dmul(a.u, b.u) : dmul(a.l, b.u)};
}
__device__ __forceinline__ DI di_add(DI a, DI b) { return DI{dadd(a.l, b.l), dadd(a.u, b.u)}; }
__device__ __forceinline__ DI di_scale(DI a, double s)
{
    return s >= 0 ? DI{dmul(s, a.l), dmul(s, a.u)} : DI{dmul(s, a.u), dmul(s, a.l)};
}
__device__ __forceinline__ double di_sqmax(DI a) { return fmax(dmul(a.l, a.l), dmul(a.u, a.u)); }

// ---------------------------------------------------------------------------
// FP32 enclosures of FP64 values, to take FP64 decisions at FP32 cost.  An
// E32 holds floats lo <= hi with lo <= x <= hi for the double x that an FP64
// expression (rounded to nearest at every step) computes.  Each operation
// maps enclosures of its FP64 operands to an enclosure of its FP64 result:
// its directed FP32 results bracket the exact result of the operation for
// every operand value in the enclosures, and as floats are doubles, rounding
// that exact result to the nearest double stays between them (rounding is
// monotone and leaves representable values fixed).  e_chk clears ok for a
// value beyond 1e30 in magnitude, an infinity or a NaN, so that no NaN or
// infinity can enter a later operation unnoticed; the caller then decides in
// FP64.
struct E32 {
    float lo, hi;
};
struct EI {  // enclosures of both ends of an FP64 interval (a DI)
    E32 l, u;
};
__device__ __forceinline__ E32 e_chk(E32 x, bool &ok)
{
    ok = ok && fabsf(x.lo) <= 1e30f && fabsf(x.hi) <= 1e30f;
    return x;
}
__device__ __forceinline__ E32 e_of(double x) { return E32{__double2float_rd(x), __double2float_ru(x)}; }
__device__ __forceinline__ E32 e_add(E32 a, E32 b) { return E32{__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi)}; }
__device__ __forceinline__ E32 e_sub(E32 a, E32 b) { return E32{__fsub_rd(a.lo, b.hi), __fsub_ru(a.hi, b.lo)}; }
__device__ __forceinline__ E32 e_neg(E32 a) { return E32{-a.hi, -a.lo}; }
__device__ __forceinline__ E32 e_min(E32 a, E32 b) { return E32{fminf(a.lo, b.lo), fminf(a.hi, b.hi)}; }
__device__ __forceinline__ E32 e_max(E32 a, E32 b) { return E32{fmaxf(a.lo, b.lo), fmaxf(a.hi, b.hi)}; }
__device__ __forceinline__ E32 e_hull(E32 a, E32 b) { return E32{fminf(a.lo, b.lo), fmaxf(a.hi, b.hi)}; }
__device__ __forceinline__ E32 e_mul(E32 a, E32 b)
{
    const float l = fminf(fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
                          fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)));
    const float h = fmaxf(fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi)),
                          fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi)));
    return E32{l, h};
}
// a / d for d > 0 (d.lo > 0)
__device__ __forceinline__ E32 e_div_pos(E32 a, E32 d)
{
    return E32{fminf(__fdiv_rd(a.lo, d.lo), __fdiv_rd(a.lo, d.hi)), fmaxf(__fdiv_ru(a.hi, d.lo), __fdiv_ru(a.hi, d.hi))};
}
// sqrt of an FP64 value x >= 0
__device__ __forceinline__ E32 e_sqrt(E32 a) { return E32{__fsqrt_rd(fmaxf(a.lo, 0.f)), __fsqrt_ru(a.hi)}; }
__device__ __forceinline__ E32 e_abs(E32 a)
{
    if (a.lo >= 0.f) return a;
    if (a.hi <= 0.f) return e_neg(a);
    return E32{0.f, fmaxf(-a.lo, a.hi)};
}
// a > b: 1 certainly, 0 certainly not, -1 not settled by the enclosures
__device__ __forceinline__ int e_gt(E32 a, E32 b) { return a.lo > b.hi ? 1 : (a.hi <= b.lo ? 0 : -1); }
// a >= b, likewise
__device__ __forceinline__ int e_ge(E32 a, E32 b) { return a.lo >= b.hi ? 1 : (a.hi < b.lo ? 0 : -1); }
// the interval operations of the screen box (di_*), on enclosures
__device__ __forceinline__ EI ei_add(EI a, EI b, bool &ok)
{
    return EI{e_chk(e_add(a.l, b.l), ok), e_chk(e_add(a.u, b.u), ok)};
}
__device__ __forceinline__ EI ei_mul(EI a, EI b, bool &ok)
{
    const E32 p0 = e_mul(a.l, b.l), p1 = e_mul(a.l, b.u), p2 = e_mul(a.u, b.l), p3 = e_mul(a.u, b.u);
    return EI{e_chk(e_min(e_min(p0, p1), e_min(p2, p3)), ok), e_chk(e_max(e_max(p0, p1), e_max(p2, p3)), ok)};
}
// di_mul_pos: the product is picked by the sign of b's ends; where that sign
// is not settled, the hull of both candidates
__device__ __forceinline__ EI ei_mul_pos(EI a, EI b, bool &ok)
{
    const E32 l1 = e_mul(a.l, b.l), l2 = e_mul(a.u, b.l);
    const E32 u1 = e_mul(a.u, b.u), u2 = e_mul(a.l, b.u);
    const E32 l = b.l.lo >= 0.f ? l1 : (b.l.hi < 0.f ? l2 : e_hull(l1, l2));
    const E32 u = b.u.lo >= 0.f ? u1 : (b.u.hi < 0.f ? u2 : e_hull(u1, u2));
    return EI{e_chk(l, ok), e_chk(u, ok)};
}
// di_scale by a double s given by its enclosure se (se = e_of(s)): s >= 0
// exactly when se.lo >= 0 (rounding down keeps the sign, and -0 stays -0)
__device__ __forceinline__ EI ei_scale(EI a, E32 se, bool &ok)
{
    return se.lo >= 0.f ? EI{e_chk(e_mul(se, a.l), ok), e_chk(e_mul(se, a.u), ok)}
                        : EI{e_chk(e_mul(se, a.u), ok), e_chk(e_mul(se, a.l), ok)};
}
// di_scale by -1 (exact)
__device__ __forceinline__ EI ei_neg(EI a) { return EI{e_neg(a.u), e_neg(a.l)}; }
__device__ __forceinline__ E32 ei_sqmax(EI a) { return e_max(e_mul(a.l, a.l), e_mul(a.u, a.u)); }

// order-preserving map of a double to uint64 (-0 folded onto +0)
__device__ __forceinline__ uint64_t key_bits(double x)
{
    if (x == 0.0) x = 0.0;
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Camera / call constants passed by value to the kernels.
struct CallConst {
    int W, H;
    float fx, fy, cx, cy, near_plane;
    double R0[9];
    double t0[3];
    int n_cells;
    int64_t n_gauss;
    int m_slot[MAXV];  // slot of each pose variable in the forms, -1 if inactive
};

}  // namespace ar
