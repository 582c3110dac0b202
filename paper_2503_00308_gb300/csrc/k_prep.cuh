// k_prep.cuh -- scene preprocessing, pose-cell linearisation and the
// per-(Gaussian, cell) records of the abstract renderer.
//
//   scene_prep    : Mw = R(q) diag(exp(s)) and tau = 2 ln(255 o) per Gaussian
//                   (the Gaussian tuple <uw, Mw, o, c> of Sec. 2.2).
//   pose_prep     : v = R_wc (uw - t) and N = R_wc Mw per Gaussian for the
//                   nominal camera of the call.
//   cell_prep<M>  : linear forms of R_delta(theta) (first-order Taylor at the
//                   cell centre, remainder (1/2)(sum h_theta)^2) and of
//                   s = R_wc delta_t, per cell.
//   record_prep<M>: Algorithm 1 lines 2-8 with set-valued variables (Sec. 3.3)
//                   for one (Gaussian, cell) pair: uc, d, up, J, Mc, Mp,
//                   X = Mp Mp^T, S = d^2, P = d up, MatrixInv (Algorithm 3,
//                   k = 8, X0 = inverse of the centre matrix) and W = Conic Mp.
//                   The depth key, near-plane class and pixel box are decided
//                   in FP64; the forms that feed the per-pixel stage are FP32
//                   with outward rounding.
#pragma once
#include "ar_common.cuh"

namespace ar {

// ---------------------------------------------------------------- scene prep
__device__ __forceinline__ void quat_rot(const float *q_in, double R[9])
{
    double q0 = q_in[0], q1 = q_in[1], q2 = q_in[2], q3 = q_in[3];
    double n = sqrt(dadd(dadd(dadd(dmul(q0, q0), dmul(q1, q1)), dmul(q2, q2)), dmul(q3, q3)));
    double w = q0 / n, x = q1 / n, y = q2 / n, z = q3 / n;
    R[0] = dsub(1.0, dmul(2.0, dadd(dmul(y, y), dmul(z, z))));
    R[1] = dmul(2.0, dsub(dmul(x, y), dmul(w, z)));
    R[2] = dmul(2.0, dadd(dmul(x, z), dmul(w, y)));
    R[3] = dmul(2.0, dadd(dmul(x, y), dmul(w, z)));
    R[4] = dsub(1.0, dmul(2.0, dadd(dmul(x, x), dmul(z, z))));
    R[5] = dmul(2.0, dsub(dmul(y, z), dmul(w, x)));
    R[6] = dmul(2.0, dsub(dmul(x, z), dmul(w, y)));
    R[7] = dmul(2.0, dadd(dmul(y, z), dmul(w, x)));
    R[8] = dsub(1.0, dmul(2.0, dadd(dmul(x, x), dmul(y, y))));
}

__device__ __forceinline__ void mat3(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s = dadd(s, dmul(A[3 * i + k], B[3 * k + j]));
            C[3 * i + j] = s;
        }
}

// ----------------------------------------------------------------- cells
__device__ __forceinline__ void rot3(int axis, double a, double R[9], double D[9])
{
    double c = cos(a), s = sin(a);
    for (int e = 0; e < 9; ++e) { R[e] = 0; D[e] = 0; }
    if (axis == 0) {
        R[0] = 1; R[4] = c; R[5] = -s; R[7] = s; R[8] = c;
        D[4] = -s; D[5] = -c; D[7] = c; D[8] = -s;
    } else if (axis == 1) {
        R[0] = c; R[2] = s; R[4] = 1; R[6] = -s; R[8] = c;
        D[0] = -s; D[2] = c; D[6] = -c; D[8] = -s;
    } else {
        R[0] = c; R[1] = -s; R[3] = s; R[4] = c; R[8] = 1;
        D[0] = -s; D[1] = -c; D[3] = c; D[4] = -s;
    }
}

// One thread per cell.
template <int M>
__global__ void cell_prep_kernel(const double *__restrict__ cells_lo, const double *__restrict__ cells_hi,
                                 CallConst cc, CellData<M> *__restrict__ out)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cc.n_cells) return;
    CellData<M> &cd = out[c];
    double ctr[MAXV], h[MAXV];
    for (int k = 0; k < MAXV; ++k) {
        double lo = cells_lo[MAXV * c + k], hi = cells_hi[MAXV * c + k];
        ctr[k] = dmul(0.5, dadd(lo, hi));
        h[k] = dmul(0.5, dsub(hi, lo));
    }
    // R_delta = Rx Ry Rz at the centre and its partial derivatives
    double X[9], dX[9], Y[9], dY[9], Z[9], dZ[9], T[9], R[9], dR[3][9];
    rot3(0, ctr[3], X, dX);
    rot3(1, ctr[4], Y, dY);
    rot3(2, ctr[5], Z, dZ);
    mat3(X, Y, T); mat3(T, Z, R);
    mat3(dX, Y, T); mat3(T, Z, dR[0]);
    mat3(X, dY, T); mat3(T, Z, dR[1]);
    mat3(X, Y, T); mat3(T, dZ, dR[2]);
    double hs = dadd(dadd(h[3], h[4]), h[5]);
    double rem = dmul(0.5, dmul(hs, hs));
    for (int e = 0; e < 9; ++e) {
        for (int j = 0; j <= M; ++j) { cd.rd_lo[e][j] = 0; cd.rd_hi[e][j] = 0; }
        for (int k = 0; k < 3; ++k) {
            int sl = cc.m_slot[3 + k];
            if (sl >= 0) { double v = dmul(dR[k][e], h[3 + k]); cd.rd_lo[e][sl] = v; cd.rd_hi[e][sl] = v; }
        }
        cd.rd_lo[e][M] = dsub(R[e], rem);
        cd.rd_hi[e][M] = dadd(R[e], rem);
    }
    for (int a = 0; a < 3; ++a) {
        for (int j = 0; j <= M; ++j) cd.s[a][j] = 0;
        double kk = 0;
        for (int k = 0; k < 3; ++k) {
            int sl = cc.m_slot[k];
            if (sl >= 0) cd.s[a][sl] = dmul(cc.R0[3 * a + k], h[k]);
            kk = dadd(kk, dmul(cc.R0[3 * a + k], ctr[k]));
        }
        cd.s[a][M] = kk;
    }
    for (int j = 0; j < M; ++j) cd.g[j] = 0;
    for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int b = 0; b < 3; ++b) s = dadd(s, dmul(R[3 * b + 2], cc.R0[3 * b + k]));
        int sl = cc.m_slot[k];
        if (sl >= 0) cd.g[sl] = dmul(-s, h[k]);
    }
    for (int e = 0; e < 9; ++e) {
        DF<M> lo, hi;
        for (int j = 0; j < M; ++j) { lo.c[j] = cd.rd_lo[e][j]; hi.c[j] = cd.rd_hi[e][j]; }
        lo.k = cd.rd_lo[e][M]; hi.k = cd.rd_hi[e][M];
        cd.rd_int[e][0] = df_min(lo);
        cd.rd_int[e][1] = df_max(hi);
    }
    for (int a = 0; a < 3; ++a) {
        DF<M> f;
        for (int j = 0; j < M; ++j) f.c[j] = cd.s[a][j];
        f.k = cd.s[a][M];
        cd.s_int[a][0] = df_min(f);
        cd.s_int[a][1] = df_max(f);
    }
    for (int e = 0; e < 9; ++e)
        for (int t = 0; t < 2; ++t) {
            cd.rd_int32[e][t][0] = __double2float_rd(cd.rd_int[e][t]);
            cd.rd_int32[e][t][1] = __double2float_ru(cd.rd_int[e][t]);
        }
    for (int a = 0; a < 3; ++a)
        for (int t = 0; t < 2; ++t) {
            cd.s_int32[a][t][0] = __double2float_rd(cd.s_int[a][t]);
            cd.s_int32[a][t][1] = __double2float_ru(cd.s_int[a][t]);
        }
    {
        const double gx = dmul(GUARD, (double)cc.W), gy = dmul(GUARD, (double)cc.H);
        const double gc[4] = {dadd((double)cc.cx, gx), dsub((double)cc.cx, gx), dadd((double)cc.cy, gy),
                              dsub((double)cc.cy, gy)};
        for (int i = 0; i < 4; ++i) {
            cd.guard32[i][0] = __double2float_rd(gc[i]);
            cd.guard32[i][1] = __double2float_ru(gc[i]);
        }
        cd.slack32[0] = __double2float_rd(BOX_SLACK);
        cd.slack32[1] = __double2float_ru(BOX_SLACK);
    }
    // per-cell parts of the depth chain (see record_decide): R_delta[b][2]
    // has coefficients on the rotation slots only and s_b on the translation
    // slots only, so the products xm * (-s_b) and their sums over b are the
    // same for every Gaussian of the cell
    {
        int nt = 0, na = 0;
        for (int k = 0; k < MAXV; ++k) {
            if (cc.m_slot[k] < 0) continue;
            ++na;
            if (k < 3) ++nt;
        }
        cd.n_t = nt;
        cd.n_a = na;
        for (int j = 0; j < M; ++j) cd.dd_t[j] = 0.0;
        for (int b = 0; b < 3; ++b) {
            const int e = 3 * b + 2;
            DF<M> lo, hi;
            for (int j = 0; j < M; ++j) { lo.c[j] = cd.rd_lo[e][j]; hi.c[j] = cd.rd_hi[e][j]; }
            lo.k = cd.rd_lo[e][M]; hi.k = cd.rd_hi[e][M];
            const double xl = df_min(lo), xh = df_max(hi);
            const double xm = dmul(0.5, dadd(xl, xh));
            cd.dx[b][0] = xl; cd.dx[b][1] = xh; cd.dx[b][2] = xm;
            for (int j = 0; j < nt; ++j) {
                const double t = dmul(xm, dsub(0.0, cd.s[b][j]));
                cd.dd_t[j] = b == 0 ? t : dadd(cd.dd_t[j], t);
            }
        }
        for (int j = 0; j < M; ++j) cd.kd_t[j] = dsub(cd.dd_t[j], cd.g[j]);
        auto enc = [](double x, float *o) {
            o[0] = __double2float_rd(x);
            o[1] = __double2float_ru(x);
        };
        for (int b = 0; b < 3; ++b) {
            for (int k = 0; k < 3; ++k) enc(cd.dx[b][k], cd.dx32[b][k]);
            for (int j = 0; j <= M; ++j) {
                enc(cd.s[b][j], cd.s32[b][j]);
                enc(cd.rd_lo[3 * b + 2][j], cd.rdd32[b][0][j]);
                enc(cd.rd_hi[3 * b + 2][j], cd.rdd32[b][1][j]);
            }
        }
        for (int j = 0; j < M; ++j) enc(cd.dd_t[j], cd.ddt32[j]);
    }
    // FP64 value-chain copies, widened to cover the rounding of sin, cos and
    // the Taylor terms (a relative 1e-14 is far above their few-ulp error);
    // the lower and upper forms share their coefficients
    for (int e = 0; e < 12; ++e) {
        const double *lo = e < 9 ? cd.rd_lo[e] : cd.s[e - 9];
        const double *hi = e < 9 ? cd.rd_hi[e] : cd.s[e - 9];
        SB<M, double> &b = e < 9 ? cd.rd64[e] : cd.s64[e - 9];
        double mag = 1.0;
        for (int j = 0; j <= M; ++j) mag = __dadd_ru(mag, fmax(fabs(lo[j]), fabs(hi[j])));
        const double pad = __dmul_ru(1e-14, mag);
        for (int j = 0; j < M; ++j) b.c[j] = lo[j];
        b.klo = __dsub_rd(lo[M], pad);
        b.khi = __dadd_ru(hi[M], pad);
        sb_finish(b);
    }
}

// FP32 form -> FP64 (exact); an FP64 form passes through
template <int M>
__device__ __forceinline__ const SB<M, double> &to_f64(const SB<M, double> &b) { return b; }
template <int M>
__device__ __forceinline__ SB<M, double> to_f64(const SB<M, float> &b)
{
    SB<M, double> d;
    for (int j = 0; j < M; ++j) d.c[j] = b.c[j];
    d.klo = b.klo;
    d.khi = b.khi;
    sb_finish(d);
    return d;
}

// FP64 sound form -> outward FP32 form: coefficients rounded to nearest,
// their error over the box moved into the outward-rounded constants.  Returns
// a bound, over the box, of how far either FP32 form lies outside the FP64
// one (the conversion gap).
template <int M>
__device__ __forceinline__ double sb_to_f32(const SB<M, double> &d, SB<M, float> &b)
{
    double e = 0;
    for (int j = 0; j < M; ++j) {
        b.c[j] = (float)d.c[j];
        e = __dadd_ru(e, fabs(d.c[j] - (double)b.c[j]));
    }
    b.klo = __double2float_rd(__dsub_rd(d.klo, e));
    b.khi = __double2float_ru(__dadd_ru(d.khi, e));
    sb_finish(b);
    return __dadd_ru(e, fmax(__dsub_ru(d.klo, (double)b.klo), __dsub_ru((double)b.khi, d.khi)));
}
// FP64 sound form -> record precision (FP32 outward, or FP64 as it is)
template <int M>
__device__ __forceinline__ double sb_to_rec(const SB<M, double> &d, SB<M, float> &b) { return sb_to_f32<M>(d, b); }
template <int M>
__device__ __forceinline__ double sb_to_rec(const SB<M, double> &d, SB<M, double> &b)
{
    b = d;
    return 0.0;
}

// scalars in the record precision, rounded down / up
__device__ __forceinline__ void rec_dn(double x, float &y) { y = __double2float_rd(x); }
__device__ __forceinline__ void rec_dn(double x, double &y) { y = x; }
__device__ __forceinline__ void rec_up(double x, float &y) { y = __double2float_ru(x); }
__device__ __forceinline__ void rec_up(double x, double &y) { y = x; }
// the flags word: a float's bit pattern, or a double's value
__device__ __forceinline__ void rec_put_flags(float *dst, uint32_t f) { *dst = __uint_as_float(f); }
__device__ __forceinline__ void rec_put_flags(double *dst, uint32_t f) { *dst = (double)f; }

// ------------------------------------------------------------- records
// c[M], -klo, khi, r (the S and R entries of a record; the lower end negated)
template <int M, class R>
__device__ __forceinline__ void store_sb(R *dst, const SB<M, R> &b)
{
#pragma unroll
    for (int j = 0; j < M; ++j) dst[j] = b.c[j];
    dst[M] = -b.klo;
    dst[M + 1] = b.khi;
    dst[M + 2] = b.r;
}
// c[M], -klo, khi, -vlo, vhi, r, mid (the W entries, the lower ends negated;
// mid = sb_mid(b), the slope the pixel stage's product Delta W takes for
// Delta, kept in the padding)
template <int M, class R>
__device__ __forceinline__ void store_sbw(R *dst, const SB<M, R> &b)
{
    static_assert(M + 5 < Rec<M>::WS, "the W entry has no room for its midpoint");
#pragma unroll
    for (int j = 0; j < M; ++j) dst[j] = b.c[j];
    dst[M] = -b.klo;
    dst[M + 1] = b.khi;
    dst[M + 2] = -b.vlo;
    dst[M + 3] = b.vhi;
    dst[M + 4] = b.r;
    dst[M + 5] = sb_mid(b);
}

template <int M, class R>
__device__ __forceinline__ bool sb_finite(const SB<M, R> &b)
{
    return isfinite(b.vlo) && isfinite(b.vhi) && isfinite(b.klo) && isfinite(b.khi) && isfinite(b.r);
}

struct PrepCount {
    uint32_t triples, fallback, valid, tiles, split;
};

// ---- screen box (Algorithm 1 lines 3-5 on intervals): the pixel box of the
// centres that can lie in the ellipse m <= tau at some pose of the cell with
// d > near, the projected-mean pixel centre mu_px (the expansion point of the
// pixel stage) and the frustum guard band.  Inputs: the concretised R_delta
// entries Ri and s, the Gaussian's v and N, its depth interval [dlo, dhi] and
// tau.  Returns SCREEN_DROP when the pair reaches no pixel, SCREEN_KEEP with
// box and mu_px set (and straddle set where the guard band is crossed).
enum { SCREEN_DROP = 0, SCREEN_KEEP = 1, SCREEN_UNDECIDED = 2 };

// The definition, in FP64 with round-to-nearest steps in a fixed order.
static __device__ __noinline__ int screen_fp64(const double (*rd_int)[2], const double (*s_int)[2], const double *vl,
                                               const double *vh, const double *N, double dlo, double dhi, double tau,
                                               const CallConst &cc, PixBox &box, double *mu_px, bool &straddle)
{
    const double nearp = (double)cc.near_plane;
    DI Ri[9], vs[3];
    for (int e = 0; e < 9; ++e) Ri[e] = DI{rd_int[e][0], rd_int[e][1]};
    for (int b = 0; b < 3; ++b) vs[b] = DI{dsub(vl[b], s_int[b][1]), dsub(vh[b], s_int[b][0])};
    const double dl = fmax(dlo, nearp);
    DI D = {dl, dhi};
    DI ucx = di_add(di_add(di_mul(Ri[0], vs[0]), di_mul(Ri[3], vs[1])), di_mul(Ri[6], vs[2]));
    DI ucy = di_add(di_add(di_mul(Ri[1], vs[0]), di_mul(Ri[4], vs[1])), di_mul(Ri[7], vs[2]));
    const double fx = cc.fx, fy = cc.fy, cx = cc.cx, cy = cc.cy;
    // D > 0, so min(u / D_lo, u / D_hi) is u / D_hi for u >= 0 and u / D_lo
    // below (the same rounded quotient: division is monotone in D)
    DI mux = {dadd(cx, dmul(fx, ucx.l / (ucx.l >= 0 ? D.u : D.l))), dadd(cx, dmul(fx, ucx.u / (ucx.u >= 0 ? D.l : D.u)))};
    DI muy = {dadd(cy, dmul(fy, ucy.l / (ucy.l >= 0 ? D.u : D.l))), dadd(cy, dmul(fy, ucy.u / (ucy.u >= 0 ? D.l : D.u)))};
    // frustum guard band (3DGS convention): a mean outside it at every pose
    // of the cell drops the pair; outside it at some pose makes the lower
    // alpha 0
    {
        const double gx = dmul(GUARD, (double)cc.W), gy = dmul(GUARD, (double)cc.H);
        const double ml = dsub(mux.l, dmul(BOX_SLACK, dadd(1.0, fabs(mux.l))));
        const double mh = dadd(mux.u, dmul(BOX_SLACK, dadd(1.0, fabs(mux.u))));
        const double nl = dsub(muy.l, dmul(BOX_SLACK, dadd(1.0, fabs(muy.l))));
        const double nh = dadd(muy.u, dmul(BOX_SLACK, dadd(1.0, fabs(muy.u))));
        if (ml > dadd(cx, gx) || mh < dsub(cx, gx) || nl > dadd(cy, gy) || nh < dsub(cy, gy)) return SCREEN_DROP;
        if (!(ml >= dsub(cx, gx) && mh <= dadd(cx, gx) && nl >= dsub(cy, gy) && nh <= dadd(cy, gy)))
            straddle = true;
    }
    double X00 = 0, X11 = 0;
    for (int c = 0; c < 3; ++c) {
        DI m[3];
        for (int a = 0; a < 3; ++a)
            m[a] = di_add(di_add(di_scale(Ri[a], N[c]), di_scale(Ri[3 + a], N[3 + c])), di_scale(Ri[6 + a], N[6 + c]));
        DI p0 = di_scale(di_add(di_mul_pos(D, m[0]), di_scale(di_mul(ucx, m[2]), -1.0)), fx);
        DI p1 = di_scale(di_add(di_mul_pos(D, m[1]), di_scale(di_mul(ucy, m[2]), -1.0)), fy);
        X00 = dadd(X00, di_sqmax(p0));
        X11 = dadd(X11, di_sqmax(p1));
    }
    const double dl2 = dmul(dl, dl);
    const double rx = sqrt(dmul(tau, X00)) / dl2, ry = sqrt(dmul(tau, X11)) / dl2;
    double xl = dsub(mux.l, rx), xh = dadd(mux.u, rx), yl = dsub(muy.l, ry), yh = dadd(muy.u, ry);
    xl = dsub(xl, dmul(BOX_SLACK, dadd(1.0, fabs(xl))));
    xh = dadd(xh, dmul(BOX_SLACK, dadd(1.0, fabs(xh))));
    yl = dsub(yl, dmul(BOX_SLACK, dadd(1.0, fabs(yl))));
    yh = dadd(yh, dmul(BOX_SLACK, dadd(1.0, fabs(yh))));
    if (!(xh >= xl) || !(yh >= yl)) return SCREEN_DROP;
    double fx0 = ceil(dsub(xl, 0.5)), fx1 = floor(dsub(xh, 0.5));
    double fy0 = ceil(dsub(yl, 0.5)), fy1 = floor(dsub(yh, 0.5));
    fx0 = fmax(fx0, 0.0); fy0 = fmax(fy0, 0.0);
    fx1 = fmin(fx1, (double)(cc.W - 1)); fy1 = fmin(fy1, (double)(cc.H - 1));
    if (fx0 > fx1 || fy0 > fy1) return SCREEN_DROP;
    box = PixBox{(int)fx0, (int)fx1, (int)fy0, (int)fy1};
    mu_px[0] = floor(fmin(fmax(0.5 * (mux.l + mux.u), -1e6), 1e6)) + 0.5;
    mu_px[1] = floor(fmin(fmax(0.5 * (muy.l + muy.u), -1e6), 1e6)) + 0.5;
    return SCREEN_KEEP;
}

// The enclosures screen_fp32 starts from: the concretised R_delta entries
// and v - s (enc: the enclosures of v_lo, v_hi, N that pose_prep_kernel
// stored)
template <int M>
__device__ __forceinline__ void screen_inputs_fp32(const CellData<M> &cd, const float *enc, EI *Ri, EI *vs, bool &ok)
{
    for (int e = 0; e < 9; ++e)
        Ri[e] = EI{E32{cd.rd_int32[e][0][0], cd.rd_int32[e][0][1]}, E32{cd.rd_int32[e][1][0], cd.rd_int32[e][1][1]}};
    for (int b = 0; b < 3; ++b)
        vs[b] = EI{e_chk(e_sub(E32{enc[2 * b], enc[2 * b + 1]}, E32{cd.s_int32[b][1][0], cd.s_int32[b][1][1]}), ok),
                   e_chk(e_sub(E32{enc[6 + 2 * b], enc[7 + 2 * b]}, E32{cd.s_int32[b][0][0], cd.s_int32[b][0][1]}),
                         ok)};
}

// The first decisions of screen_fp32, from enclosures D of the depth ends
// (max(d_lo, near), d_hi): the camera-frame x, y and the projected mean's
// interval (ucx, ucy, mux, muy), then the frustum guard band: SCREEN_DROP,
// SCREEN_KEEP inside the band, SCREEN_STRADDLE across it, or
// SCREEN_UNDECIDED where the enclosures do not settle it.
enum { SCREEN_STRADDLE = 3 };
template <int M>
__device__ __forceinline__ int screen_guard_fp32(const CellData<M> &cd, const EI *Ri, const EI *vs, const EI &D,
                                                 const CallConst &cc, EI &ucx, EI &ucy, EI &mux, EI &muy, bool &ok)
{
    ucx = ei_add(ei_add(ei_mul(Ri[0], vs[0], ok), ei_mul(Ri[3], vs[1], ok), ok), ei_mul(Ri[6], vs[2], ok), ok);
    ucy = ei_add(ei_add(ei_mul(Ri[1], vs[0], ok), ei_mul(Ri[4], vs[1], ok), ok), ei_mul(Ri[7], vs[2], ok), ok);
    // the intrinsics are floats: exact
    const E32 fx = {cc.fx, cc.fx}, fy = {cc.fy, cc.fy}, cx = {cc.cx, cc.cx}, cy = {cc.cy, cc.cy};
    // u / D_hi or u / D_lo by the sign of u; where the sign is not settled,
    // the enclosure of either quotient
    auto qlo = [&](E32 u) {
        const E32 a = e_div_pos(u, D.u), b = e_div_pos(u, D.l);
        return u.lo >= 0.f ? a : (u.hi < 0.f ? b : e_hull(a, b));
    };
    auto qhi = [&](E32 u) {
        const E32 a = e_div_pos(u, D.l), b = e_div_pos(u, D.u);
        return u.lo >= 0.f ? a : (u.hi < 0.f ? b : e_hull(a, b));
    };
    mux = EI{e_chk(e_add(cx, e_mul(fx, qlo(ucx.l))), ok), e_chk(e_add(cx, e_mul(fx, qhi(ucx.u))), ok)};
    muy = EI{e_chk(e_add(cy, e_mul(fy, qlo(ucy.l))), ok), e_chk(e_add(cy, e_mul(fy, qhi(ucy.u))), ok)};
    if (!ok) return SCREEN_UNDECIDED;
    const E32 one = {1.f, 1.f}, slack = {cd.slack32[0], cd.slack32[1]};
    auto widen_dn = [&](E32 x) { return e_sub(x, e_mul(slack, e_add(one, e_abs(x)))); };
    auto widen_up = [&](E32 x) { return e_add(x, e_mul(slack, e_add(one, e_abs(x)))); };
    const E32 cxp = {cd.guard32[0][0], cd.guard32[0][1]}, cxm = {cd.guard32[1][0], cd.guard32[1][1]};
    const E32 cyp = {cd.guard32[2][0], cd.guard32[2][1]}, cym = {cd.guard32[3][0], cd.guard32[3][1]};
    const E32 ml = widen_dn(mux.l), mh = widen_up(mux.u), nl = widen_dn(muy.l), nh = widen_up(muy.u);
    // drop: ml > cx + gx || mh < cx - gx || nl > cy + gy || nh < cy - gy
    const int d0 = e_gt(ml, cxp), d1 = e_gt(cxm, mh), d2 = e_gt(nl, cyp), d3 = e_gt(cym, nh);
    if (d0 == 1 || d1 == 1 || d2 == 1 || d3 == 1) return SCREEN_DROP;
    if (d0 < 0 || d1 < 0 || d2 < 0 || d3 < 0) return SCREEN_UNDECIDED;
    // inside: ml >= cx - gx && mh <= cx + gx && nl >= cy - gy && nh <= cy + gy
    const int i0 = e_ge(ml, cxm), i1 = e_ge(cxp, mh), i2 = e_ge(nl, cym), i3 = e_ge(cyp, nh);
    if (i0 < 0 || i1 < 0 || i2 < 0 || i3 < 0) return SCREEN_UNDECIDED;
    return (i0 && i1 && i2 && i3) ? SCREEN_KEEP : SCREEN_STRADDLE;
}

// FP32 enclosures of the depth chain's ends dlo, dhi (record_decide), step
// for step on enclosures of its operands; ok is cleared where a value leaves
// the checked range or a sign the chain branches on is not settled.  Every
// FP64 result of the chain, rounded to nearest, lies in these enclosures.
template <int M>
__device__ __forceinline__ void depth_fp32(const CellData<M> &cd, const float *enc, E32 &dlo, E32 &dhi, bool &ok)
{
    const int n_t = cd.n_t, n_a = cd.n_a;
    const E32 half = {0.5f, 0.5f};
    auto E = [](const float *p) { return E32{p[0], p[1]}; };
    E32 ddr[M];
    E32 dlk = {0.f, 0.f}, dhk = {0.f, 0.f};
    for (int b = 0; b < 3; ++b) {
        const E32 xl = E(cd.dx32[b][0]), xh = E(cd.dx32[b][1]), xm = E(cd.dx32[b][2]);
        const E32 ylk = e_sub(E32{enc[2 * b], enc[2 * b + 1]}, E(cd.s32[b][M]));
        const E32 yhk = e_sub(E32{enc[6 + 2 * b], enc[7 + 2 * b]}, E(cd.s32[b][M]));
        E32 yl = ylk, yh = yhk;
        for (int j = 0; j < n_t; ++j) {
            yl = e_sub(yl, e_abs(E(cd.s32[b][j])));
            yh = e_add(yh, e_abs(E(cd.s32[b][j])));
        }
        const E32 ym = e_mul(half, e_add(yl, yh));
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < n_t || j >= n_a) continue;
            const E32 t = e_mul(ym, E(cd.rdd32[b][0][j]));
            ddr[j] = b == 0 ? t : e_add(ddr[j], t);
        }
        // the chain branches on ym >= 0 and xm >= 0 (xm: rounding down keeps the sign)
        if (!(ym.lo >= 0.f) && !(ym.hi < 0.f)) {
            ok = false;
            return;
        }
        const bool yp = ym.lo >= 0.f, xp = xm.lo >= 0.f;
        E32 lk = e_add(e_mul(ym, E(cd.rdd32[b][yp ? 0 : 1][M])), e_mul(xm, xp ? ylk : yhk));
        lk = e_sub(lk, e_mul(half, e_add(e_mul(xl, yl), e_mul(xh, yh))));
        E32 hk = e_add(e_mul(ym, E(cd.rdd32[b][yp ? 1 : 0][M])), e_mul(xm, xp ? yhk : ylk));
        hk = e_sub(hk, e_mul(half, e_add(e_mul(xh, yl), e_mul(xl, yh))));
        dlk = b == 0 ? lk : e_add(dlk, lk);
        dhk = b == 0 ? hk : e_add(dhk, hk);
    }
    dlo = dlk;
    dhi = dhk;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (j >= n_a) continue;
        const E32 c = e_abs(j < n_t ? E(cd.ddt32[j]) : ddr[j]);
        dlo = e_sub(dlo, c);
        dhi = e_add(dhi, c);
    }
    e_chk(dlo, ok);
    e_chk(dhi, ok);
}

// The same decisions from FP32 enclosures (E32) of every FP64 value above,
// step for step: where each comparison, ceil and floor of screen_fp64 is
// settled by the enclosures, it has the same outcome as in FP64; otherwise
// (or when a value leaves the checked range) SCREEN_UNDECIDED.  GB300's FP64
// rate is about 1/64 of its FP32 rate, and the FP64 path is then taken by a
// small fraction of the pairs.
template <int M>
__device__ __forceinline__ int screen_fp32(const CellData<M> &cd, const float *enc, double dlo, double dhi,
                                           double tau, const CallConst &cc, PixBox &box, double *mu_px,
                                           bool &straddle)
{
    bool ok = true;
    const double nearp = (double)cc.near_plane;
    EI Ri[9], vs[3];
    screen_inputs_fp32(cd, enc, Ri, vs, ok);
    E32 Ne[9];
    for (int i = 0; i < 9; ++i) Ne[i] = E32{enc[12 + 2 * i], enc[13 + 2 * i]};
    const double dl = fmax(dlo, nearp);
    const EI D = {e_of(dl), e_of(dhi)};
    EI ucx, ucy, mux, muy;
    const int g = screen_guard_fp32(cd, Ri, vs, D, cc, ucx, ucy, mux, muy, ok);
    if (g == SCREEN_DROP) return SCREEN_DROP;
    if (g == SCREEN_UNDECIDED) return SCREEN_UNDECIDED;
    if (g == SCREEN_STRADDLE) straddle = true;
    const E32 fx = {cc.fx, cc.fx}, fy = {cc.fy, cc.fy};
    const E32 one = {1.f, 1.f}, slack = {cd.slack32[0], cd.slack32[1]};
    auto widen_dn = [&](E32 x) { return e_sub(x, e_mul(slack, e_add(one, e_abs(x)))); };
    auto widen_up = [&](E32 x) { return e_add(x, e_mul(slack, e_add(one, e_abs(x)))); };
    E32 X00 = {0.f, 0.f}, X11 = {0.f, 0.f};
    for (int c = 0; c < 3; ++c) {
        EI m[3];
        for (int a = 0; a < 3; ++a)
            m[a] = ei_add(ei_add(ei_scale(Ri[a], Ne[c], ok), ei_scale(Ri[3 + a], Ne[3 + c], ok), ok),
                          ei_scale(Ri[6 + a], Ne[6 + c], ok), ok);
        const EI p0 = ei_scale(ei_add(ei_mul_pos(D, m[0], ok), ei_neg(ei_mul(ucx, m[2], ok)), ok), fx, ok);
        const EI p1 = ei_scale(ei_add(ei_mul_pos(D, m[1], ok), ei_neg(ei_mul(ucy, m[2], ok)), ok), fy, ok);
        X00 = e_chk(e_add(X00, ei_sqmax(p0)), ok);
        X11 = e_chk(e_add(X11, ei_sqmax(p1)), ok);
    }
    const E32 dl2 = e_mul(e_of(dl), e_of(dl)), t = e_of(tau);
    const E32 rx = e_chk(e_div_pos(e_sqrt(e_mul(t, X00)), dl2), ok);
    const E32 ry = e_chk(e_div_pos(e_sqrt(e_mul(t, X11)), dl2), ok);
    if (!ok) return SCREEN_UNDECIDED;
    const E32 xl = widen_dn(e_sub(mux.l, rx)), xh = widen_up(e_add(mux.u, rx));
    const E32 yl = widen_dn(e_sub(muy.l, ry)), yh = widen_up(e_add(muy.u, ry));
    // (xh >= xl and yh >= yl hold: the enclosures are finite and ordered)
    if (e_ge(xh, xl) != 1 || e_ge(yh, yl) != 1) return SCREEN_UNDECIDED;
    const E32 half = {0.5f, 0.5f};
    const E32 ax = e_sub(xl, half), bx = e_sub(xh, half), ay = e_sub(yl, half), by = e_sub(yh, half);
    float fx0 = ceilf(ax.lo), fx1 = floorf(bx.lo), fy0 = ceilf(ay.lo), fy1 = floorf(by.lo);
    if (fx0 != ceilf(ax.hi) || fx1 != floorf(bx.hi) || fy0 != ceilf(ay.hi) || fy1 != floorf(by.hi))
        return SCREEN_UNDECIDED;
    fx0 = fmaxf(fx0, 0.f); fy0 = fmaxf(fy0, 0.f);
    fx1 = fminf(fx1, (float)(cc.W - 1)); fy1 = fminf(fy1, (float)(cc.H - 1));
    if (fx0 > fx1 || fy0 > fy1) return SCREEN_DROP;
    // the midpoint of the mean's interval, clamped, floored (0.5 scales exactly)
    float mp[2];
    const EI mu2[2] = {mux, muy};
    for (int k = 0; k < 2; ++k) {
        const E32 sm = e_add(mu2[k].l, mu2[k].u);
        const float a = floorf(fminf(fmaxf(0.5f * sm.lo, -1e6f), 1e6f)), b = floorf(fminf(fmaxf(0.5f * sm.hi, -1e6f), 1e6f));
        if (a != b) return SCREEN_UNDECIDED;
        mp[k] = a;
    }
    box = PixBox{(int)fx0, (int)fx1, (int)fy0, (int)fy1};
    mu_px[0] = (double)mp[0] + 0.5;
    mu_px[1] = (double)mp[1] + 0.5;
    return SCREEN_KEEP;
}

// The decision part of one (Gaussian, cell) pair: depth forms, near-plane
// class, depth key, pixel box and projected-mean interval, all in FP64.  It
// writes the pair's key interval and box, and the scalar fields of its record
// (o, tau, colour, flags F_STRADDLE / F_OPEN, the pixel centre mu); returns
// the flags word, or -1 when the pair contributes to no pixel.  RO is the
// precision of the stored record: float for the batched renderer (FP32 value
// chain with outward rounding), double for the plain FP64 renderer, where
// the same steps run with every value kept in FP64.
template <int M, class RO = float>
__device__ __forceinline__ int64_t record_decide(const double *__restrict__ vN, const GParam *__restrict__ gp,
                                                 const CallConst &cc, const CellData<M> &cd, int cell, int64_t g,
                                                 int TS, RO *__restrict__ recs, PixBox *__restrict__ boxes,
                                                 double *__restrict__ keys, PrepCount &pc)
{
    using RL = Rec<M>;
    const int64_t ri = (int64_t)cell * cc.n_gauss + g;
    PixBox box = {-1, -1, -1, -1};
    boxes[ri] = box;
    const GParam P = gp[g];
    const double tau = P.tau_hi;  // the largest cutoff exponent of the opacity box
    if (!(tau >= 0)) return -1;   // o < 1/255: never above the cutoff
    // v as an interval over the mean's box (lo = hi without one), then N
    const double *vl = vN + VN_STRIDE * g, *vh = vl + 3, *N = vl + 6;

    // ---- FP64 decision chain: depth d = sum_b R_delta[b][2] (v_b - s_b) by
    // averaged McCormick products (the lower form of x y is y_m x + x_m y -
    // (x_lo y_lo + x_hi y_hi)/2 with each operand's side chosen by the sign of
    // the other's midpoint, the upper one likewise), summed, then its bounds,
    // the near-plane class and the depth key.  These are the round-to-nearest
    // IEEE operations of that statement on the full forms, in its order, less
    // the ones whose operand is a coefficient that is zero by construction
    // (R_delta[b][2] lives on the rotation slots, s_b on the translation
    // slots; adding, subtracting or scaling zero changes no value but the sign
    // of a zero, which the bounds never see) and less the per-cell parts the
    // cell kernel computed.  So dlo, dhi, klo and khi are bit-identical to the
    // plain statement.
    const int n_t = cd.n_t, n_a = cd.n_a;
    double ddr[M];  // rotation-slot coefficients of d
    double dlk = 0.0, dhk = 0.0;  // constants of d's lower and upper forms
    for (int b = 0; b < 3; ++b) {
        const int e = 3 * b + 2;
        const double xl = cd.dx[b][0], xh = cd.dx[b][1], xm = cd.dx[b][2];
        // v_b - s_b: constants of its lower and upper forms
        const double ylk = dsub(vl[b], cd.s[b][M]), yhk = dsub(vh[b], cd.s[b][M]);
        double yl = ylk, yh = yhk;
        for (int j = 0; j < n_t; ++j) {
            yl = dsub(yl, fabs(cd.s[b][j]));
            yh = dadd(yh, fabs(cd.s[b][j]));
        }
        const double ym = dmul(0.5, dadd(yl, yh));
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < n_t || j >= n_a) continue;
            const double t = dmul(ym, cd.rd_lo[e][j]);
            ddr[j] = b == 0 ? t : dadd(ddr[j], t);
        }
        double lk = dadd(dmul(ym, ym >= 0 ? cd.rd_lo[e][M] : cd.rd_hi[e][M]), dmul(xm, xm >= 0 ? ylk : yhk));
        lk = dsub(lk, dmul(0.5, dadd(dmul(xl, yl), dmul(xh, yh))));
        double hk = dadd(dmul(ym, ym >= 0 ? cd.rd_hi[e][M] : cd.rd_lo[e][M]), dmul(xm, xm >= 0 ? yhk : ylk));
        hk = dsub(hk, dmul(0.5, dadd(dmul(xh, yl), dmul(xl, yh))));
        dlk = b == 0 ? lk : dadd(dlk, lk);
        dhk = b == 0 ? hk : dadd(dhk, hk);
    }
    double dlo = dlk, dhi = dhk, klo = dlk, khi = dhk;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (j >= n_a) continue;
        const double c = j < n_t ? cd.dd_t[j] : ddr[j];   // d's coefficient
        const double ck = j < n_t ? cd.kd_t[j] : ddr[j];  // the key form's (d minus the shared term g)
        dlo = dsub(dlo, fabs(c));
        dhi = dadd(dhi, fabs(c));
        klo = dsub(klo, fabs(ck));
        khi = dadd(khi, fabs(ck));
    }
    const double nearp = (double)cc.near_plane;
    if (!(dhi > nearp)) return -1;
    bool straddle = !(dlo > nearp);
    {
        double pad = dmul(KEY_SLACK, dadd(1.0, fmax(fabs(klo), fabs(khi))));
        klo = dsub(klo, pad);
        khi = dadd(khi, pad);
    }
    // screen box, projected-mean pixel centre and guard band: decided from
    // FP32 enclosures of the FP64 values where they settle every decision,
    // else in FP64 (the same values either way)
    double mu_px[2];
    int sr = screen_fp32<M>(cd, reinterpret_cast<const float *>(vl + VN_ENC), dlo, dhi, tau, cc, box, mu_px,
                            straddle);
    if (sr == SCREEN_UNDECIDED)
        sr = screen_fp64(cd.rd_int, cd.s_int, vl, vh, N, dlo, dhi, tau, cc, box, mu_px, straddle);
    if (sr == SCREEN_DROP) return -1;
    RO *rec = recs + ri * RL::WIDTH;
    const uint32_t flags = (straddle ? F_STRADDLE : 0u) | (klo < khi ? F_OPEN : 0u);
    // the opacity box: the lower forms are cut from tau(o_lo), the upper ones
    // from tau(o_hi); the colour box: c_lo for the lower sum, c_hi the upper
    rec[RL::O] = P.o_hi;
    rec[RL::O_LO] = P.o_lo;
    rec_dn(P.tau_lo, rec[RL::TAU_DN]);
    rec_up(P.tau_hi, rec[RL::TAU_UP]);
    for (int k = 0; k < 3; ++k) {
        rec[RL::COL + k] = P.c_lo[k];
        rec[RL::COL_HI + k] = P.c_hi[k];
    }
    // pixel centre near the projected mean, the expansion point of R = mu S - P
    rec[RL::MU_X] = (RO)mu_px[0];
    rec[RL::MU_Y] = (RO)mu_px[1];
    rec_put_flags(rec + RL::FLAGS, flags);
    keys[2 * ri] = klo;
    keys[2 * ri + 1] = khi;
    boxes[ri] = box;
    pc.triples = (uint32_t)(box.x1 - box.x0 + 1) * (uint32_t)(box.y1 - box.y0 + 1);
    pc.valid = 1;
    pc.tiles = (uint32_t)(box.x1 / TS - box.x0 / TS + 1) * (uint32_t)(box.y1 / TS - box.y0 / TS + 1);
    return flags;
}

// MatrixInv (Algorithm 3) on X, FP64 forms over a box (X10 = X01): X0 is
// the inverse of the centre matrix (adjustment (1) of Sec. 3.1), in FP64 as
// the oracle takes it, so that rho, and with it the assertion of Algorithm 3
// and the Taylor order, is the oracle's up to FP64 rounding; E = I - X X0 and
// rho are formed in FP64, E is rounded outward to the series precision RS,
// the series T = sum_{i=1..k} E^i runs in RS, and Conic = X0 (I + T) +- Eps
// is assembled in FP64 with the same X0.  (The assembly's constants are of the size of X0; in
// FP32 their outward rounding would widen every entry of W = Conic Mp by a
// few u of its size, which the Mahalanobis term of far pixels multiplies by
// 2 |q|^2.  T is small, ||T|| <= rho / (1 - rho), so its FP32 error is not.)
// The order starts at the default KTAYLOR and grows while the remainder
// bound rho^(k+1) / (1 - rho) exceeds EPS_TOL (relative to ||X0||_F), up to
// KMAX (adjustment (3)).  Returns MI_FAIL when the centre matrix is not
// positive definite or rho >= RHO_MAX, MI_KHIGH (without running the series)
// when the order would exceed KC, else MI_OK.  (KC = KTAYLOR fixes the series
// length at compile time.)
enum { MI_FAIL = 0, MI_OK = 1, MI_KHIGH = 2 };
template <int M, class RS, int KC = KMAX>
__device__ __forceinline__ int matinv_box(const SB<M, double> X[4], SB<M, double> conic[4])
{
    typedef SB<M, RS> B;
    typedef SB<M, double> BD;
    typedef SAcc<M, double> AD;
    const double h00 = 0.5 * (X[0].vlo + X[0].vhi), h01 = 0.5 * (X[1].vlo + X[1].vhi);
    const double h11 = 0.5 * (X[3].vlo + X[3].vhi);
    const double det = h00 * h11 - h01 * h01;
    if (!(det > 0.0) || !(h00 > 0.0) || !isfinite(det)) return false;
    const double X0[4] = {h11 / det, -h01 / det, -h01 / det, h00 / det};
    B E[4];
    double rho2 = 0.0;
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            AD p;
            const double dl = (r == s) ? 1.0 : 0.0;
            p.init(dl, dl);
            p.term(-X0[s], X[2 * r]);
            p.term(-X0[2 + s], X[2 * r + 1]);
            const BD e64 = p.result();
            const double m = fmax(fabs(e64.vlo), fabs(e64.vhi));
            rho2 = __fma_ru(m, m, rho2);
            sb_to_rec<M>(e64, E[2 * r + s]);
        }
    const double rho64 = __dsqrt_ru(rho2);
    if (!(rho64 < RHO_MAX)) return false;
    int k = KTAYLOR;
    {
        double rk = 1.0;  // rho^(k+1), for the adaptive order
        for (int i = 0; i <= KTAYLOR; ++i) rk *= rho64;
        // (only whether the order exceeds KC matters when KC < KMAX)
        constexpr int kstop = KC < KMAX ? KC + 1 : KMAX;
        while (k < kstop && rk / (1.0 - rho64) > EPS_TOL) {
            rk *= rho64;
            ++k;
        }
    }
    if (k > KC) return MI_KHIGH;
    if (KC == KTAYLOR) k = KTAYLOR;
    // T = sum_{i=1..k} (I - X X0)^i, so that Xp = X0 (I + T) = X0 + X0 T: the
    // identity term is added as an exact constant at the end
    B P[4], Ssum[4];
    for (int e = 0; e < 4; ++e) {
        P[e] = E[e];
        Ssum[e] = E[e];
    }
#pragma unroll 1
    for (int i = 2; i <= k; ++i) {
        B Q[4];
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s) {
                SAcc<M, RS> p;
                p.init(0, 0);
                p.mul(P[2 * r], E[s]);
                p.mul(P[2 * r + 1], E[2 + s]);
                Q[2 * r + s] = p.result();
            }
        for (int e = 0; e < 4; ++e) { P[e] = Q[e]; Ssum[e] = sb_add<M, RS>(Ssum[e], Q[e]); }
    }
    // Eps = ||X0||_F rho^(k+1) / (1 - rho), and the assembly, in FP64
    const double *X0d = X0;
    double nX0 = 0.0;
    for (int e = 0; e < 4; ++e) nX0 = __fma_ru(X0d[e], X0d[e], nX0);
    nX0 = __dsqrt_ru(nX0);
    double rk = 1.0;
    for (int i = 0; i <= k; ++i) rk = __dmul_ru(rk, rho64);
    const double eps = __ddiv_ru(__dmul_ru(nX0, rk), __dsub_rd(1.0, rho64));
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            AD p;
            // X0[r][s] + eps-widening, then + X0 T
            p.init(__dsub_rd(X0d[2 * r + s], eps), __dadd_ru(X0d[2 * r + s], eps));
            p.term(X0d[2 * r], to_f64<M>(Ssum[s]));
            p.term(X0d[2 * r + 1], to_f64<M>(Ssum[2 + s]));
            conic[2 * r + s] = p.result();
        }
    return true;
}

// x restricted to the sub-box p = ctr + h p' of the cell, as a form over p'
// (h is a power of two, so the coefficients scale exactly; the constants
// take c . ctr rounded outward).
template <int M>
__device__ __forceinline__ SB<M, double> sb_restrict(const SB<M, double> &x, const double *ctr, const double *h)
{
    SB<M, double> y;
    double klo = x.klo, khi = x.khi;
    for (int j = 0; j < M; ++j) {
        y.c[j] = x.c[j] * h[j];
        klo = __fma_rd(x.c[j], ctr[j], klo);
        khi = __fma_ru(x.c[j], ctr[j], khi);
    }
    y.klo = __dsub_rd(klo, 1e-300);  // covers a subnormal c h
    y.khi = __dadd_ru(khi, 1e-300);
    sb_finish(y);
    return y;
}

// The pose variable a piece is bisected along: the one on which X varies most
// there (the largest sum over X00, X01, X11 of |c_j|; the first on a tie).
template <int M>
__device__ __forceinline__ int split_var(const SB<M, double> Xr[4])
{
    int js = 0;
    double best = -1.0;
    for (int j = 0; j < M; ++j) {
        const double v = fabs(Xr[0].c[j]) + fabs(Xr[1].c[j]) + fabs(Xr[3].c[j]);
        if (v > best) {
            best = v;
            js = j;
        }
    }
    return js;
}

// Adjustment (2) of Sec. 3.1, for a cell on which MatrixInv failed: the cell
// is bisected along split_var, depth first and lower half first, and each
// piece that still fails is bisected again, down to SPLIT_DEPTH bisections,
// until MatrixInv holds on every piece.  The pieces' outputs are forms over
// different boxes, so they are joined as constant forms: each entry is
// bounded by the least lower and the greatest upper concretised bound over
// the pieces.  Returns the number of pieces, or 0 if a piece at the depth
// limit still fails.  At most one pending sibling per level waits on the
// stack, so SPLIT_DEPTH + 1 entries suffice.
template <int M, class RS>
__device__ __noinline__ int matinv_split(const SB<M, double> X[4], SB<M, double> conic[4])
{
    struct Piece {
        double ctr[M], h[M];
        int depth;
    };
    Piece st[SPLIT_DEPTH + 1];
    int top = 0;
    double lo[4], hi[4];
    for (int e = 0; e < 4; ++e) {
        lo[e] = Num<double>::BIG;
        hi[e] = -Num<double>::BIG;
    }
    // push the two halves of a piece, the upper one first
    auto push_halves = [&](const double *ctr, const double *h, int depth, const SB<M, double> Xr[4]) {
        const int js = split_var<M>(Xr);
        for (int side = 1; side >= 0; --side) {
            Piece &q = st[top++];
            for (int j = 0; j < M; ++j) {
                q.ctr[j] = ctr[j];
                q.h[j] = h[j];
            }
            q.h[js] = 0.5 * h[js];
            q.ctr[js] = side ? ctr[js] + q.h[js] : ctr[js] - q.h[js];
            q.depth = depth + 1;
        }
    };
    {
        double ctr[M], h[M];
        for (int j = 0; j < M; ++j) {
            ctr[j] = 0.0;
            h[j] = 1.0;
        }
        push_halves(ctr, h, 0, X);
    }
    int pieces = 0;
    while (top > 0) {
        const Piece q = st[--top];
        SB<M, double> Xr[4];
        for (int e = 0; e < 4; ++e) Xr[e] = sb_restrict<M>(X[e], q.ctr, q.h);
        SB<M, double> C[4];
        if (matinv_box<M, RS>(Xr, C) == MI_OK) {
            for (int e = 0; e < 4; ++e) {
                lo[e] = fmin(lo[e], C[e].vlo);
                hi[e] = fmax(hi[e], C[e].vhi);
            }
            ++pieces;
        } else if (q.depth < SPLIT_DEPTH) {
            push_halves(q.ctr, q.h, q.depth, Xr);
        } else {
            return 0;
        }
    }
    for (int e = 0; e < 4; ++e) conic[e] = sb_cst<M, double>(lo[e], hi[e]);
    return pieces;
}

// Split modes of record_value (see there).
enum { SPLIT_INLINE = 0, SPLIT_DEFER = 1, SPLIT_WARP = 2 };

// A piece of the pose cell for matinv_split_warp, packed in 64 bits: for each
// slot j, bits 9j..9j+2 hold its bisection depth d_j and bits 9j+3..9j+8 its
// index i_j, the piece being ctr_j = (2 i_j + 1) 2^-d_j - 1, h_j = 2^-d_j
// (exact dyadic numbers, the same as repeated halving gives).
__device__ __forceinline__ uint64_t piece_child(uint64_t pc, int js, int upper)
{
    const uint64_t f = (pc >> (9 * js)) & 511u;
    const uint64_t d = f & 7u, i = f >> 3;
    const uint64_t g = (d + 1) | (((2 * i + (uint64_t)upper)) << 3);
    return (pc & ~((uint64_t)511u << (9 * js))) | (g << (9 * js));
}
template <int M>
__device__ __forceinline__ void piece_box(uint64_t pc, double *ctr, double *h)
{
    for (int j = 0; j < M; ++j) {
        const uint32_t f = (uint32_t)(pc >> (9 * j)) & 511u;
        const int d = (int)(f & 7u), i = (int)(f >> 3);
        h[j] = ldexp(1.0, -d);
        ctr[j] = (double)(2 * i + 1) * h[j] - 1.0;
    }
}

// matinv_split with the 32 lanes of a warp, for a pair on whose cell
// MatrixInv failed: the same pieces (each failing piece bisected along its
// own split_var, down to SPLIT_DEPTH), tried level by level with one piece
// per lane; the hull and the outcome do not depend on the order.  Every lane
// passes the same X and gets the same result; list is the warp's 2 x 64
// shared-memory piece lists.  Returns the number of pieces, or 0 if a piece
// at the depth limit still fails.
template <int M, class RS>
__device__ __noinline__ int matinv_split_warp(const SB<M, double> X[4], SB<M, double> conic[4], uint64_t *list)
{
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    double lo[4], hi[4];
    for (int e = 0; e < 4; ++e) {
        lo[e] = Num<double>::BIG;
        hi[e] = -Num<double>::BIG;
    }
    int pieces = 0;
    bool failed = false;
    {
        const int js = split_var<M>(X);
        if (lane == 0) {
            list[0] = piece_child(0, js, 0);
            list[1] = piece_child(0, js, 1);
        }
    }
    __syncwarp();
    int cnt = 2, cur = 0;
    for (int depth = 1; depth <= SPLIT_DEPTH && cnt > 0; ++depth) {
        int next = 0;
        for (int base = 0; base < cnt; base += 32) {
            const int i = base + lane;
            bool need = false;
            uint64_t pc = 0;
            int js = 0;
            if (i < cnt) {
                pc = list[cur * 64 + i];
                double ctr[M], h[M];
                piece_box<M>(pc, ctr, h);
                SB<M, double> Xr[4];
                for (int e = 0; e < 4; ++e) Xr[e] = sb_restrict<M>(X[e], ctr, h);
                SB<M, double> C[4];
                if (matinv_box<M, RS>(Xr, C) == MI_OK) {
                    for (int e = 0; e < 4; ++e) {
                        lo[e] = fmin(lo[e], C[e].vlo);
                        hi[e] = fmax(hi[e], C[e].vhi);
                    }
                    ++pieces;
                } else if (depth < SPLIT_DEPTH) {
                    need = true;
                    js = split_var<M>(Xr);
                } else {
                    failed = true;
                }
            }
            const unsigned m = __ballot_sync(full, need);
            if (need) {
                const int at = next + 2 * __popc(m & ((1u << lane) - 1u));
                list[(cur ^ 1) * 64 + at] = piece_child(pc, js, 0);
                list[(cur ^ 1) * 64 + at + 1] = piece_child(pc, js, 1);
            }
            next += 2 * __popc(m);
        }
        __syncwarp();
        if (__any_sync(full, failed)) return 0;
        cnt = next;
        cur ^= 1;
    }
    for (int off = 16; off > 0; off >>= 1) {
        pieces += __shfl_xor_sync(full, pieces, off);
        for (int e = 0; e < 4; ++e) {
            lo[e] = fmin(lo[e], __shfl_xor_sync(full, lo[e], off));
            hi[e] = fmax(hi[e], __shfl_xor_sync(full, hi[e], off));
        }
    }
    for (int e = 0; e < 4; ++e) conic[e] = sb_cst<M, double>(lo[e], hi[e]);
    return pieces;
}

// The value part of one (Gaussian, cell) pair: the forms the per-pixel stage
// reads, S = d^2 and R = mu S - P (Algorithm 1 lines 2-8 with set-valued
// variables), MatrixInv (Algorithm 3) and W = Conic Mp.  v points at the
// Gaussian's v (3) and N (9); rec holds the scalar fields record_decide wrote,
// mu_x / mu_y and flags are their values; fx, fy, cx, cy the intrinsics.  Writes the forms and the flags word
// (with F_FALLBACK where the MatrixInv assertion fails or a form is not
// finite) and returns that word.  SPLIT: where MatrixInv fails on the cell,
// SPLIT_INLINE splits it in this thread (matinv_split), SPLIT_DEFER returns
// the flags with F_SPLIT_PENDING before writing W and the flags (and with
// F_KHIGH_PENDING where the cell's Taylor order would exceed KTAYLOR), and
// SPLIT_WARP (all 32 lanes of a warp call it for one deferred pair, with the
// warp's split_list) splits it with the warp (matinv_split_warp).
template <int M, class RO = float, int SPLIT = SPLIT_INLINE>
__device__ __forceinline__ uint32_t record_value(const double *__restrict__ v, float fx, float fy, float cx, float cy,
                                                 const CellData<M> &cd, RO mux, RO muy, uint32_t flags, RO *rec,
                                                 uint64_t *split_list = nullptr)
{
    using RL = Rec<M>;
    using NO = Num<RO>;
    typedef SB<M, RO> B;
    typedef SB<M, double> BD;
    typedef SAcc<M, double> AD;
    // v: lower ends (3), upper ends (3) over the mean's box, then N (9)
    const double *N = v + 6;
    bool ok = true;
    // ---- FP64 value chain (directed rounding): uc, S, P, Mc, J, Mp, X, E.
    // These are differences of large, nearly equal terms (S u - P, I - X X0,
    // Conic Mp); carrying them in FP64 keeps their FP32 images accurate.
    BD uc64[3];
    {
        double vabs = 1.0;
        for (int b = 0; b < 3; ++b) vabs += fmax(fabs(v[b]), fabs(v[3 + b]));
        const double ev = __dmul_ru(1e-14, vabs);
        BD vm[3];
        for (int b = 0; b < 3; ++b) {
            AD p;
            p.init(__dsub_rd(v[b], ev), __dadd_ru(v[3 + b], ev));
            p.term(-1.0, cd.s64[b]);
            vm[b] = p.result();
        }
        for (int a = 0; a < 3; ++a) {
            AD p;
            p.init(0.0, 0.0);
            p.mul(cd.rd64[a], vm[0]);
            p.mul(cd.rd64[3 + a], vm[1]);
            p.mul(cd.rd64[6 + a], vm[2]);
            uc64[a] = p.result();
        }
    }
    const BD &d64 = uc64[2];
    {
        // S = d^2 and P = d up folded into R = mu S - P around a pixel centre
        // mu near the projected mean (see Rec)
        BD u0, u1;
        AD p;
        p.init(0.0, 0.0); p.term((double)fx, uc64[0]); p.term((double)cx, uc64[2]); u0 = p.result();
        p.init(0.0, 0.0); p.term((double)fy, uc64[1]); p.term((double)cy, uc64[2]); u1 = p.result();
        const BD S = sb_sqr<M, double>(d64);
        const BD Px = sb_mul<M, double>(d64, u0);
        const BD Py = sb_mul<M, double>(d64, u1);
        BD Rx, Ry;
        p.init(0.0, 0.0); p.term_same_side((double)mux, S); p.term(-1.0, Px); Rx = p.result();
        p.init(0.0, 0.0); p.term_same_side((double)muy, S); p.term(-1.0, Py); Ry = p.result();
        B S32, Rx32, Ry32;
        const double gap = sb_to_rec<M>(S, S32);
        sb_to_rec<M>(Rx, Rx32);
        sb_to_rec<M>(Ry, Ry32);
        ok = ok && sb_finite(S32) && sb_finite(Rx32) && sb_finite(Ry32);
        store_sb<M>(rec + RL::S, S32);
        store_sb<M>(rec + RL::RX, Rx32);
        store_sb<M>(rec + RL::RY, Ry32);
        rec_up(gap, rec[RL::GAP_S]);
    }
    BD Mp64[6];
    {
        BD Mc[9];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                AD p;
                p.init(0.0, 0.0);
                p.term(N[c], cd.rd64[a]);
                p.term(N[3 + c], cd.rd64[3 + a]);
                p.term(N[6 + c], cd.rd64[6 + a]);
                Mc[3 * a + c] = p.result();
            }
        BD J00, J02, J11, J12;
        AD p;
        p.init(0.0, 0.0); p.term((double)fx, d64); J00 = p.result();
        p.init(0.0, 0.0); p.term(-(double)fx, uc64[0]); J02 = p.result();
        p.init(0.0, 0.0); p.term((double)fy, d64); J11 = p.result();
        p.init(0.0, 0.0); p.term(-(double)fy, uc64[1]); J12 = p.result();
        for (int c = 0; c < 3; ++c) {
            p.init(0.0, 0.0); p.mul(J00, Mc[c]); p.mul(J02, Mc[6 + c]); Mp64[c] = p.result();
            p.init(0.0, 0.0); p.mul(J11, Mc[3 + c]); p.mul(J12, Mc[6 + c]); Mp64[3 + c] = p.result();
        }
    }
    // ---- MatrixInv (Algorithm 3) with the adaptive order and, where its
    // assertion fails on the cell, the input splitting of Sec. 3.1
    bool fallback = false;
    // Conic as FP64 forms (see matinv_box: the series in the record
    // precision, the assembly in FP64)
    SB<M, double> conic[4];
    {
        BD X[4];
        {
            AD p;
            p.init(0.0, 0.0); p.sqr(Mp64[0]); p.sqr(Mp64[1]); p.sqr(Mp64[2]); X[0] = p.result();
            p.init(0.0, 0.0); p.sqr(Mp64[3]); p.sqr(Mp64[4]); p.sqr(Mp64[5]); X[3] = p.result();
            p.init(0.0, 0.0); p.mul(Mp64[0], Mp64[3]); p.mul(Mp64[1], Mp64[4]); p.mul(Mp64[2], Mp64[5]); X[1] = p.result();
            X[2] = X[1];
        }
        if (SPLIT == SPLIT_WARP) {
            // a deferred pair (MatrixInv failed on its cell): the warp splits it
            if (matinv_split_warp<M, RO>(X, conic, split_list) > 0) flags |= F_SPLIT;
            else fallback = true;
        } else {
            // deferring: a pair whose order would exceed the default goes to a
            // pass of its own, so that warps do not wait on a few long series
            const int mi = matinv_box<M, RO, SPLIT == SPLIT_DEFER ? KTAYLOR : KMAX>(X, conic);
            if (SPLIT == SPLIT_DEFER && mi == MI_KHIGH) return flags | F_KHIGH_PENDING;
            if (mi == MI_FAIL) {
                if (SPLIT == SPLIT_DEFER) return flags | F_SPLIT_PENDING;
                if (matinv_split<M, RO>(X, conic) > 0) flags |= F_SPLIT;
                else fallback = true;
            }
        }
        if (!fallback)
            for (int e = 0; e < 4; ++e)
                if (!sb_finite(conic[e])) fallback = true;
    }
    if (!fallback) {
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                // W = Conic Mp in FP64
                AD p;
                p.init(0.0, 0.0);
                p.mul(conic[2 * r], Mp64[c]);
                p.mul(conic[2 * r + 1], Mp64[3 + c]);
                B w;
                sb_to_rec<M>(p.result(), w);
                if (!sb_finite(w)) fallback = true;
                store_sbw<M>(rec + RL::W0 + (3 * r + c) * RL::WS, w);
            }
    }
    if (!ok) fallback = true;
    if (fallback) flags |= F_FALLBACK;
    rec_put_flags(rec + RL::FLAGS, flags);
    return flags;
}

// grid: x over Gaussians, y over cells.  One thread per (Gaussian, cell).
// VALUE = false builds only the decision part (the value part is then built
// on demand by the renderer).
// counters: [0] pixel-Gaussian-cell triples in boxes, [1] MatrixInv
// fallbacks, [2] pairs present, [3] (pair, tile) entries, [4] pairs whose
// MatrixInv needed input splitting.
template <int M, class RO = float, bool VALUE = true>
// (five 128-thread blocks per SM: the FP64 chain needs warps to hide its
// latency more than registers; measured 9.41 -> 9.14 ms on 19M pairs, six
// blocks spill and lose)
__global__ void __launch_bounds__(128, 5) record_prep_kernel(
    const double *__restrict__ vN, const GParam *__restrict__ gp, CallConst cc,
    const CellData<M> *__restrict__ cells, int TS,
    RO *__restrict__ recs, PixBox *__restrict__ boxes, double *__restrict__ keys,
    unsigned long long *__restrict__ counters, int cells_fast)
{
    // cells_fast: the grid's x is the cell, so that the blocks of all cells
    // over one range of Gaussians run together and share that range's vN
    // rows in L2 (a scene's rows can exceed L2: 240 B per Gaussian)
    const int cell = cells_fast ? blockIdx.x : blockIdx.y;
    const int64_t g = (cells_fast ? blockIdx.y : blockIdx.x) * (int64_t)blockDim.x + threadIdx.x;
    PrepCount pc = {0, 0, 0, 0, 0};
    if (g < cc.n_gauss) {
        const int64_t fl = record_decide<M, RO>(vN, gp, cc, cells[cell], cell, g, TS, recs, boxes, keys, pc);
        if (VALUE && fl >= 0) {
            RO *rec = recs + ((int64_t)cell * cc.n_gauss + g) * Rec<M>::WIDTH;
            const uint32_t f = record_value<M, RO>(vN + VN_STRIDE * g, cc.fx, cc.fy, cc.cx, cc.cy, cells[cell], rec[Rec<M>::MU_X],
                                                   rec[Rec<M>::MU_Y], (uint32_t)fl, rec);
            pc.fallback = (f & F_FALLBACK) ? 1u : 0u;
            pc.split = (f & F_SPLIT) ? 1u : 0u;
        }
    }
    const uint32_t t = __reduce_add_sync(0xffffffffu, pc.triples);
    const uint32_t f = __reduce_add_sync(0xffffffffu, pc.fallback);
    const uint32_t v = __reduce_add_sync(0xffffffffu, pc.valid);
    const uint32_t e = __reduce_add_sync(0xffffffffu, pc.tiles);
    const uint32_t sp = __reduce_add_sync(0xffffffffu, pc.split);
    if ((threadIdx.x & 31) == 0) {
        if (t) atomicAdd(&counters[0], (unsigned long long)t);
        if (f) atomicAdd(&counters[1], (unsigned long long)f);
        if (v) atomicAdd(&counters[2], (unsigned long long)v);
        if (e) atomicAdd(&counters[3], (unsigned long long)e);
        if (sp) atomicAdd(&counters[4], (unsigned long long)sp);
    }
}

// The certain drops of the decision part, from FP32 enclosures (depth_fp32,
// screen_guard_fp32): a pair whose opacity stays below the cutoff, whose
// depth lies behind the near plane, or whose projected mean lies outside the
// frustum guard band over the whole cell gets an absent box and no record,
// as the FP64 chain would decide; the other pairs are listed (in no
// particular order) for record_prep_list_kernel, so that its warps run the
// FP64 chain on full warps of pairs that need it.
template <int M>
__global__ void __launch_bounds__(128) cull_kernel(const double *__restrict__ vN, const GParam *__restrict__ gp,
                                                   CallConst cc, const CellData<M> *__restrict__ cells,
                                                   PixBox *__restrict__ boxes, uint32_t *__restrict__ list,
                                                   uint32_t *__restrict__ count, int cells_fast)
{
    const int cell = cells_fast ? blockIdx.x : blockIdx.y;  // (see record_prep_kernel)
    const int64_t g = (cells_fast ? blockIdx.y : blockIdx.x) * (int64_t)blockDim.x + threadIdx.x;
    bool keep = false;
    const int64_t ri = (int64_t)cell * cc.n_gauss + g;
    if (g < cc.n_gauss) {
        boxes[ri] = PixBox{-1, -1, -1, -1};
        keep = gp[g].tau_hi >= 0;  // else o < 1/255: never above the cutoff
        if (keep) {
            const CellData<M> &cd = cells[cell];
            const float *enc = reinterpret_cast<const float *>(vN + VN_STRIDE * g + VN_ENC);
            bool ok = true;
            E32 el, eh;
            depth_fp32<M>(cd, enc, el, eh, ok);
            const float nearf = cc.near_plane;
            if (ok && eh.hi <= nearf) keep = false;  // d_hi <= near: behind the near plane
            if (ok && keep && eh.lo > nearf) {
                EI Ri[9], vs[3], ucx, ucy, mux, muy;
                screen_inputs_fp32(cd, enc, Ri, vs, ok);
                const EI D = {E32{fmaxf(el.lo, nearf), fmaxf(el.hi, nearf)}, eh};
                if (ok && screen_guard_fp32(cd, Ri, vs, D, cc, ucx, ucy, mux, muy, ok) == SCREEN_DROP) keep = false;
            }
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (m) {
        const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
        uint32_t at = 0;
        if (lane == leader) at = atomicAdd(count, (uint32_t)__popc(m));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (keep) list[at + __popc(m & ((1u << lane) - 1u))] = (uint32_t)ri;
    }
}

// record_prep_kernel over the pairs cull_kernel listed (grid-stride; the
// count is read on the device)
template <int M, class RO, bool VALUE>
__global__ void __launch_bounds__(128, 5) record_prep_list_kernel(
    const double *__restrict__ vN, const GParam *__restrict__ gp, CallConst cc,
    const CellData<M> *__restrict__ cells, int TS, RO *__restrict__ recs, PixBox *__restrict__ boxes,
    double *__restrict__ keys, unsigned long long *__restrict__ counters, const uint32_t *__restrict__ list,
    const uint32_t *__restrict__ count)
{
    const uint32_t n = *count;
    unsigned long long acc[5] = {0, 0, 0, 0, 0};  // a thread takes several pairs: 64-bit sums
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        if (i >= n) continue;
        const int64_t ri = list[i];
        const int cell = (int)(ri / cc.n_gauss);
        const int64_t g = ri - (int64_t)cell * cc.n_gauss;
        PrepCount pc = {0, 0, 0, 0, 0};
        const int64_t fl = record_decide<M, RO>(vN, gp, cc, cells[cell], cell, g, TS, recs, boxes, keys, pc);
        if (VALUE && fl >= 0) {
            RO *rec = recs + ri * Rec<M>::WIDTH;
            const uint32_t f = record_value<M, RO>(vN + VN_STRIDE * g, cc.fx, cc.fy, cc.cx, cc.cy, cells[cell],
                                                   rec[Rec<M>::MU_X], rec[Rec<M>::MU_Y], (uint32_t)fl, rec);
            pc.fallback = (f & F_FALLBACK) ? 1u : 0u;
            pc.split = (f & F_SPLIT) ? 1u : 0u;
        }
        acc[0] += pc.triples;
        acc[1] += pc.fallback;
        acc[2] += pc.valid;
        acc[3] += pc.tiles;
        acc[4] += pc.split;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
        for (int d = 16; d; d >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], d);
        if ((threadIdx.x & 31) == 0 && acc[k]) atomicAdd(&counters[k], acc[k]);
    }
}

// Builds the value part of the records listed in work[0, *count) (pair
// indices within the batch, cell * n_gauss + g), whose decision part the
// record kernel wrote.  Grid-stride over the list; the grid is sized on the
// host without knowing the count.
// counters: [0] MatrixInv fallbacks among the records built, [1] records
// built, [2] records whose MatrixInv needed input splitting.  A pair whose
// MatrixInv fails on its cell is appended to the front of list (split_count
// counts them) and finished by split_build_kernel; one whose Taylor order
// exceeds the default is appended to the back (list_cap - 1 downwards;
// khigh_count counts them) and finished by khigh_build_kernel.
template <int M>
__global__ void __launch_bounds__(128) record_build_kernel(
    const double *__restrict__ vN, float fx, float fy, float cx, float cy, const CellData<M> *__restrict__ cells,
    int64_t n_gauss, const uint32_t *__restrict__ work, const uint32_t *__restrict__ count, float *__restrict__ recs,
    unsigned long long *__restrict__ counters, uint32_t *__restrict__ split_list, uint32_t *__restrict__ split_count,
    uint32_t list_cap, uint32_t *__restrict__ khigh_count)
{
    using RL = Rec<M>;
    const uint32_t n = *count;
    uint32_t built = 0, fb = 0, sp = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t p = work[i];
        const int cell = (int)(p / (uint64_t)n_gauss);
        const int64_t g = (int64_t)p - (int64_t)cell * n_gauss;
        float *rec = recs + (size_t)p * RL::WIDTH;
        const uint32_t f = record_value<M, float, SPLIT_DEFER>(vN + VN_STRIDE * g, fx, fy, cx, cy, cells[cell],
                                                              rec[RL::MU_X], rec[RL::MU_Y],
                                                              __float_as_uint(rec[RL::FLAGS]), rec);
        if (f & F_SPLIT_PENDING) split_list[atomicAdd(split_count, 1u)] = p;
        if (f & F_KHIGH_PENDING) split_list[list_cap - 1u - atomicAdd(khigh_count, 1u)] = p;
        ++built;
        if (f & F_FALLBACK) ++fb;
        if (f & F_SPLIT) ++sp;
    }
    if (counters) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, fb);
        const uint32_t b = __reduce_add_sync(0xffffffffu, built);
        const uint32_t c = __reduce_add_sync(0xffffffffu, sp);
        if ((threadIdx.x & 31) == 0) {
            if (a) atomicAdd(&counters[0], (unsigned long long)a);
            if (b) atomicAdd(&counters[1], (unsigned long long)b);
            if (c) atomicAdd(&counters[2], (unsigned long long)c);
        }
    }
}

// Finishes the records of the pairs record_build_kernel deferred (list[0,
// *count)): one warp per pair, every lane running the value chain of the pair
// (the same values), the warp splitting its cell (SPLIT_WARP).  Grid-stride
// over the list by warps, pair i on block i mod gridDim.x first, so that a
// short list puts one pair on each SM instead of four on a few SMs sharing
// their FP64 pipes.  counters as in record_build_kernel ([0] fallbacks,
// [2] splits; the pairs were counted as built there).
template <int M>
__global__ void __launch_bounds__(128) split_build_kernel(
    const double *__restrict__ vN, float fx, float fy, float cx, float cy, const CellData<M> *__restrict__ cells,
    int64_t n_gauss, const uint32_t *__restrict__ list, const uint32_t *__restrict__ count, float *__restrict__ recs,
    unsigned long long *__restrict__ counters)
{
    using RL = Rec<M>;
    __shared__ uint64_t pieces[4][2 * 64];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t n = *count;
    uint32_t fb = 0, sp = 0;
    for (uint32_t i = (uint32_t)w * gridDim.x + blockIdx.x; i < n; i += gridDim.x * 4) {
        const uint32_t p = list[i];
        const int cell = (int)(p / (uint64_t)n_gauss);
        const int64_t g = (int64_t)p - (int64_t)cell * n_gauss;
        float *rec = recs + (size_t)p * RL::WIDTH;
        const uint32_t f0 = __float_as_uint(rec[RL::FLAGS]);
        __syncwarp();
        const uint32_t f = record_value<M, float, SPLIT_WARP>(vN + VN_STRIDE * g, fx, fy, cx, cy, cells[cell],
                                                             rec[RL::MU_X], rec[RL::MU_Y], f0, rec, pieces[w]);
        if (lane == 0) {
            if (f & F_FALLBACK) ++fb;
            if (f & F_SPLIT) ++sp;
        }
    }
    if (counters && lane == 0) {
        if (fb) atomicAdd(&counters[0], (unsigned long long)fb);
        if (sp) atomicAdd(&counters[2], (unsigned long long)sp);
    }
}

// Finishes the records of the pairs record_build_kernel deferred for their
// Taylor order (list[list_cap - 1 - i], i < *count): one thread per pair, as
// record_build_kernel without deferral.  counters as there ([0], [2]).
template <int M>
__global__ void __launch_bounds__(128) khigh_build_kernel(
    const double *__restrict__ vN, float fx, float fy, float cx, float cy, const CellData<M> *__restrict__ cells,
    int64_t n_gauss, const uint32_t *__restrict__ list, uint32_t list_cap, const uint32_t *__restrict__ count,
    float *__restrict__ recs, unsigned long long *__restrict__ counters)
{
    using RL = Rec<M>;
    const uint32_t n = *count;
    uint32_t fb = 0, sp = 0;
    // pair i on block i mod gridDim.x first (a short list spreads over the SMs)
    for (uint32_t i = threadIdx.x * gridDim.x + blockIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t p = list[list_cap - 1u - i];
        const int cell = (int)(p / (uint64_t)n_gauss);
        const int64_t g = (int64_t)p - (int64_t)cell * n_gauss;
        float *rec = recs + (size_t)p * RL::WIDTH;
        const uint32_t f = record_value<M, float>(vN + VN_STRIDE * g, fx, fy, cx, cy, cells[cell], rec[RL::MU_X],
                                                  rec[RL::MU_Y], __float_as_uint(rec[RL::FLAGS]), rec);
        if (f & F_FALLBACK) ++fb;
        if (f & F_SPLIT) ++sp;
    }
    if (counters) {
        const uint32_t a = __reduce_add_sync(0xffffffffu, fb);
        const uint32_t c = __reduce_add_sync(0xffffffffu, sp);
        if ((threadIdx.x & 31) == 0) {
            if (a) atomicAdd(&counters[0], (unsigned long long)a);
            if (c) atomicAdd(&counters[2], (unsigned long long)c);
        }
    }
}

}  // namespace ar
