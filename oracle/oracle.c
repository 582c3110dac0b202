/*
 * FP64 CPU oracle for abstract rendering of Gaussian-splat scenes
 * (Li, Ji, Zhong, Zhang, Mitra, "Abstract Rendering: Computing All that is Seen
 * in Gaussian Splat Scenes", arXiv 2503.00308).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, double-precision
 * statement of what the CUDA path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header or table with the CUDA library; the two meet only through the seeded
 * input generator.
 *
 * Everything is straight loops in the order of the paper's algorithms:
 *   - GSplat, Algorithm 1 (Sec. 2.2), with either blend:
 *       BlendSort, Algorithm 2 (depth sort + cumulative product), and
 *       BlendInd,  Algorithm 4 (pairwise Ind, O(N^2)).
 *   - AbstractSplat (Sec. 3.3): Algorithm 1 with every variable replaced by a
 *     pair of linear bounds over the pose cell, Conic replaced by MatrixInv
 *     (Algorithm 3, Sec. 3.1) and BlendSort by BlendInd (Sec. 3.2).
 *
 * Linear bounds.  A pose cell is a box over delta = (tx,ty,tz,rx,ry,rz); each
 * coordinate is written delta_k = ctr_k + h_k * p_k with p in [-1,1]^6.  A
 * "bounded scalar" is a pair of affine forms lo(p) <= v <= hi(p), the
 * piecewise-linear relation of Sec. 2.1 with a single piece.  Concretising a
 * form over the box gives  k - sum|c|  (lower) or  k + sum|c|  (upper).
 *
 * Relaxations the paper delegates to CROWN and does not print are fixed here
 * (each is a sound choice; all collapse to the exact value on a point cell):
 *   Mul x*y    : average of the two McCormick planes of each side.
 *   Square x^2 : tangent at the interval midpoint (lower), secant (upper).
 *   Exp        : Table 2 -- tangent at the lower end, secant (upper), on
 *                [x_lo, min(x_hi, 0)] because x = -m/2 <= 0.
 *   R(theta)   : first-order Taylor form at the cell centre, remainder
 *                +-(1/2)(h_rx+h_ry+h_rz)^2 (every second partial of an entry of
 *                Rx Ry Rz has magnitude <= 1).
 *   Ind        : three-valued from depth-key intervals (Table 2 Ind, split at 0).
 *   Prod       : interval transmittance products; colour sums kept as forms.
 *   Cutoff     : a = 0 where o*exp(-m/2) < 1/255, relaxed soundly with ramps
 *                whose width shrinks to zero with the cell.
 *
 * Parity of the "tightness" of these choices against the paper's CROWN numbers
 * is unpinned (the paper's scenes are not available); their soundness and their
 * exactness on point cells are pinned by the test-suite.  The values of each
 * relaxation are pinned by hand-worked closed forms: Mul, Square and Exp one
 * by one (bs_mul, bs_sq, bs_exp), the opacity stage with its clip and cutoff
 * ramps (alpha_from_m) in every branch, and one Gaussian's whole pixel chain
 * on a case whose Mahalanobis term has a closed form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 6            /* pose variables tx ty tz rx ry rz */
#define KTAYLOR 8       /* MatrixInv Taylor order, default k = 8 (Sec. 3.3 footnote) */
#define KMAX 24         /* adjustment (3) of Sec. 3.1: k grows from KTAYLOR up to KMAX */
#define SPLIT_DEPTH 6   /* adjustment (2) of Sec. 3.1: at most 6 bisections of a pose cell */

/* Algorithm constants shared by definition with the CUDA path (not by code). */
static const double RHO_MAX = 1.0 - 1.0 / 1024.0;  /* MatrixInv usable while ||I-X X0|| < RHO_MAX */
static const double CUT_RAMP = 0.5;   /* widest cutoff ramp, in units of m */
static const double CLIP_RAMP = 0.25; /* blend width of the upper-alpha clip to o */
static const double KEY_SLACK = 1e-9; /* relative widening of depth keys */
static const double GUARD = 0.65;     /* guard band: 1.3 x the half-extent, as a fraction of W and H */
static const double BOX_SLACK = 1e-9; /* relative widening of screen boxes */
static const double ALPHA_MIN = 1.0 / 255.0;
static const double EPS_TOL = 5.9604644775390625e-8;  /* 2^-24: k grows until Eps <= EPS_TOL ||X0||_F */

typedef struct { double c[NV]; double k; } lf;   /* sum_i c_i p_i + k */
typedef struct { lf lo, hi; } bs;                 /* lo(p) <= v <= hi(p) */

/* ------------------------------------------------------------------ forms */

static double lf_min(const lf *f) { double s = f->k; for (int i = 0; i < NV; ++i) s -= fabs(f->c[i]); return s; }
static double lf_max(const lf *f) { double s = f->k; for (int i = 0; i < NV; ++i) s += fabs(f->c[i]); return s; }
static double bs_min(const bs *b) { return lf_min(&b->lo); }
static double bs_max(const bs *b) { return lf_max(&b->hi); }

static lf lf_cst(double v) { lf f; memset(&f, 0, sizeof f); f.k = v; return f; }
static lf lf_scale(const lf *a, double s) { lf r; for (int i = 0; i < NV; ++i) r.c[i] = s * a->c[i]; r.k = s * a->k; return r; }
static lf lf_add(const lf *a, const lf *b) { lf r; for (int i = 0; i < NV; ++i) r.c[i] = a->c[i] + b->c[i]; r.k = a->k + b->k; return r; }
static lf lf_sub(const lf *a, const lf *b) { lf r; for (int i = 0; i < NV; ++i) r.c[i] = a->c[i] - b->c[i]; r.k = a->k - b->k; return r; }

static bs bs_cst(double v) { bs b; b.lo = lf_cst(v); b.hi = lf_cst(v); return b; }
static bs bs_add(bs a, bs b) { bs r; r.lo = lf_add(&a.lo, &b.lo); r.hi = lf_add(&a.hi, &b.hi); return r; }
static bs bs_sub(bs a, bs b) { bs r; r.lo = lf_sub(&a.lo, &b.hi); r.hi = lf_sub(&a.hi, &b.lo); return r; }
static bs bs_addc(bs a, double v) { a.lo.k += v; a.hi.k += v; return a; }
/* constant * bounded scalar: a negative factor swaps the sides */
static bs bs_scale(bs a, double s)
{
    bs r;
    if (s >= 0) { r.lo = lf_scale(&a.lo, s); r.hi = lf_scale(&a.hi, s); }
    else        { r.lo = lf_scale(&a.hi, s); r.hi = lf_scale(&a.lo, s); }
    return r;
}

/* x*y: the lower planes y_lo x + x_lo y - x_lo y_lo and y_hi x + x_hi y - x_hi y_hi
 * averaged give  y_m x + x_m y - (x_lo y_lo + x_hi y_hi)/2 <= x y ; the upper
 * planes averaged give  y_m x + x_m y - (x_hi y_lo + x_lo y_hi)/2 >= x y, with
 * x_m, y_m the interval midpoints.  x and y are then replaced by the side of
 * their bounds that keeps the inequality (the sign of the slope decides). */
static bs bs_mul(bs x, bs y)
{
    double xl = bs_min(&x), xh = bs_max(&x), yl = bs_min(&y), yh = bs_max(&y);
    double xm = 0.5 * (xl + xh), ym = 0.5 * (yl + yh);
    bs r;
    lf a, b;
    a = lf_scale(ym >= 0 ? &x.lo : &x.hi, ym);
    b = lf_scale(xm >= 0 ? &y.lo : &y.hi, xm);
    r.lo = lf_add(&a, &b);
    r.lo.k -= 0.5 * (xl * yl + xh * yh);
    a = lf_scale(ym >= 0 ? &x.hi : &x.lo, ym);
    b = lf_scale(xm >= 0 ? &y.hi : &y.lo, xm);
    r.hi = lf_add(&a, &b);
    r.hi.k -= 0.5 * (xh * yl + xl * yh);
    return r;
}

/* x^2: tangent at the midpoint c (2c x - c^2) below, secant (xl+xh) x - xl xh above. */
static bs bs_sq(bs x)
{
    double xl = bs_min(&x), xh = bs_max(&x), c = 0.5 * (xl + xh), s = xl + xh;
    bs r;
    r.lo = lf_scale(c >= 0 ? &x.lo : &x.hi, 2.0 * c);
    r.lo.k -= c * c;
    r.hi = lf_scale(s >= 0 ? &x.hi : &x.lo, s);
    r.hi.k -= xl * xh;
    return r;
}

/* -------------------------------------------------------- scene and pose */

/* rotation of a unit quaternion (w,x,y,z) */
static void quat_to_R(const double q_in[4], double R[9])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void mat3_mul(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

/* Rx(a), Ry(b), Rz(g) and their first derivatives */
static void rot_x(double a, double R[9], double D[9])
{
    double c = cos(a), s = sin(a);
    double r[9] = {1, 0, 0, 0, c, -s, 0, s, c}, d[9] = {0, 0, 0, 0, -s, -c, 0, c, -s};
    memcpy(R, r, sizeof r); memcpy(D, d, sizeof d);
}
static void rot_y(double b, double R[9], double D[9])
{
    double c = cos(b), s = sin(b);
    double r[9] = {c, 0, s, 0, 1, 0, -s, 0, c}, d[9] = {-s, 0, c, 0, 0, 0, -c, 0, -s};
    memcpy(R, r, sizeof r); memcpy(D, d, sizeof d);
}
static void rot_z(double g, double R[9], double D[9])
{
    double c = cos(g), s = sin(g);
    double r[9] = {c, -s, 0, s, c, 0, 0, 0, 1}, d[9] = {-s, -c, 0, c, -s, 0, 0, 0, 0};
    memcpy(R, r, sizeof r); memcpy(D, d, sizeof d);
}

/* camera-frame perturbation R_delta = Rx(rx) Ry(ry) Rz(rz); optionally its partials */
static void rot_delta(const double th[3], double R[9], double dR[3][9])
{
    double X[9], dX[9], Y[9], dY[9], Z[9], dZ[9], T[9];
    rot_x(th[0], X, dX); rot_y(th[1], Y, dY); rot_z(th[2], Z, dZ);
    mat3_mul(X, Y, T); mat3_mul(T, Z, R);
    if (dR) {
        mat3_mul(dX, Y, T); mat3_mul(T, Z, dR[0]);
        mat3_mul(X, dY, T); mat3_mul(T, Z, dR[1]);
        mat3_mul(X, Y, T);  mat3_mul(T, dZ, dR[2]);
    }
}

typedef struct {
    int W, H;
    double fx, fy, cx, cy, near_plane;
    double R0[9];   /* nominal world->camera rotation */
    double t0[3];   /* nominal camera centre */
} camera;

static camera make_camera(const double *intr, const double *R0, const double *t0)
{
    camera c;
    c.W = (int)intr[0]; c.H = (int)intr[1];
    c.fx = intr[2]; c.fy = intr[3]; c.cx = intr[4]; c.cy = intr[5]; c.near_plane = intr[6];
    memcpy(c.R0, R0, sizeof c.R0); memcpy(c.t0, t0, sizeof c.t0);
    return c;
}

/* covariance factor Mw = R(q) diag(exp(s)) (the footnote of Sec. 2.2 allows any
 * square-root factor: Cov = Mw Mw^T) */
static void cov_factor(const double *ls, const double *q, double Mw[9])
{
    double R[9];
    quat_to_R(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mw[3 * i + j] = R[3 * i + j] * exp(ls[j]);
}

/* ============================================================ GSplat ===== */

/* Per-Gaussian quantities of Algorithm 1 at one concrete pose. */
typedef struct {
    double d, up[2], Mp[6], conic[4], o, tau, c[3];
    int alive;
} gconc;

static void gsplat_gaussian(const camera *cam, const double Rwc[9], const double t[3],
                            const double *uw, const double *ls, const double *q, double o,
                            const double *rgb, gconc *g)
{
    double Mw[9], Mc[9], uc[3], diff[3];
    cov_factor(ls, q, Mw);
    for (int a = 0; a < 3; ++a) diff[a] = uw[a] - t[a];
    for (int a = 0; a < 3; ++a) uc[a] = Rwc[3 * a] * diff[0] + Rwc[3 * a + 1] * diff[1] + Rwc[3 * a + 2] * diff[2];
    mat3_mul(Rwc, Mw, Mc);
    g->d = uc[2];
    g->up[0] = cam->fx * uc[0] + cam->cx * uc[2];
    g->up[1] = cam->fy * uc[1] + cam->cy * uc[2];
    /* J of Algorithm 1 (the usual projection Jacobian scaled by d^2) */
    double J[6] = {cam->fx * uc[2], 0, -cam->fx * uc[0], 0, cam->fy * uc[2], -cam->fy * uc[1]};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            g->Mp[3 * r + c] = J[3 * r] * Mc[c] + J[3 * r + 1] * Mc[3 + c] + J[3 * r + 2] * Mc[6 + c];
    double X[4];
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s)
            X[2 * r + s] = g->Mp[3 * r] * g->Mp[3 * s] + g->Mp[3 * r + 1] * g->Mp[3 * s + 1] + g->Mp[3 * r + 2] * g->Mp[3 * s + 2];
    double det = X[0] * X[3] - X[1] * X[2];
    g->conic[0] = X[3] / det; g->conic[1] = -X[1] / det; g->conic[2] = -X[2] / det; g->conic[3] = X[0] / det;
    g->o = o;
    g->tau = (o > 0) ? 2.0 * log(255.0 * o) : -INFINITY;
    for (int k = 0; k < 3; ++k) g->c[k] = rgb[k];
    g->alive = (g->d > cam->near_plane) && (det > 0) && (o > 0);
    if (g->alive) {
        /* frustum guard band (3DGS convention): the projected mean must lie
         * within 1.3 times the image half-extent around the principal point */
        const double gx = GUARD * cam->W, gy = GUARD * cam->H;
        const double u = cam->cx + cam->fx * uc[0] / uc[2], w = cam->cy + cam->fy * uc[1] / uc[2];
        g->alive = (u >= cam->cx - gx) && (u <= cam->cx + gx) && (w >= cam->cy - gy) && (w <= cam->cy + gy);
    }
}

/* effective opacity at pixel u (Algorithm 1, lines 9-10) with the 1/255 cutoff */
static double gsplat_alpha(const gconc *g, double ux, double uy)
{
    if (!g->alive) return 0.0;
    double D[2] = {g->d * g->d * ux - g->d * g->up[0], g->d * g->d * uy - g->d * g->up[1]};
    double q[3], m = 0;
    for (int c = 0; c < 3; ++c) {
        double w0 = g->conic[0] * g->Mp[c] + g->conic[1] * g->Mp[3 + c];
        double w1 = g->conic[2] * g->Mp[c] + g->conic[3] * g->Mp[3 + c];
        q[c] = D[0] * w0 + D[1] * w1;
        m += q[c] * q[c];
    }
    if (m > g->tau) return 0.0;
    return g->o * exp(-0.5 * m);
}

static void pose_camera(const camera *cam, const double *delta, double Rwc[9], double t[3])
{
    double Rd[9], RdT[9];
    rot_delta(delta + 3, Rd, NULL);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RdT[3 * i + j] = Rd[3 * j + i];
    mat3_mul(RdT, cam->R0, Rwc);
    for (int k = 0; k < 3; ++k) t[k] = cam->t0[k] + delta[k];
}

typedef struct { double key; int idx; } keyidx;
static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *x = a, *y = b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return x->idx - y->idx;
}

/* Concrete render of the whole image at one pose.  blend = 0: BlendSort
 * (Algorithm 2); blend = 1: BlendInd (Algorithm 4).  out is [H][W][3]. */
int orc_render_concrete(const double *uw, const double *ls, const double *quat, const double *opac,
                        const double *rgb, int64_t n, const double *intr, const double *R0,
                        const double *t0, const double *delta, int blend, double *out)
{
    camera cam = make_camera(intr, R0, t0);
    double Rwc[9], t[3];
    pose_camera(&cam, delta, Rwc, t);
    gconc *G = (gconc *)malloc(sizeof(gconc) * (size_t)(n > 0 ? n : 1));
    double *a = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    keyidx *order = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    if (!G || !a || !order) { free(G); free(a); free(order); return 1; }
    for (int64_t i = 0; i < n; ++i)
        gsplat_gaussian(&cam, Rwc, t, uw + 3 * i, ls + 3 * i, quat + 4 * i, opac[i], rgb + 3 * i, &G[i]);
    for (int64_t i = 0; i < n; ++i) { order[i].key = G[i].d; order[i].idx = (int)i; }
    qsort(order, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int py = 0; py < cam.H; ++py)
        for (int px = 0; px < cam.W; ++px) {
            double ux = px + 0.5, uy = py + 0.5, pc[3] = {0, 0, 0};
            for (int64_t i = 0; i < n; ++i) a[i] = gsplat_alpha(&G[i], ux, uy);
            if (blend == 0) {
                /* BlendSort: as, cs sorted by depth; Ts = cumulative product of (1 - as) */
                double Ts = 1.0;
                for (int64_t r = 0; r < n; ++r) {
                    int i = order[r].idx;
                    for (int ch = 0; ch < 3; ++ch) pc[ch] += Ts * a[i] * G[i].c[ch];
                    Ts *= 1.0 - a[i];
                }
            } else {
                /* BlendInd: V[i][j] = 1 - a[j] Ind(d[i] - d[j]); T[i] = prod_j V[i][j] */
                for (int64_t i = 0; i < n; ++i) {
                    if (a[i] == 0.0) continue;
                    double T = 1.0;
                    for (int64_t j = 0; j < n; ++j)
                        if (G[i].d - G[j].d > 0) T *= 1.0 - a[j];
                    for (int ch = 0; ch < 3; ++ch) pc[ch] += T * a[i] * G[i].c[ch];
                }
            }
            double *o = out + 3 * ((size_t)py * cam.W + px);
            for (int ch = 0; ch < 3; ++ch) o[ch] = pc[ch] < 0 ? 0 : (pc[ch] > 1 ? 1 : pc[ch]);
        }
    free(G); free(a); free(order);
    return 0;
}

/* The concrete effective opacity of one Gaussian at one pixel and pose (for tests). */
double orc_concrete_alpha(const double *uw, const double *ls, const double *quat, double opac,
                          const double *intr, const double *R0, const double *t0, const double *delta,
                          double ux, double uy)
{
    camera cam = make_camera(intr, R0, t0);
    double Rwc[9], t[3], rgb[3] = {0, 0, 0};
    gconc g;
    pose_camera(&cam, delta, Rwc, t);
    gsplat_gaussian(&cam, Rwc, t, uw, ls, quat, opac, rgb, &g);
    return gsplat_alpha(&g, ux, uy);
}

/* ====================================================== AbstractSplat ===== */

typedef struct {
    double ctr[NV], h[NV];
    bs Rd[9];      /* R_delta entries as forms over the rotation variables */
    bs s[3];       /* s = R0 * delta_t (exact) */
    double Rc[9];  /* R_delta at the cell centre */
} cellforms;

/* Pose linearisation of one cell. */
static void cell_setup(const camera *cam, const double *lo, const double *hi, cellforms *cf)
{
    for (int k = 0; k < NV; ++k) { cf->ctr[k] = 0.5 * (lo[k] + hi[k]); cf->h[k] = 0.5 * (hi[k] - lo[k]); }
    double R[9], dR[3][9];
    rot_delta(cf->ctr + 3, R, dR);
    memcpy(cf->Rc, R, sizeof R);
    double hs = cf->h[3] + cf->h[4] + cf->h[5];
    double rem = 0.5 * hs * hs;
    for (int e = 0; e < 9; ++e) {
        lf f = lf_cst(R[e]);
        for (int k = 0; k < 3; ++k) f.c[3 + k] = dR[k][e] * cf->h[3 + k];
        cf->Rd[e].lo = f; cf->Rd[e].lo.k -= rem;
        cf->Rd[e].hi = f; cf->Rd[e].hi.k += rem;
    }
    for (int a = 0; a < 3; ++a) {
        lf f = lf_cst(0);
        for (int k = 0; k < 3; ++k) { f.c[k] = cam->R0[3 * a + k] * cf->h[k]; f.k += cam->R0[3 * a + k] * cf->ctr[k]; }
        cf->s[a].lo = f; cf->s[a].hi = f;
    }
}

void orc_rot_forms(const double *lo, const double *hi, double *out /* 9 x (lo[7], hi[7]) */)
{
    camera cam; memset(&cam, 0, sizeof cam); cam.R0[0] = cam.R0[4] = cam.R0[8] = 1;
    cellforms cf;
    cell_setup(&cam, lo, hi, &cf);
    for (int e = 0; e < 9; ++e) {
        for (int i = 0; i < NV; ++i) { out[14 * e + i] = cf.Rd[e].lo.c[i]; out[14 * e + 7 + i] = cf.Rd[e].hi.c[i]; }
        out[14 * e + 6] = cf.Rd[e].lo.k; out[14 * e + 13] = cf.Rd[e].hi.k;
    }
}

/* MatrixInv (Algorithm 3) on a 2x2 matrix of bounded scalars.  Returns 0 and
 * fills conic on success, 1 when the reference matrix is not positive
 * definite or ||I - X X0|| >= RHO_MAX (the assertion of Algorithm 3 fails).
 * k > 0 fixes the Taylor order; k <= 0 applies adjustment (3) of Sec. 3.1:
 * starting from the default KTAYLOR, k grows while the remainder bound Eps
 * exceeds EPS_TOL ||X0||_F, up to KMAX.  The order used goes to *k_out. */
static int matrix_inv(const bs X[4], int k, bs conic[4], double *rho_out, int *k_out)
{
    double Xh[4];
    for (int e = 0; e < 4; ++e) Xh[e] = 0.5 * (bs_min(&X[e]) + bs_max(&X[e]));
    double det = Xh[0] * Xh[3] - Xh[1] * Xh[2];
    if (rho_out) *rho_out = INFINITY;
    if (!(det > 0) || !(Xh[0] > 0)) return 1;
    /* X0 = inverse of the centre matrix (Sec. 3.1, adjustment (1)) */
    double X0[4] = {Xh[3] / det, -Xh[1] / det, -Xh[2] / det, Xh[0] / det};
    /* IXX0 = I - X X0 : X0 is constant, so this is an exact linear map */
    bs E[4];
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            bs v = bs_add(bs_scale(X[2 * r], X0[s]), bs_scale(X[2 * r + 1], X0[2 + s]));
            E[2 * r + s] = bs_addc(bs_scale(v, -1.0), r == s ? 1.0 : 0.0);
        }
    /* Norm(IXX0): Frobenius norm of the entrywise magnitude bound over the cell */
    double rho2 = 0;
    for (int e = 0; e < 4; ++e) {
        double m = fmax(fabs(bs_min(&E[e])), fabs(bs_max(&E[e])));
        rho2 += m * m;
    }
    double rho = sqrt(rho2);
    if (rho_out) *rho_out = rho;
    if (!(rho < RHO_MAX)) return 1;
    /* Eps / ||X0|| = rho^(k+1) / (1 - rho) decides the adaptive order */
    if (k <= 0) {
        k = KTAYLOR;
        while (k < KMAX && pow(rho, k + 1) / (1.0 - rho) > EPS_TOL) ++k;
    }
    if (k_out) *k_out = k;
    /* Sum_{i=0..k} Pow(IXX0, i) with Pow evaluated left to right */
    bs P[4], S[4];
    for (int e = 0; e < 4; ++e) { P[e] = E[e]; S[e] = bs_addc(E[e], (e == 0 || e == 3) ? 1.0 : 0.0); }
    for (int i = 2; i <= k; ++i) {
        bs Q[4];
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s)
                Q[2 * r + s] = bs_add(bs_mul(P[2 * r], E[s]), bs_mul(P[2 * r + 1], E[2 + s]));
        for (int e = 0; e < 4; ++e) { P[e] = Q[e]; S[e] = bs_add(S[e], Q[e]); }
    }
    /* Xp = X0 * Sum (X0 constant) and the remainder bound Eps */
    double nX0 = sqrt(X0[0] * X0[0] + X0[1] * X0[1] + X0[2] * X0[2] + X0[3] * X0[3]);
    double eps = nX0 * pow(rho, k + 1) / (1.0 - rho);
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            bs v = bs_add(bs_scale(S[s], X0[2 * r]), bs_scale(S[2 + s], X0[2 * r + 1]));
            v.lo.k -= eps; v.hi.k += eps;
            conic[2 * r + s] = v;
        }
    return 0;
}

/* Interval forms of a 2x2 matrix whose entries are independent: entry e =
 * mid_e + half_e * p_e (symmetric != 0: entries 1 and 2 are the same
 * variable p_1, so Xl/Xu must agree there). */
static void interval_forms(const double *Xl, const double *Xu, int symmetric, bs X[4])
{
    for (int e = 0; e < 4; ++e) {
        lf f = lf_cst(0.5 * (Xl[e] + Xu[e]));
        f.c[(symmetric && e == 2) ? 1 : e] = 0.5 * (Xu[e] - Xl[e]);
        X[e].lo = f; X[e].hi = f;
    }
}

/* A form over the cell restricted to the sub-box p = ctr + h p' (p' in
 * [-1,1]^NV), written over p'. */
static lf lf_restrict(const lf *f, const double ctr[NV], const double h[NV])
{
    lf r;
    r.k = f->k;
    for (int i = 0; i < NV; ++i) { r.c[i] = f->c[i] * h[i]; r.k += f->c[i] * ctr[i]; }
    return r;
}

/* The pose variable along which a piece is bisected: the one on which X
 * varies most there, i.e. the largest sum over X00, X01, X11 of the larger
 * |coefficient| of the two sides (the first such variable on a tie). */
static int split_var(const bs Xr[4])
{
    int js = 0;
    double best = -1.0;
    for (int j = 0; j < NV; ++j) {
        double v = 0;
        for (int e = 0; e < 4; ++e) {
            if (e == 2) continue;  /* X10 = X01 */
            v += fmax(fabs(Xr[e].lo.c[j]), fabs(Xr[e].hi.c[j]));
        }
        if (v > best) { best = v; js = j; }
    }
    return js;
}

typedef struct {
    double lo[4], hi[4];  /* hull of the pieces' concretised outputs */
    int pieces;           /* pieces MatrixInv succeeded on */
    int kmax;             /* largest Taylor order used */
    double margin;        /* smallest |rho - RHO_MAX| over the boxes tried */
} splitacc;

/* Adjustment (2) of Sec. 3.1: divide the input range until the assertion of
 * Algorithm 3 holds.  The linear bounds of X are taken on the piece p = ctr
 * + h p' of the pose cell (depth bisections deep) and MatrixInv runs there;
 * a piece on which the assertion fails is bisected along split_var, the
 * lower half first, down to SPLIT_DEPTH bisections.  The pieces' outputs are
 * forms over different boxes, so they are joined as constants: the least
 * lower and the greatest upper concretised bound of each entry.  Returns 1 if
 * a piece at the depth limit still fails. */
static int matinv_split(const bs X[4], const double ctr[NV], const double h[NV], int depth, splitacc *a)
{
    bs Xr[4], C[4];
    for (int e = 0; e < 4; ++e) {
        Xr[e].lo = lf_restrict(&X[e].lo, ctr, h);
        Xr[e].hi = lf_restrict(&X[e].hi, ctr, h);
    }
    double rho;
    int k = 0;
    const int st = matrix_inv(Xr, 0, C, &rho, &k);
    a->margin = fmin(a->margin, fabs(rho - RHO_MAX));
    if (st == 0) {
        for (int e = 0; e < 4; ++e) { a->lo[e] = fmin(a->lo[e], bs_min(&C[e])); a->hi[e] = fmax(a->hi[e], bs_max(&C[e])); }
        ++a->pieces;
        if (k > a->kmax) a->kmax = k;
        return 0;
    }
    if (depth >= SPLIT_DEPTH) return 1;
    const int js = split_var(Xr);
    double c2[NV], h2[NV];
    memcpy(c2, ctr, sizeof c2);
    memcpy(h2, h, sizeof h2);
    h2[js] = 0.5 * h[js];
    c2[js] = ctr[js] - h2[js];
    if (matinv_split(X, c2, h2, depth + 1, a)) return 1;
    c2[js] = ctr[js] + h2[js];
    return matinv_split(X, c2, h2, depth + 1, a);
}

/* MatrixInv over the whole cell (adaptive order); where its assertion fails,
 * MatrixInv with input splitting (matinv_split from the whole cell), conic
 * then holding constant forms.  Returns 1 when even the split fails (the R5
 * fallback).  *pieces is 0 when no split was needed. */
static int matrix_inv_cell(const bs X[4], bs conic[4], double *rho, int *korder, int *pieces, double *margin)
{
    *pieces = 0;
    *korder = 0;
    const int st = matrix_inv(X, 0, conic, rho, korder);
    *margin = fabs(*rho - RHO_MAX);
    if (st == 0) return 0;
    splitacc a;
    for (int e = 0; e < 4; ++e) { a.lo[e] = INFINITY; a.hi[e] = -INFINITY; }
    a.pieces = 0;
    a.kmax = 0;
    a.margin = *margin;
    double ctr[NV], h[NV];
    for (int j = 0; j < NV; ++j) { ctr[j] = 0.0; h[j] = 1.0; }
    const int fail = matinv_split(X, ctr, h, 0, &a);
    *margin = a.margin;
    if (fail) return 1;
    for (int e = 0; e < 4; ++e) { conic[e].lo = lf_cst(a.lo[e]); conic[e].hi = lf_cst(a.hi[e]); }
    *pieces = a.pieces;
    *korder = a.kmax;
    return 0;
}

/* Interval-matrix entry points for the pins (entries as in interval_forms).
 * They return the concretised bounds of MatrixInv's output.
 * orc_matrixinv_interval: MatrixInv on the whole box, order k (k <= 0: the
 * adaptive order); returns 1 where the assertion fails.
 * orc_matrixinv_cell: the pipeline's MatrixInv (adaptive order, input
 * splitting where the assertion fails) on a symmetric box; info gets the
 * pieces (0: no split), the Taylor order and rho on the whole box; returns 1
 * if the split fails, 2 if the box is not symmetric. */
int orc_matrixinv_interval(const double *Xl, const double *Xu, int k, int symmetric,
                           double *out_l, double *out_u, double *rho)
{
    bs X[4], C[4];
    interval_forms(Xl, Xu, symmetric, X);
    int st = matrix_inv(X, k, C, rho, NULL);
    if (st) return st;
    for (int e = 0; e < 4; ++e) { out_l[e] = bs_min(&C[e]); out_u[e] = bs_max(&C[e]); }
    return 0;
}

int orc_matrixinv_cell(const double *Xl, const double *Xu, int symmetric, double *out_l, double *out_u,
                       double *info)
{
    bs X[4], C[4];
    if (Xl[1] != Xl[2] || Xu[1] != Xu[2]) return 2;  /* the split works on symmetric boxes */
    interval_forms(Xl, Xu, symmetric, X);
    double rho, margin;
    int korder, pieces;
    int st = matrix_inv_cell(X, C, &rho, &korder, &pieces, &margin);
    info[0] = pieces; info[1] = korder; info[2] = rho;
    if (st) return st;
    for (int e = 0; e < 4; ++e) { out_l[e] = bs_min(&C[e]); out_u[e] = bs_max(&C[e]); }
    return 0;
}

/* Primitive relaxations on raw forms, for the pins.  Each form is 7 doubles
 * (6 coefficients, then the constant); a bounded scalar is lo form, hi form. */
static bs unpack_bs(const double *v)
{
    bs b;
    for (int i = 0; i < NV; ++i) { b.lo.c[i] = v[i]; b.hi.c[i] = v[7 + i]; }
    b.lo.k = v[6]; b.hi.k = v[13];
    return b;
}
static void pack_bs(const bs *b, double *v)
{
    for (int i = 0; i < NV; ++i) { v[i] = b->lo.c[i]; v[7 + i] = b->hi.c[i]; }
    v[6] = b->lo.k; v[13] = b->hi.k;
}
void orc_relax_mul(const double *x, const double *y, double *out) { bs r = bs_mul(unpack_bs(x), unpack_bs(y)); pack_bs(&r, out); }
void orc_relax_sq(const double *x, double *out) { bs r = bs_sq(unpack_bs(x)); pack_bs(&r, out); }
static bs bs_exp(bs x);
void orc_relax_exp(const double *x, double *out) { bs r = bs_exp(unpack_bs(x)); pack_bs(&r, out); }

/* Per-(Gaussian, cell) record of the abstract pipeline (steps of Algorithm 1
 * up to W = Conic * Mp). */
typedef struct {
    int valid;          /* contributes somewhere in the image */
    int straddle;       /* depth interval straddles the near plane */
    int fallback;       /* MatrixInv failed even with input splitting: a in [0, o] on the box */
    double rho;         /* ||I - X X0|| bound on the whole cell (INFINITY if X0 undefined) */
    int pieces;         /* pieces of the input split (0: MatrixInv held on the whole cell) */
    int korder;         /* Taylor order used (the largest over the pieces) */
    double rho_margin;  /* smallest |rho - RHO_MAX| over the boxes MatrixInv was tried on */
    double klo, khi;    /* depth-key interval */
    int px0, px1, py0, py1;  /* pixel box whose centres may see the Gaussian */
    bs S, Px, Py;       /* S = d^2, P = d * up */
    bs W[6];            /* W = Conic * Mp, row-major 2x3 */
    /* scene parameters as boxes (Sec. 4.5; lo = hi without boxes): opacity,
     * its cutoff exponent tau = 2 ln(255 o) at both ends, colour */
    double o_lo, o_hi, tau_lo, tau_hi, c_lo[3], c_hi[3];
} grec;

/* Interval helpers for the screen box (sound enclosures, no correlation). */
typedef struct { double l, u; } ival;
static ival iv_mul(ival a, ival b)
{
    double p[4] = {a.l * b.l, a.l * b.u, a.u * b.l, a.u * b.u};
    ival r = {p[0], p[0]};
    for (int i = 1; i < 4; ++i) { r.l = fmin(r.l, p[i]); r.u = fmax(r.u, p[i]); }
    return r;
}
static ival iv_scale(ival a, double s) { ival r = s >= 0 ? (ival){s * a.l, s * a.u} : (ival){s * a.u, s * a.l}; return r; }
static ival iv_add(ival a, ival b) { ival r = {a.l + b.l, a.u + b.u}; return r; }
static double iv_sqmax(ival a) { return fmax(a.l * a.l, a.u * a.u); }

/* Scene-parameter boxes for the abstract render (Sec. 4.5): per Gaussian 14
 * doubles, mean lo[3], hi[3] (world frame), opacity lo, hi, colour lo[3],
 * hi[3]; each Gaussian's parameters range over their boxes independently.
 * Set for the calls that follow (NULL clears them). */
static double *g_boxes = NULL;
static int64_t g_boxes_n = 0;

int orc_set_boxes(const double *boxes, int64_t n)
{
    free(g_boxes);
    g_boxes = NULL;
    g_boxes_n = 0;
    if (!boxes || n <= 0) return 0;
    g_boxes = (double *)malloc(sizeof(double) * 14 * (size_t)n);
    if (!g_boxes) return 1;
    memcpy(g_boxes, boxes, sizeof(double) * 14 * (size_t)n);
    g_boxes_n = n;
    return 0;
}

static const double *box_of(int64_t i) { return (g_boxes && i < g_boxes_n) ? g_boxes + 14 * i : NULL; }

static void gaussian_record(const camera *cam, const cellforms *cf, const double *uw, const double *ls,
                            const double *q, double o, const double *rgb, const double *pb, grec *g)
{
    memset(g, 0, sizeof *g);
    /* the parameters, as boxes (lo = hi = the nominal value without one) */
    double uwl[3], uwh[3];
    for (int k = 0; k < 3; ++k) {
        uwl[k] = pb ? pb[k] : uw[k];
        uwh[k] = pb ? pb[3 + k] : uw[k];
        g->c_lo[k] = pb ? pb[8 + k] : rgb[k];
        g->c_hi[k] = pb ? pb[11 + k] : rgb[k];
    }
    g->o_lo = pb ? pb[6] : o;
    g->o_hi = pb ? pb[7] : o;
    g->tau_lo = (g->o_lo > 0) ? 2.0 * log(255.0 * g->o_lo) : -INFINITY;
    g->tau_hi = (g->o_hi > 0) ? 2.0 * log(255.0 * g->o_hi) : -INFINITY;
    g->rho = INFINITY;
    if (!(g->tau_hi >= 0)) return;   /* o < 1/255: never reaches the cutoff */

    /* a1: camera-frame mean v = R0 (uw - t0), an interval over the mean's box
     * (each product taken at the end of the box its sign selects), and N = R0 Mw */
    double Mw[9], N[9], vl[3], vh[3];
    cov_factor(ls, q, Mw);
    mat3_mul(cam->R0, Mw, N);
    for (int a = 0; a < 3; ++a) {
        vl[a] = 0;
        vh[a] = 0;
        for (int b = 0; b < 3; ++b) {
            const double r = cam->R0[3 * a + b], dl = uwl[b] - cam->t0[b], dh = uwh[b] - cam->t0[b];
            vl[a] += r >= 0 ? r * dl : r * dh;
            vh[a] += r >= 0 ? r * dh : r * dl;
        }
    }
    /* Algorithm 1, line 2: uc = R_delta^T (v - s) */
    bs vms[3], uc[3];
    for (int b = 0; b < 3; ++b) {
        bs vb;
        vb.lo = lf_cst(vl[b]);
        vb.hi = lf_cst(vh[b]);
        vms[b] = bs_sub(vb, cf->s[b]);
    }
    for (int a = 0; a < 3; ++a) {
        uc[a] = bs_mul(cf->Rd[a], vms[0]);   /* R_delta[0][a] */
        uc[a] = bs_add(uc[a], bs_mul(cf->Rd[3 + a], vms[1]));
        uc[a] = bs_add(uc[a], bs_mul(cf->Rd[6 + a], vms[2]));
    }
    bs d = uc[2];                                  /* line 7 */
    double dlo = bs_min(&d), dhi = bs_max(&d);
    if (!(dhi > cam->near_plane)) return;          /* entirely at or behind the near plane */
    g->straddle = !(dlo > cam->near_plane);

    /* depth key: d minus the translation-only linear term shared by all Gaussians */
    lf gk = lf_cst(0);
    for (int k = 0; k < 3; ++k) {
        double s = 0;
        for (int b = 0; b < 3; ++b) s += cf->Rc[3 * b + 2] * cam->R0[3 * b + k];
        gk.c[k] = -s * cf->h[k];
    }
    lf kl = lf_sub(&d.lo, &gk), kh = lf_sub(&d.hi, &gk);
    g->klo = lf_min(&kl); g->khi = lf_max(&kh);
    double kpad = KEY_SLACK * (1.0 + fmax(fabs(g->klo), fabs(g->khi)));
    g->klo -= kpad; g->khi += kpad;

    /* line 5: up = K uc */
    bs up0 = bs_add(bs_scale(uc[0], cam->fx), bs_scale(uc[2], cam->cx));
    bs up1 = bs_add(bs_scale(uc[1], cam->fy), bs_scale(uc[2], cam->cy));
    /* line 3: Mc = R_delta^T N  (N constant) */
    bs Mc[9];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            bs s = bs_scale(cf->Rd[a], N[c]);
            s = bs_add(s, bs_scale(cf->Rd[3 + a], N[3 + c]));
            s = bs_add(s, bs_scale(cf->Rd[6 + a], N[6 + c]));
            Mc[3 * a + c] = s;
        }

    /* screen box: centres of pixels that can lie in the ellipse m <= tau for
     * some pose of the cell with d > near.  Interval arithmetic in FP64 on
     * the concretised rotation entries; the mean is mu = c + f uc / d and the
     * half-extent of the ellipse is sqrt(tau X_rr) / d^2 (X = d^4 Sigma_2D). */
    {
        ival Ri[9], vs[3];
        for (int e = 0; e < 9; ++e) { Ri[e].l = bs_min(&cf->Rd[e]); Ri[e].u = bs_max(&cf->Rd[e]); }
        for (int b = 0; b < 3; ++b) { vs[b].l = vl[b] - bs_max(&cf->s[b]); vs[b].u = vh[b] - bs_min(&cf->s[b]); }
        double dl = fmax(dlo, cam->near_plane);
        ival D = {dl, dhi};
        ival ucx = iv_add(iv_add(iv_mul(Ri[0], vs[0]), iv_mul(Ri[3], vs[1])), iv_mul(Ri[6], vs[2]));
        ival ucy = iv_add(iv_add(iv_mul(Ri[1], vs[0]), iv_mul(Ri[4], vs[1])), iv_mul(Ri[7], vs[2]));
        ival mux = {cam->cx + cam->fx * fmin(ucx.l / D.l, ucx.l / D.u), cam->cx + cam->fx * fmax(ucx.u / D.l, ucx.u / D.u)};
        ival muy = {cam->cy + cam->fy * fmin(ucy.l / D.l, ucy.l / D.u), cam->cy + cam->fy * fmax(ucy.u / D.l, ucy.u / D.u)};
        /* frustum guard band: a mean outside it at every pose of the cell
         * drops the pair; outside it at some pose makes the lower alpha 0 */
        {
            const double gx = GUARD * cam->W, gy = GUARD * cam->H;
            const double ml = mux.l - BOX_SLACK * (1 + fabs(mux.l)), mh = mux.u + BOX_SLACK * (1 + fabs(mux.u));
            const double nl = muy.l - BOX_SLACK * (1 + fabs(muy.l)), nh = muy.u + BOX_SLACK * (1 + fabs(muy.u));
            if (ml > cam->cx + gx || mh < cam->cx - gx || nl > cam->cy + gy || nh < cam->cy - gy) return;
            if (!(ml >= cam->cx - gx && mh <= cam->cx + gx && nl >= cam->cy - gy && nh <= cam->cy + gy))
                g->straddle = 1;
        }
        double X00 = 0, X11 = 0;
        for (int c = 0; c < 3; ++c) {
            ival m[3];
            for (int a = 0; a < 3; ++a)
                m[a] = iv_add(iv_add(iv_scale(Ri[a], N[c]), iv_scale(Ri[3 + a], N[3 + c])), iv_scale(Ri[6 + a], N[6 + c]));
            ival p0 = iv_scale(iv_add(iv_mul(D, m[0]), iv_scale(iv_mul(ucx, m[2]), -1.0)), cam->fx);
            ival p1 = iv_scale(iv_add(iv_mul(D, m[1]), iv_scale(iv_mul(ucy, m[2]), -1.0)), cam->fy);
            X00 += iv_sqmax(p0); X11 += iv_sqmax(p1);
        }
        double rx = sqrt(g->tau_hi * X00) / (dl * dl), ry = sqrt(g->tau_hi * X11) / (dl * dl);
        double xl = mux.l - rx, xh = mux.u + rx, yl = muy.l - ry, yh = muy.u + ry;
        xl -= BOX_SLACK * (1 + fabs(xl)); xh += BOX_SLACK * (1 + fabs(xh));
        yl -= BOX_SLACK * (1 + fabs(yl)); yh += BOX_SLACK * (1 + fabs(yh));
        if (!(xh >= xl) || !(yh >= yl)) return;      /* NaN guard */
        double fx0 = ceil(xl - 0.5), fx1 = floor(xh - 0.5), fy0 = ceil(yl - 0.5), fy1 = floor(yh - 0.5);
        fx0 = fmax(fx0, 0); fy0 = fmax(fy0, 0);
        fx1 = fmin(fx1, cam->W - 1); fy1 = fmin(fy1, cam->H - 1);
        if (fx0 > fx1 || fy0 > fy1) return;
        g->px0 = (int)fx0; g->px1 = (int)fx1; g->py0 = (int)fy0; g->py1 = (int)fy1;
    }
    g->valid = 1;

    /* line 4 and 6: J and Mp = J Mc (J entries are forms; products by Mul) */
    bs J00 = bs_scale(d, cam->fx), J02 = bs_scale(uc[0], -cam->fx);
    bs J11 = bs_scale(d, cam->fy), J12 = bs_scale(uc[1], -cam->fy);
    bs Mp[6];
    for (int c = 0; c < 3; ++c) {
        Mp[c] = bs_add(bs_mul(J00, Mc[c]), bs_mul(J02, Mc[6 + c]));
        Mp[3 + c] = bs_add(bs_mul(J11, Mc[3 + c]), bs_mul(J12, Mc[6 + c]));
    }
    /* line 8 argument: X = Mp Mp^T (squares on the diagonal) */
    bs X[4];
    X[0] = bs_add(bs_add(bs_sq(Mp[0]), bs_sq(Mp[1])), bs_sq(Mp[2]));
    X[3] = bs_add(bs_add(bs_sq(Mp[3]), bs_sq(Mp[4])), bs_sq(Mp[5]));
    X[1] = bs_add(bs_add(bs_mul(Mp[0], Mp[3]), bs_mul(Mp[1], Mp[4])), bs_mul(Mp[2], Mp[5]));
    X[2] = X[1];
    /* line 9 factors: S = d*d, P = d*up */
    g->S = bs_sq(d);
    g->Px = bs_mul(d, up0);
    g->Py = bs_mul(d, up1);
    /* line 8: Conic <- MatrixInv(X; X0, k), with the adaptive order and the
     * input splitting of Sec. 3.1 */
    bs conic[4];
    if (matrix_inv_cell(X, conic, &g->rho, &g->korder, &g->pieces, &g->rho_margin)) { g->fallback = 1; return; }
    /* W = Conic * Mp, so that q = Delta^T W */
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            g->W[3 * r + c] = bs_add(bs_mul(conic[2 * r], Mp[c]), bs_mul(conic[2 * r + 1], Mp[3 + c]));
}

static double clamp01(double x) { return x < 0 ? 0 : (x > 1 ? 1 : x); }

/* Exp relaxation of Table 2 on x <= 0.  x is a bounded scalar; its range
 * [x_lo, x_hi] is concretised from its forms and x_hi is clipped at 0 (the
 * argument is x = -m/2 and m >= 0, so no pose reaches x > 0).  With
 * E = exp(x_lo):
 *   lower: the tangent at x_lo,  E (1 + x - x_lo),  applied to the lower form;
 *   upper: the secant over [x_lo, x_hi],  E + s (x - x_lo),
 *          s = (exp(x_hi) - E) / (x_hi - x_lo)  (s = E on a point interval),
 *          applied to the upper form.
 * Both slopes are positive, so each side takes its own side's form. */
static bs bs_exp(bs x)
{
    double xl = bs_min(&x), xu = fmin(bs_max(&x), 0.0);
    if (xu < xl) xu = xl;
    double El = exp(xl);
    double slope = (xu > xl) ? (exp(xu) - El) / (xu - xl) : El;
    bs e;
    e.lo = lf_scale(&x.lo, El); e.lo.k += El * (1.0 - xl);
    e.hi = lf_scale(&x.hi, slope); e.hi.k += El - slope * xl;
    return e;
}

/* Effective-opacity bounds of one Gaussian at one pixel from its Mahalanobis
 * term m (Algorithm 1 line 10 relaxed): a = o Exp(-m/2), then the upper clip
 * to o and the two 1/255 cutoff ramps.  Produces lower/upper forms and their
 * scalar enclosure. */
typedef struct { lf L, U; double alo, ahi; double mlo, mhi, ramp; } galpha;

static void alpha_from_m(const bs *m, double o_lo, double o_hi, double tau_lo, double tau_hi, int straddle,
                         galpha *r)
{
    double mlo = bs_min(m), mhi = bs_max(m);
    r->mlo = mlo; r->mhi = mhi;
    /* Exp on x = -m/2 (x.lo = -m.hi/2, x.hi = -m.lo/2) */
    bs x;
    x.lo = lf_scale(&m->hi, -0.5);
    x.hi = lf_scale(&m->lo, -0.5);
    bs e = bs_exp(x);
    /* a = o e with o in [o_lo, o_hi] and e >= 0: o_lo below, o_hi above */
    lf La = lf_scale(&e.lo, o_lo), Ua = lf_scale(&e.hi, o_hi);
    /* upper side: blend toward the constant o when the form's maximum exceeds o */
    double amax = lf_max(&Ua);
    double lam = clamp01((o_hi * (1.0 + CLIP_RAMP) - amax) / (o_hi * CLIP_RAMP));
    lf U1 = lf_scale(&Ua, lam); U1.k += (1.0 - lam) * o_hi;
    /* cutoff ramps: width shrinks with the m interval, zero on a point cell */
    double ramp = fmin(CUT_RAMP, mhi - mlo);
    if (!(ramp > 0)) ramp = 0;
    r->ramp = ramp;
    /* the upper form is cut where m > tau(o_hi) for every pose (no opacity in
     * the box is then visible); the lower one keeps a margin of 1/255 unless
     * m <= tau(o_lo) at every pose (no opacity in the box is then cut) */
    double psi2 = (mlo <= tau_hi) ? 0.0 : (ramp > 0 ? clamp01((mlo - tau_hi) / ramp) : 1.0);
    double psi = (mhi > tau_lo) ? 1.0 : (ramp > 0 ? clamp01((mhi - tau_lo + ramp) / ramp) : 0.0);
    r->U = lf_scale(&U1, 1.0 - psi2);
    lf L2 = La; L2.k -= psi * ALPHA_MIN;
    double l2min = lf_min(&L2), l2max = lf_max(&L2);
    double mu = (l2min >= 0) ? 1.0 : ((l2max <= 0) ? 0.0 : l2max / (l2max - l2min));
    r->L = lf_scale(&L2, mu);
    if (straddle) r->L = lf_cst(0);
    r->alo = fmax(0.0, lf_min(&r->L));
    r->ahi = fmin(o_hi, lf_max(&r->U));
}

/* The Mahalanobis term of one Gaussian at pixel u (Algorithm 1 line 9):
 * Delta = d^2 u - d up = S u - P (u constant), q = Delta^T W, m = q q^T. */
static bs gaussian_m(const grec *g, double ux, double uy)
{
    bs Dx = bs_sub(bs_scale(g->S, ux), g->Px);
    bs Dy = bs_sub(bs_scale(g->S, uy), g->Py);
    bs m = bs_cst(0);
    for (int c = 0; c < 3; ++c) {
        bs qc = bs_add(bs_mul(Dx, g->W[c]), bs_mul(Dy, g->W[3 + c]));
        m = bs_add(m, bs_sq(qc));
    }
    return m;
}

/* Effective-opacity bounds of one Gaussian at one pixel (Algorithm 1 lines
 * 9-10 relaxed). */
static void gaussian_alpha(const grec *g, double ux, double uy, galpha *r)
{
    if (g->fallback) {
        r->L = lf_cst(0); r->U = lf_cst(g->o_hi); r->alo = 0; r->ahi = g->o_hi;
        r->mlo = -INFINITY; r->mhi = INFINITY; r->ramp = 0;
        return;
    }
    bs m = gaussian_m(g, ux, uy);
    alpha_from_m(&m, g->o_lo, g->o_hi, g->tau_lo, g->tau_hi, g->straddle, r);
}

/* Abstract render of one cell over the pixel window [px0,px1] x [py0,py1].
 * out_lo/out_hi are [H][W][3] (only the window is written).  fragile, if
 * given, is [H][W] and marks pixels where a threshold decision that the FP32
 * path takes in single precision lies within a relative 1e-3 of its
 * threshold (both outcomes are sound there).  cond, if given, is [H][W] and
 * holds an estimate of how far single-precision evaluation of the same
 * bounds can move them: each Gaussian's m interval is computed from terms
 * of magnitude about |m_lo| + |m_hi|, so in FP32 its ends move by about
 * 32 u (|m_lo| + |m_hi|) (u = 2^-24, 32 covering the chain of products),
 * its opacity bounds by half of that times a (a_hi only while m_lo > 0: below
 * that the upper secant ends at x = 0 and a_hi = o), and the pixel colour by
 * at most 2 T_hi times that (d colour / d a_i is at most 2 T_i). */
/* Abstract BlendSort (Algorithm 2 with an abstract Sort), the comparison of
 * Example 2.  Sort is abstracted by rank ranges: Gaussian i of the pixel has
 * rank at least the number of Gaussians certainly in front of it (k_hi(j) <
 * k_lo(i)) and at most the number possibly in front (k_lo(j) < k_hi(i)), so
 * the Gaussian at rank r is one of those whose range holds r, and a, c a at
 * rank r lie in the hull of theirs.  Algorithm 2's sum over ranks then takes
 * the hulls: lower sum of min c_lo a_lo times the product of (1 - max a_hi)
 * before it, upper sum of max c_hi a_hi times the product of (1 - min a_lo).
 * Sound for distinct depths (a Gaussian may enter several ranks' hulls: the
 * index uncertainty Sec. 3.2 removes with BlendInd).  Interval bounds. */
static void blend_sort_abstract(const grec *G, const int64_t *idx, const galpha *A, int64_t K, double out_lo[3],
                                double out_hi[3])
{
    int64_t *rmin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    int64_t *rmax = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    for (int ch = 0; ch < 3; ++ch) { out_lo[ch] = 0; out_hi[ch] = 0; }
    if (!rmin || !rmax) { free(rmin); free(rmax); for (int ch = 0; ch < 3; ++ch) out_hi[ch] = 1; return; }
    for (int64_t a = 0; a < K; ++a) {
        const grec *gi = &G[idx[a]];
        rmin[a] = 0;
        rmax[a] = 0;
        for (int64_t b = 0; b < K; ++b) {
            if (b == a) continue;
            const grec *gj = &G[idx[b]];
            if (gj->khi < gi->klo) ++rmin[a];
            if (gj->klo < gi->khi) ++rmax[a];
        }
    }
    for (int ch = 0; ch < 3; ++ch) {
        double Tlo = 1.0, Thi = 1.0, slo = 0.0, shi = 0.0;
        for (int64_t r = 0; r < K; ++r) {
            double amin = INFINITY, amax = -INFINITY, calo = INFINITY, cahi = -INFINITY;
            for (int64_t a = 0; a < K; ++a) {
                if (r < rmin[a] || r > rmax[a]) continue;
                const grec *gi = &G[idx[a]];
                amin = fmin(amin, A[a].alo);
                amax = fmax(amax, A[a].ahi);
                calo = fmin(calo, gi->c_lo[ch] * A[a].alo);
                cahi = fmax(cahi, gi->c_hi[ch] * A[a].ahi);
            }
            slo += calo * Tlo;
            shi += cahi * Thi;
            Tlo *= 1.0 - amax;
            Thi *= 1.0 - amin;
        }
        out_lo[ch] = clamp01(slo);
        out_hi[ch] = clamp01(shi);
    }
    free(rmin);
    free(rmax);
}

/* Upper transmittance of the a-th Gaussian of a pixel as an affine form
 * (transmittance kept relational in the pose, upper side):
 * T(i) = prod over j certainly in front of i (k_hi(j) < k_lo(i)) of (1 - a_j),
 * the factors taken in increasing k_hi(j) (ties by Gaussian index), which is
 * the order in which a depth sweep meets their upper endpoints; `order` lists
 * the pixel's Gaussians in that order.  With the running product y <= y_hi
 * bounded above by the form F and the next factor x = 1 - a_j in
 * [1 - a_hi(j), 1 - a_lo(j)] bounded above by the form X_j, the McCormick
 * plane (y_hi - y)(x - x_lo) >= 0 gives
 *   y x <= y_hi X_j + x_lo (F - y_hi),
 * sound because y_hi >= 0 and x_lo >= 0 weight upper bounds.  y_hi is the
 * interval product, updated alongside.  X_j = 1 - L_j where a_lo(j) > 0 (there
 * L_j >= a_lo(j) on the whole cell, so X_j <= 1 - a_lo(j)), else the constant
 * 1; then F <= y_hi at every pose, step by step, and the term the colour sum
 * gains from F is never positive.  Returns F and y_hi. */
/* One factor of the chain below: F <- y_hi X + x_lo (F - y_hi), then
 * y_hi <- y_hi (1 - a_lo), with x_lo = 1 - a_hi and X = 1 - L where a_lo > 0,
 * else 1. */
static void transmittance_step(lf *F, double *yhi, const lf *L, double alo, double ahi)
{
    const double xlo = 1.0 - ahi;
    lf X = lf_cst(1.0);
    if (alo > 0.0) {
        X = lf_scale(L, -1.0);
        X.k += 1.0;
    }
    lf t1 = lf_scale(&X, *yhi);
    F->k -= *yhi;
    lf t2 = lf_scale(F, xlo);
    *F = lf_add(&t1, &t2);
    *yhi *= 1.0 - alo;
}

static void upper_transmittance(const grec *G, const int64_t *idx, const galpha *A, const int64_t *order, int64_t K,
                                int64_t a, lf *F_out, double *yhi_out)
{
    const grec *gi = &G[idx[a]];
    lf F = lf_cst(1.0);
    double yhi = 1.0;
    for (int64_t u = 0; u < K && G[idx[order[u]]].khi < gi->klo; ++u) {
        const galpha *Aj = &A[order[u]];
        transmittance_step(&F, &yhi, &Aj->L, Aj->alo, Aj->ahi);
    }
    *F_out = F;
    *yhi_out = yhi;
}

/* The chain of upper_transmittance on given factors (for tests): K factors
 * with lower opacity forms L (K x 7: six coefficients, then the constant)
 * and opacity bounds [alo, ahi]; F (7 doubles) and y_hi out. */
int orc_transmittance_chain(const double *L, const double *alo, const double *ahi, int K, double *F_out,
                            double *yhi_out)
{
    lf F = lf_cst(1.0);
    double yhi = 1.0;
    for (int j = 0; j < K; ++j) {
        lf Lj;
        for (int v = 0; v < NV; ++v) Lj.c[v] = L[7 * j + v];
        Lj.k = L[7 * j + 6];
        transmittance_step(&F, &yhi, &Lj, alo[j], ahi[j]);
    }
    for (int v = 0; v < NV; ++v) F_out[v] = F.c[v];
    F_out[6] = F.k;
    *yhi_out = yhi;
    return 0;
}

/* the pixel's Gaussians by increasing (k_hi, Gaussian index) */
static const grec *g_sort_G;
static const int64_t *g_sort_idx;
#pragma omp threadprivate(g_sort_G, g_sort_idx)
static int by_khi(const void *x, const void *y)
{
    const int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    const double ka = g_sort_G[g_sort_idx[a]].khi, kb = g_sort_G[g_sort_idx[b]].khi;
    if (ka != kb) return ka < kb ? -1 : 1;
    return g_sort_idx[a] < g_sort_idx[b] ? -1 : (g_sort_idx[a] > g_sort_idx[b]);
}

static int render_abstract_impl(const double *uw, const double *ls, const double *quat, const double *opac,
                                const double *rgb, int64_t n, const double *intr, const double *R0,
                                const double *t0, const double *cell_lo, const double *cell_hi,
                                int px0, int px1, int py0, int py1, double *out_lo, double *out_hi,
                                uint8_t *fragile, double *cond, int blend_mode)
{
    const int sort_blend = blend_mode == 1, tight = blend_mode == 2;
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
    grec *G = (grec *)malloc(sizeof(grec) * (size_t)(n > 0 ? n : 1));
    if (!G) return 1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        gaussian_record(&cam, &cf, uw + 3 * i, ls + 3 * i, quat + 4 * i, opac[i], rgb + 3 * i, box_of(i), &G[i]);

    int npx = px1 - px0 + 1, npy = py1 - py0 + 1;
    int status = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int pix = 0; pix < npx * npy; ++pix) {
        int px = px0 + pix % npx, py = py0 + pix / npx;
        double ux = px + 0.5, uy = py + 0.5;
        int64_t cap = 256, K = 0;
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * cap);
        galpha *A = (galpha *)malloc(sizeof(galpha) * cap);
        int frag = 0;
        if (!idx || !A) { status = 1; free(idx); free(A); continue; }
        for (int64_t i = 0; i < n; ++i) {
            const grec *g = &G[i];
            if (!g->valid || px < g->px0 || px > g->px1 || py < g->py0 || py > g->py1) continue;
            if (K == cap) {
                cap *= 2;
                idx = (int64_t *)realloc(idx, sizeof(int64_t) * cap);
                A = (galpha *)realloc(A, sizeof(galpha) * cap);
                if (!idx || !A) { status = 1; break; }
            }
            idx[K] = i;
            gaussian_alpha(g, ux, uy, &A[K]);
            /* threshold decisions the FP32 path takes in single precision */
            /* rho is FP64 on both sides, from the same X0 (the inverse of the
             * centre matrix, Sec. 3.1 adjustment (1)); their X forms differ by
             * FP64 rounding only, far below this margin */
            if (g->rho_margin < 1e-9) frag = 1;
            if (!g->fallback && A[K].ramp < 0.05) {
                /* a narrow ramp makes the cutoff nearly a step in m */
                double tol = 1e-3 * fmax(1.0, g->tau_hi), rp = A[K].ramp;
                if (A[K].mhi > g->tau_lo - rp - tol && A[K].mhi < g->tau_lo + tol) frag = 1;
                if (A[K].mlo > g->tau_hi - tol && A[K].mlo < g->tau_hi + rp + tol) frag = 1;
            }
            ++K;
        }
        if (!idx || !A) { free(idx); free(A); continue; }
        if (sort_blend) {
            double bl[3], bh[3];
            blend_sort_abstract(G, idx, A, K, bl, bh);
            size_t o = 3 * ((size_t)py * cam.W + px);
            for (int ch = 0; ch < 3; ++ch) { out_lo[o + ch] = bl[ch]; out_hi[o + ch] = bh[ch]; }
            if (fragile) fragile[(size_t)py * cam.W + px] = (uint8_t)frag;
            if (cond) cond[(size_t)py * cam.W + px] = 0.0;
            free(idx); free(A);
            continue;
        }
        /* BlendInd with interval Prod: for each i, T_lo over j that may be in
         * front (not certainly behind), T_hi over j certainly in front */
        lf lo[3], hi[3];
        double est = 0.0, kplain[3] = {0.0, 0.0, 0.0};
        int64_t *order = NULL;
        if (tight) {
            order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
            if (!order) { status = 1; free(idx); free(A); continue; }
            for (int64_t u = 0; u < K; ++u) order[u] = u;
            g_sort_G = G;
            g_sort_idx = idx;
            qsort(order, (size_t)K, sizeof(int64_t), by_khi);
        }
        for (int ch = 0; ch < 3; ++ch) { lo[ch] = lf_cst(0); hi[ch] = lf_cst(0); }
        for (int64_t a = 0; a < K; ++a) {
            const grec *gi = &G[idx[a]];
            double Tlo = 1.0, Thi = 1.0;
            for (int64_t b = 0; b < K; ++b) {
                if (b == a) continue;
                const grec *gj = &G[idx[b]];
                if (gj->khi < gi->klo) {               /* Ind(d_i - d_j) = 1 on the whole cell */
                    Tlo *= 1.0 - A[b].ahi;
                    Thi *= 1.0 - A[b].alo;
                } else if (gj->klo < gi->khi) {        /* Ind(d_i - d_j) in {0, 1} */
                    Tlo *= 1.0 - A[b].ahi;
                }                                      /* else Ind(d_i - d_j) = 0 */
            }
            if (!gi->fallback && isfinite(A[a].mlo) && isfinite(A[a].mhi)) {
                /* a_hi moves with m_lo only while m_lo > 0 (else the secant ends at
                 * x = 0 and a_hi = o); a_lo moves with m_hi in proportion to itself */
                double em = 32.0 * 5.9604644775390625e-8 * (fabs(A[a].mlo) + fabs(A[a].mhi));
                double da = 0.5 * em * ((A[a].mlo > 0 ? A[a].ahi : 0.0) + A[a].alo);
                est += 2.0 * Thi * da;
            }
            /* relational upper transmittance: FU(p) >= T(i) at every pose */
            lf dU = lf_cst(0.0);
            if (tight) {
                lf FU;
                double PB;
                upper_transmittance(G, idx, A, order, K, a, &FU, &PB);
                /* McCormick upper plane of T a: T_hi U + a_lo (FU - T_hi) */
                FU.k -= PB;
                dU = lf_scale(&FU, A[a].alo);
                Thi = PB;
            }
            for (int ch = 0; ch < 3; ++ch) {
                /* colour in [c_lo, c_hi] and L', U' >= 0 over the cell */
                lf t = lf_scale(&A[a].L, Tlo * gi->c_lo[ch]);
                lo[ch] = lf_add(&lo[ch], &t);
                t = lf_scale(&A[a].U, Thi * gi->c_hi[ch]);
                kplain[ch] += t.k;
                if (tight) {
                    lf t2 = lf_scale(&dU, gi->c_hi[ch]);
                    t = lf_add(&t, &t2);
                }
                hi[ch] = lf_add(&hi[ch], &t);
            }
        }
        size_t o = 3 * ((size_t)py * cam.W + px);
        for (int ch = 0; ch < 3; ++ch) {
            out_lo[o + ch] = clamp01(lf_min(&lo[ch]));
            out_hi[o + ch] = clamp01(lf_max(&hi[ch]));
        }
        if (tight) {
            /* saturation: where the constants of the interval terms alone sum
             * to 1 or more in every channel, the interval blend's upper bound
             * is 1 and the relational one is taken as 1 too (a sweep can stop
             * there, as it does for the interval blend).  Near the threshold
             * the single-precision sums may decide the other way: fragile. */
            const double kmin = fmin(kplain[0], fmin(kplain[1], kplain[2]));
            if (kmin >= 1.0)
                for (int ch = 0; ch < 3; ++ch) out_hi[o + ch] = 1.0;
            if (fabs(kmin - 1.0) < 1e-3) frag = 1;
        }
        if (fragile) fragile[(size_t)py * cam.W + px] = (uint8_t)frag;
        if (cond) cond[(size_t)py * cam.W + px] = est;
        free(order);
        free(idx); free(A);
    }
    free(G);
    return status;
}

int orc_render_abstract(const double *uw, const double *ls, const double *quat, const double *opac,
                        const double *rgb, int64_t n, const double *intr, const double *R0,
                        const double *t0, const double *cell_lo, const double *cell_hi,
                        int px0, int px1, int py0, int py1, double *out_lo, double *out_hi,
                        uint8_t *fragile, double *cond)
{
    return render_abstract_impl(uw, ls, quat, opac, rgb, n, intr, R0, t0, cell_lo, cell_hi, px0, px1, py0, py1,
                                out_lo, out_hi, fragile, cond, 0);
}

/* The same with the relational upper transmittance of upper_transmittance. */
int orc_render_abstract_tight(const double *uw, const double *ls, const double *quat, const double *opac,
                              const double *rgb, int64_t n, const double *intr, const double *R0,
                              const double *t0, const double *cell_lo, const double *cell_hi,
                              int px0, int px1, int py0, int py1, double *out_lo, double *out_hi,
                              uint8_t *fragile, double *cond)
{
    return render_abstract_impl(uw, ls, quat, opac, rgb, n, intr, R0, t0, cell_lo, cell_hi, px0, px1, py0, py1,
                                out_lo, out_hi, fragile, cond, 2);
}

/* The same with the abstract BlendSort of blend_sort_abstract (Example 2). */
int orc_render_abstract_sort(const double *uw, const double *ls, const double *quat, const double *opac,
                             const double *rgb, int64_t n, const double *intr, const double *R0,
                             const double *t0, const double *cell_lo, const double *cell_hi,
                             int px0, int px1, int py0, int py1, double *out_lo, double *out_hi)
{
    return render_abstract_impl(uw, ls, quat, opac, rgb, n, intr, R0, t0, cell_lo, cell_hi, px0, px1, py0, py1,
                                out_lo, out_hi, NULL, NULL, 1);
}

/* Per-Gaussian record summary for one cell (for tests): valid, straddle,
 * fallback, klo, khi, px0, px1, py0, py1, rho, pieces, korder, rho_margin ->
 * 13 doubles per Gaussian. */
int orc_records(const double *uw, const double *ls, const double *quat, const double *opac,
                const double *rgb, int64_t n, const double *intr, const double *R0, const double *t0,
                const double *cell_lo, const double *cell_hi, double *out)
{
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        grec g;
        gaussian_record(&cam, &cf, uw + 3 * i, ls + 3 * i, quat + 4 * i, opac[i], rgb + 3 * i, box_of(i), &g);
        double *o = out + 13 * i;
        o[0] = g.valid; o[1] = g.straddle; o[2] = g.fallback; o[3] = g.klo; o[4] = g.khi;
        o[5] = g.px0; o[6] = g.px1; o[7] = g.py0; o[8] = g.py1; o[9] = g.rho;
        o[10] = g.pieces; o[11] = g.korder; o[12] = g.rho_margin;
    }
    return 0;
}

/* Thread count for the OpenMP loops (returns the count in effect). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Soundness harness: renders the scene at each of npose poses (BlendSort) and
 * compares with the bounds lo/hi ([H][W][3]).  Returns the largest violation
 * max(lo - img, img - hi, 0) and writes the number of violating values. */
double orc_check_samples(const double *uw, const double *ls, const double *quat, const double *opac,
                         const double *rgb, int64_t n, const double *intr, const double *R0,
                         const double *t0, const double *poses, int64_t npose, const double *lo,
                         const double *hi, double tol, int64_t *nviol)
{
    camera cam = make_camera(intr, R0, t0);
    size_t npix = (size_t)cam.W * cam.H * 3;
    double worst = 0;
    int64_t count = 0;
#pragma omp parallel
    {
        double *img = (double *)malloc(sizeof(double) * npix);
        double w_local = 0;
        int64_t c_local = 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < npose; ++p) {
            if (!img) continue;
            orc_render_concrete(uw, ls, quat, opac, rgb, n, intr, R0, t0, poses + 6 * p, 0, img);
            for (size_t e = 0; e < npix; ++e) {
                double v = fmax(lo[e] - img[e], img[e] - hi[e]);
                if (v > tol) ++c_local;
                if (v > w_local) w_local = v;
            }
        }
#pragma omp critical
        {
            if (w_local > worst) worst = w_local;
            count += c_local;
        }
        free(img);
    }
    if (nviol) *nviol = count;
    return worst;
}

/* Per-pixel range of the concrete renders over npose poses (the paper's
 * "empirical" bounds of Sec. 4.2): emp_lo/emp_hi are [H][W][3]. */
void orc_empirical_bounds(const double *uw, const double *ls, const double *quat, const double *opac,
                          const double *rgb, int64_t n, const double *intr, const double *R0,
                          const double *t0, const double *poses, int64_t npose, double *emp_lo,
                          double *emp_hi)
{
    camera cam = make_camera(intr, R0, t0);
    size_t npix = (size_t)cam.W * cam.H * 3;
    for (size_t e = 0; e < npix; ++e) { emp_lo[e] = INFINITY; emp_hi[e] = -INFINITY; }
#pragma omp parallel
    {
        double *img = (double *)malloc(sizeof(double) * npix);
        double *l = (double *)malloc(sizeof(double) * npix), *h = (double *)malloc(sizeof(double) * npix);
        if (l && h)
            for (size_t e = 0; e < npix; ++e) { l[e] = INFINITY; h[e] = -INFINITY; }
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < npose; ++p) {
            if (!img || !l || !h) continue;
            orc_render_concrete(uw, ls, quat, opac, rgb, n, intr, R0, t0, poses + 6 * p, 0, img);
            for (size_t e = 0; e < npix; ++e) { l[e] = fmin(l[e], img[e]); h[e] = fmax(h[e], img[e]); }
        }
#pragma omp critical
        {
            if (l && h)
                for (size_t e = 0; e < npix; ++e) { emp_lo[e] = fmin(emp_lo[e], l[e]); emp_hi[e] = fmax(emp_hi[e], h[e]); }
        }
        free(img); free(l); free(h);
    }
}

/* Per-Gaussian details at one pixel of one cell (for diagnosis): for each
 * Gaussian whose pixel box holds the pixel, 12 doubles: index, mlo, mhi,
 * ramp, alo, ahi, klo, khi, L.k, U.k, flags (1 fallback, 2 straddle), rho.
 * Returns the number of Gaussians written (at most cap). */
int orc_pixel_detail(const double *uw, const double *ls, const double *quat, const double *opac,
                     const double *rgb, int64_t n, const double *intr, const double *R0, const double *t0,
                     const double *cell_lo, const double *cell_hi, int px, int py, double *out, int cap)
{
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
    int k = 0;
    for (int64_t i = 0; i < n && k < cap; ++i) {
        grec g;
        gaussian_record(&cam, &cf, uw + 3 * i, ls + 3 * i, quat + 4 * i, opac[i], rgb + 3 * i, box_of(i), &g);
        if (!g.valid || px < g.px0 || px > g.px1 || py < g.py0 || py > g.py1) continue;
        galpha a;
        gaussian_alpha(&g, px + 0.5, py + 0.5, &a);
        double *o = out + 12 * k;
        o[0] = (double)i; o[1] = a.mlo; o[2] = a.mhi; o[3] = a.ramp; o[4] = a.alo; o[5] = a.ahi;
        o[6] = g.klo; o[7] = g.khi; o[8] = a.L.k; o[9] = a.U.k; o[10] = g.fallback + 2 * g.straddle; o[11] = g.rho;
        ++k;
    }
    return k;
}

/* The opacity stage alone, for the pins: m as a packed bounded scalar (14
 * doubles: lower coefficients, lower constant, upper coefficients, upper
 * constant), the opacity box, the two cutoff exponents tau = 2 ln(255 o) and
 * the near-plane straddle flag.  out: L (7), U (7), alo, ahi, mlo, mhi, ramp. */
void orc_alpha_from_m(const double *m, double o_lo, double o_hi, double tau_lo, double tau_hi, int straddle,
                      double *out)
{
    bs mm = unpack_bs(m);
    galpha a;
    alpha_from_m(&mm, o_lo, o_hi, tau_lo, tau_hi, straddle, &a);
    for (int i = 0; i < NV; ++i) { out[i] = a.L.c[i]; out[7 + i] = a.U.c[i]; }
    out[6] = a.L.k; out[13] = a.U.k;
    out[14] = a.alo; out[15] = a.ahi; out[16] = a.mlo; out[17] = a.mhi; out[18] = a.ramp;
}

/* gaussian_alpha of one (Gaussian, cell) pair at one pixel, for the pins:
 * out = m (14, packed as above), L (7), U (7), alo, ahi, mlo, mhi, ramp,
 * then the record's o_lo, o_hi, tau_lo, tau_hi, fallback, straddle (39
 * doubles).  Returns 0 if the pair is valid. */
int orc_pixel_alpha(const double *uw, const double *ls, const double *quat, const double *opac,
                    const double *rgb, int64_t n, const double *intr, const double *R0, const double *t0,
                    const double *cell_lo, const double *cell_hi, int64_t gi, int px, int py, double *out)
{
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
    if (gi < 0 || gi >= n) return 1;
    grec g;
    gaussian_record(&cam, &cf, uw + 3 * gi, ls + 3 * gi, quat + 4 * gi, opac[gi], rgb + 3 * gi, box_of(gi), &g);
    if (!g.valid) return 1;
    galpha a;
    gaussian_alpha(&g, px + 0.5, py + 0.5, &a);
    memset(out, 0, 14 * sizeof(double));
    if (!g.fallback) {
        bs m = gaussian_m(&g, px + 0.5, py + 0.5);
        pack_bs(&m, out);
    }
    for (int i = 0; i < NV; ++i) { out[14 + i] = a.L.c[i]; out[21 + i] = a.U.c[i]; }
    out[20] = a.L.k; out[27] = a.U.k;
    out[28] = a.alo; out[29] = a.ahi; out[30] = a.mlo; out[31] = a.mhi; out[32] = a.ramp;
    out[33] = g.o_lo; out[34] = g.o_hi; out[35] = g.tau_lo; out[36] = g.tau_hi;
    out[37] = g.fallback; out[38] = g.straddle;
    return 0;
}

/* Intermediate intervals of one (Gaussian, cell) pair at one pixel (for
 * diagnosis): Dx, Dy, W[0..5], q[0..2], m as (lo, hi) pairs -> 24 doubles.
 * Returns 0 if the pair is valid and not a fallback. */
int orc_pixel_trace(const double *uw, const double *ls, const double *quat, const double *opac,
                    const double *rgb, int64_t n, const double *intr, const double *R0, const double *t0,
                    const double *cell_lo, const double *cell_hi, int64_t gi, int px, int py, double *out)
{
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
    if (gi < 0 || gi >= n) return 1;
    grec g;
    gaussian_record(&cam, &cf, uw + 3 * gi, ls + 3 * gi, quat + 4 * gi, opac[gi], rgb + 3 * gi, box_of(gi), &g);
    if (!g.valid || g.fallback) return 1;
    double ux = px + 0.5, uy = py + 0.5;
    bs Dx = bs_sub(bs_scale(g.S, ux), g.Px);
    bs Dy = bs_sub(bs_scale(g.S, uy), g.Py);
    out[0] = bs_min(&Dx); out[1] = bs_max(&Dx); out[2] = bs_min(&Dy); out[3] = bs_max(&Dy);
    for (int e = 0; e < 6; ++e) { out[4 + 2 * e] = bs_min(&g.W[e]); out[5 + 2 * e] = bs_max(&g.W[e]); }
    bs m = bs_cst(0);
    for (int c = 0; c < 3; ++c) {
        bs qc = bs_add(bs_mul(Dx, g.W[c]), bs_mul(Dy, g.W[3 + c]));
        out[16 + 2 * c] = bs_min(&qc); out[17 + 2 * c] = bs_max(&qc);
        m = bs_add(m, bs_sq(qc));
    }
    out[22] = bs_min(&m); out[23] = bs_max(&m);
    return 0;
}

/* MatrixInv internals of one (Gaussian, cell) pair (for diagnosis): X00, X01,
 * X11, E[4], Mp[6], conic[4] as (lo, hi) pairs, then rho -> 35 doubles. */
int orc_record_trace(const double *uw, const double *ls, const double *quat, const double *opac,
                     const double *rgb, int64_t n, const double *intr, const double *R0, const double *t0,
                     const double *cell_lo, const double *cell_hi, int64_t gi, double *out)
{
    camera cam = make_camera(intr, R0, t0);
    cellforms cf;
    cell_setup(&cam, cell_lo, cell_hi, &cf);
    if (gi < 0 || gi >= n) return 1;
    const double *q = quat + 4 * gi;
    double Mw[9], N[9], v[3];
    cov_factor(ls + 3 * gi, q, Mw);
    mat3_mul(cam.R0, Mw, N);
    for (int a = 0; a < 3; ++a) {
        v[a] = 0;
        for (int b = 0; b < 3; ++b) v[a] += cam.R0[3 * a + b] * (uw[3 * gi + b] - cam.t0[b]);
    }
    bs vms[3], uc[3];
    for (int b = 0; b < 3; ++b) vms[b] = bs_sub(bs_cst(v[b]), cf.s[b]);
    for (int a = 0; a < 3; ++a) {
        uc[a] = bs_mul(cf.Rd[a], vms[0]);
        uc[a] = bs_add(uc[a], bs_mul(cf.Rd[3 + a], vms[1]));
        uc[a] = bs_add(uc[a], bs_mul(cf.Rd[6 + a], vms[2]));
    }
    bs d = uc[2];
    bs Mc[9];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            bs s = bs_scale(cf.Rd[a], N[c]);
            s = bs_add(s, bs_scale(cf.Rd[3 + a], N[3 + c]));
            s = bs_add(s, bs_scale(cf.Rd[6 + a], N[6 + c]));
            Mc[3 * a + c] = s;
        }
    bs J00 = bs_scale(d, cam.fx), J02 = bs_scale(uc[0], -cam.fx);
    bs J11 = bs_scale(d, cam.fy), J12 = bs_scale(uc[1], -cam.fy);
    bs Mp[6];
    for (int c = 0; c < 3; ++c) {
        Mp[c] = bs_add(bs_mul(J00, Mc[c]), bs_mul(J02, Mc[6 + c]));
        Mp[3 + c] = bs_add(bs_mul(J11, Mc[3 + c]), bs_mul(J12, Mc[6 + c]));
    }
    bs X[4];
    X[0] = bs_add(bs_add(bs_sq(Mp[0]), bs_sq(Mp[1])), bs_sq(Mp[2]));
    X[3] = bs_add(bs_add(bs_sq(Mp[3]), bs_sq(Mp[4])), bs_sq(Mp[5]));
    X[1] = bs_add(bs_add(bs_mul(Mp[0], Mp[3]), bs_mul(Mp[1], Mp[4])), bs_mul(Mp[2], Mp[5]));
    X[2] = X[1];
    out[0] = bs_min(&X[0]); out[1] = bs_max(&X[0]); out[2] = bs_min(&X[1]); out[3] = bs_max(&X[1]);
    out[4] = bs_min(&X[3]); out[5] = bs_max(&X[3]);
    double Xh[4];
    for (int e = 0; e < 4; ++e) Xh[e] = 0.5 * (bs_min(&X[e]) + bs_max(&X[e]));
    double det = Xh[0] * Xh[3] - Xh[1] * Xh[2];
    double X0[4] = {Xh[3] / det, -Xh[1] / det, -Xh[2] / det, Xh[0] / det};
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) {
            bs v2 = bs_add(bs_scale(X[2 * r], X0[s]), bs_scale(X[2 * r + 1], X0[2 + s]));
            bs E = bs_addc(bs_scale(v2, -1.0), r == s ? 1.0 : 0.0);
            out[6 + 2 * (2 * r + s)] = bs_min(&E); out[7 + 2 * (2 * r + s)] = bs_max(&E);
        }
    for (int e = 0; e < 6; ++e) { out[14 + 2 * e] = bs_min(&Mp[e]); out[15 + 2 * e] = bs_max(&Mp[e]); }
    bs C[4];
    double rho;
    if (matrix_inv(X, 0, C, &rho, NULL)) return 2;
    for (int e = 0; e < 4; ++e) { out[26 + 2 * e] = bs_min(&C[e]); out[27 + 2 * e] = bs_max(&C[e]); }
    out[34] = rho;
    return 0;
}
