// k_concrete.cu -- the concrete GSplat render (Algorithm 1, blended as in
// BlendInd, Algorithm 4) at sampled poses, in FP64, for soundness checks of
// the abstract bounds on the device.
//
// Per pose: concrete_pose_kernel builds R_wc(delta) and t; concrete_prep_kernel
// projects every Gaussian (d, up, Mp, X, Conic, W = Conic Mp, the pixel box
// of the ellipse m <= tau, the near plane and the frustum guard band); the
// Gaussians are binned into depth-ordered tile lists by the abstract
// renderer's binning (each Gaussian gives two events with equal keys, the
// second ignored); concrete_render_kernel blends each pixel front to back,
// Gaussians of equal depth as one group (Ind(0) = 0), until the transmittance
// is below CONC_T_STOP, which bounds the colour left out.
#include "ar_common.cuh"
#include "ar_launch.h"
#include "k_prep.cuh"

namespace ar {

constexpr double CONC_T_STOP = 1e-13;

// record: d, up0, up1, W0c (3), W1c (3), o, tau, c0, c1, c2, pad (16 doubles)
constexpr int CR_D = 0, CR_UP = 1, CR_W0 = 3, CR_W1 = 6, CR_O = 9, CR_TAU = 10, CR_COL = 11, CR_WIDTH = 16;

struct ConcretePose {
    double Rwc[9];
    double t[3];
};

// R_wc(delta) = R_delta^T R0 with R_delta = Rx Ry Rz, t = t0 + delta_t
__global__ void concrete_pose_kernel(const double *__restrict__ delta, CallConst cc, ConcretePose *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double X[9], Y[9], Z[9], D[9], T[9], Rd[9], RdT[9];
    rot3(0, delta[3], X, D);
    rot3(1, delta[4], Y, D);
    rot3(2, delta[5], Z, D);
    mat3(X, Y, T);
    mat3(T, Z, Rd);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RdT[3 * i + j] = Rd[3 * j + i];
    mat3(RdT, cc.R0, out->Rwc);
    for (int k = 0; k < 3; ++k) out->t[k] = dadd(cc.t0[k], delta[k]);
}

// One thread per Gaussian.  counters: [2] Gaussians present, [3] tile entries.
__global__ void __launch_bounds__(128) concrete_prep_kernel(
    const float *__restrict__ uw, const double *__restrict__ Mw, const double *__restrict__ tau_g,
    const float *__restrict__ opacity, const float *__restrict__ rgb, CallConst cc,
    const ConcretePose *__restrict__ pose, int TS, double *__restrict__ recs, PixBox *__restrict__ boxes,
    double *__restrict__ keys, unsigned long long *__restrict__ counters)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    uint32_t valid = 0, tiles = 0;
    if (g < cc.n_gauss) {
        PixBox box = {-1, -1, -1, -1};
        const double *Rwc = pose->Rwc;
        double uc[3], Mc[9];
        for (int a = 0; a < 3; ++a) {
            const double d0 = dsub((double)uw[3 * g], pose->t[0]);
            const double d1 = dsub((double)uw[3 * g + 1], pose->t[1]);
            const double d2 = dsub((double)uw[3 * g + 2], pose->t[2]);
            uc[a] = dadd(dadd(dmul(Rwc[3 * a], d0), dmul(Rwc[3 * a + 1], d1)), dmul(Rwc[3 * a + 2], d2));
        }
        mat3(Rwc, Mw + 9 * g, Mc);
        const double d = uc[2];
        const double o = opacity[g], tau = tau_g[g];
        const double up0 = dadd(dmul((double)cc.fx, uc[0]), dmul((double)cc.cx, d));
        const double up1 = dadd(dmul((double)cc.fy, uc[1]), dmul((double)cc.cy, d));
        // J = [[fx d, 0, -fx uc0], [0, fy d, -fy uc1]] (d^2 times the projection Jacobian)
        const double J[6] = {dmul((double)cc.fx, d), 0.0, dmul(-(double)cc.fx, uc[0]),
                             0.0, dmul((double)cc.fy, d), dmul(-(double)cc.fy, uc[1])};
        double Mp[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                Mp[3 * r + c] = dadd(dadd(dmul(J[3 * r], Mc[c]), dmul(J[3 * r + 1], Mc[3 + c])),
                                     dmul(J[3 * r + 2], Mc[6 + c]));
        double X[4];
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s)
                X[2 * r + s] = dadd(dadd(dmul(Mp[3 * r], Mp[3 * s]), dmul(Mp[3 * r + 1], Mp[3 * s + 1])),
                                    dmul(Mp[3 * r + 2], Mp[3 * s + 2]));
        const double det = dsub(dmul(X[0], X[3]), dmul(X[1], X[2]));
        bool alive = (d > (double)cc.near_plane) && (det > 0) && (o > 0) && (tau >= 0);
        double mux = 0, muy = 0;
        if (alive) {
            // frustum guard band (3DGS convention)
            const double gx = dmul(GUARD, (double)cc.W), gy = dmul(GUARD, (double)cc.H);
            mux = dadd((double)cc.cx, dmul((double)cc.fx, uc[0]) / d);
            muy = dadd((double)cc.cy, dmul((double)cc.fy, uc[1]) / d);
            alive = mux >= dsub((double)cc.cx, gx) && mux <= dadd((double)cc.cx, gx) &&
                    muy >= dsub((double)cc.cy, gy) && muy <= dadd((double)cc.cy, gy);
        }
        if (alive) {
            // pixel box of the ellipse m <= tau: half-extents sqrt(tau X_rr) / d^2
            const double d2 = dmul(d, d);
            const double rx = sqrt(dmul(tau, X[0])) / d2, ry = sqrt(dmul(tau, X[3])) / d2;
            double xl = dsub(mux, rx), xh = dadd(mux, rx), yl = dsub(muy, ry), yh = dadd(muy, ry);
            xl = dsub(xl, dmul(BOX_SLACK, dadd(1.0, fabs(xl))));
            xh = dadd(xh, dmul(BOX_SLACK, dadd(1.0, fabs(xh))));
            yl = dsub(yl, dmul(BOX_SLACK, dadd(1.0, fabs(yl))));
            yh = dadd(yh, dmul(BOX_SLACK, dadd(1.0, fabs(yh))));
            double fx0 = fmax(ceil(dsub(xl, 0.5)), 0.0), fx1 = fmin(floor(dsub(xh, 0.5)), (double)(cc.W - 1));
            double fy0 = fmax(ceil(dsub(yl, 0.5)), 0.0), fy1 = fmin(floor(dsub(yh, 0.5)), (double)(cc.H - 1));
            if (xh >= xl && yh >= yl && fx0 <= fx1 && fy0 <= fy1) {
                box = PixBox{(int)fx0, (int)fx1, (int)fy0, (int)fy1};
                const double conic[4] = {X[3] / det, -X[1] / det, -X[2] / det, X[0] / det};
                double *rec = recs + g * CR_WIDTH;
                rec[CR_D] = d;
                rec[CR_UP] = up0;
                rec[CR_UP + 1] = up1;
                for (int c = 0; c < 3; ++c) {
                    rec[CR_W0 + c] = dadd(dmul(conic[0], Mp[c]), dmul(conic[1], Mp[3 + c]));
                    rec[CR_W1 + c] = dadd(dmul(conic[2], Mp[c]), dmul(conic[3], Mp[3 + c]));
                }
                rec[CR_O] = o;
                rec[CR_TAU] = tau;
                for (int k = 0; k < 3; ++k) rec[CR_COL + k] = rgb[3 * g + k];
                keys[2 * g] = d;
                keys[2 * g + 1] = d;
                valid = 1;
                tiles = (uint32_t)(box.x1 / TS - box.x0 / TS + 1) * (uint32_t)(box.y1 / TS - box.y0 / TS + 1);
            }
        }
        boxes[g] = box;
    }
    const uint32_t v = __reduce_add_sync(0xffffffffu, valid);
    const uint32_t e = __reduce_add_sync(0xffffffffu, tiles);
    if ((threadIdx.x & 31) == 0) {
        if (v) atomicAdd(&counters[2], (unsigned long long)v);
        if (e) atomicAdd(&counters[3], (unsigned long long)e);
    }
}

// One CTA per tile, one thread per pixel; out is [H][W][3] of this pose.
template <int TS>
__global__ void __launch_bounds__(TS *TS) concrete_render_kernel(
    const double *__restrict__ recs, const PixBox *__restrict__ boxes, const uint32_t *__restrict__ seg_start,
    const uint32_t *__restrict__ seg_end, const uint32_t *__restrict__ entry_ev, const uint32_t *__restrict__ ev_val,
    const uint64_t *__restrict__ ev_key, int W, int H, int ntx, float *__restrict__ out)
{
    constexpr int CH = 32, NT = TS * TS;
    __shared__ __align__(16) double s_rec[CH][CR_WIDTH];
    __shared__ uint32_t s_rid[CH], s_bits[CH];
    __shared__ PixBox s_box[CH];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int px = (tile % ntx) * TS + (tid % TS), py = (tile / ntx) * TS + (tid / TS);
    const bool inside = px < W && py < H;
    const double ux = px + 0.5, uy = py + 0.5;
    const uint32_t b0 = seg_start[tile], b1 = seg_end[tile];
    double T = 1.0, Tp = 1.0, pc[3] = {0.0, 0.0, 0.0};
    bool done = !inside;
    for (uint32_t base = b0; base < b1; base += CH) {
        if (!done && T < CONC_T_STOP) done = true;
        if (__syncthreads_and(done)) break;
        const int cnt = (int)min((uint32_t)CH, b1 - base);
        if (tid < cnt) {
            const uint32_t i = base + tid;
            const uint32_t e = entry_ev[i];
            const uint32_t v = ev_val[e];
            uint32_t bits = v & 1u;
            if (i > b0 && ev_key[entry_ev[i - 1]] == ev_key[e]) bits |= 2u;
            s_rid[tid] = v >> 1;
            s_bits[tid] = bits;
            s_box[tid] = boxes[v >> 1];
        }
        __syncthreads();
        for (int t = tid; t < cnt * (CR_WIDTH / 2); t += NT) {
            const int e = t / (CR_WIDTH / 2), q = t - e * (CR_WIDTH / 2);
            reinterpret_cast<double2 *>(s_rec[e])[q] =
                reinterpret_cast<const double2 *>(recs + (size_t)s_rid[e] * CR_WIDTH)[q];
        }
        __syncthreads();
        if (done) continue;
        for (int e = 0; e < cnt; ++e) {
            const uint32_t bits = s_bits[e];
            if (!(bits & 2u)) {  // a new depth: absorb the previous group
                T = dmul(T, Tp);
                Tp = 1.0;
            }
            if (bits & 1u) continue;  // the second event of a Gaussian
            const PixBox bx = s_box[e];
            if (px < bx.x0 || px > bx.x1 || py < bx.y0 || py > bx.y1) continue;
            const double *r = s_rec[e];
            const double d = r[CR_D];
            const double D0 = dsub(dmul(dmul(d, d), ux), dmul(d, r[CR_UP]));
            const double D1 = dsub(dmul(dmul(d, d), uy), dmul(d, r[CR_UP + 1]));
            double m = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double q = dadd(dmul(D0, r[CR_W0 + c]), dmul(D1, r[CR_W1 + c]));
                m = dadd(m, dmul(q, q));
            }
            if (m > r[CR_TAU]) continue;  // below the 1/255 cutoff
            const double a = dmul(r[CR_O], exp(dmul(-0.5, m)));
            const double Ta = dmul(T, a);
            for (int ch = 0; ch < 3; ++ch) pc[ch] = dadd(pc[ch], dmul(Ta, r[CR_COL + ch]));
            Tp = dmul(Tp, dsub(1.0, a));
        }
    }
    if (inside) {
        float *o = out + ((size_t)py * W + px) * 3;
        for (int ch = 0; ch < 3; ++ch) o[ch] = (float)fmin(1.0, fmax(0.0, pc[ch]));
    }
}

int launch_concrete_pose(const double *delta, const CallConst &cc, void *pose, cudaStream_t st)
{
    concrete_pose_kernel<<<1, 32, 0, st>>>(delta, cc, (ConcretePose *)pose);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
size_t concrete_pose_bytes() { return sizeof(ConcretePose); }
int concrete_rec_width() { return CR_WIDTH; }

int launch_concrete_prep(const float *uw, const double *Mw, const double *tau, const float *opac, const float *rgb,
                         const CallConst &cc, const void *pose, int TS, double *recs, PixBox *boxes, double *keys,
                         unsigned long long *counters, cudaStream_t st)
{
    const int T = 128;
    concrete_prep_kernel<<<(unsigned)((cc.n_gauss + T - 1) / T), T, 0, st>>>(
        uw, Mw, tau, opac, rgb, cc, (const ConcretePose *)pose, TS, recs, boxes, keys, counters);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_concrete_render(const double *recs, const PixBox *boxes, const uint32_t *seg_start, const uint32_t *seg_end,
                           const uint32_t *ent_ev, const uint32_t *ev_val, const uint64_t *ev_key, int W, int H,
                           int ntx, int n_tiles, float *out, cudaStream_t st)
{
    concrete_render_kernel<16><<<n_tiles, 256, 0, st>>>(recs, boxes, seg_start, seg_end, ent_ev, ev_val, ev_key, W, H,
                                                       ntx, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace ar
