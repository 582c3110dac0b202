// k_scene.cu -- per-scene and per-call preprocessing of the Gaussians.
#include "ar_launch.h"
#include "k_prep.cuh"

namespace ar {

// Mw (row-major 3x3, FP64) and tau per Gaussian.
__global__ void scene_prep_kernel(const float *__restrict__ logscale, const float *__restrict__ quat,
                                  const float *__restrict__ opacity, int64_t n, double *__restrict__ Mw,
                                  double *__restrict__ tau)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double R[9];
    quat_rot(quat + 4 * i, R);
    double e[3];
    for (int j = 0; j < 3; ++j) e[j] = exp((double)logscale[3 * i + j]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Mw[9 * i + 3 * a + b] = dmul(R[3 * a + b], e[b]);
    double o = opacity[i];
    tau[i] = (o > 0) ? dmul(2.0, log(dmul(255.0, o))) : -INFINITY;
}

// v = R_wc (uw - t) as an interval over the mean's box [uw_lo, uw_hi] (each
// product at the end of the box its sign selects; lo = hi without a box),
// and N = R_wc Mw, for the call's nominal camera: VN_STRIDE doubles each.
__global__ void pose_prep_kernel(const float *__restrict__ uw_lo, const float *__restrict__ uw_hi,
                                 const double *__restrict__ Mw, int64_t n, CallConst cc, double *__restrict__ vN)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *o = vN + VN_STRIDE * i;
    for (int a = 0; a < 3; ++a) {
        double sl = 0, sh = 0;
        for (int b = 0; b < 3; ++b) {
            const double r = cc.R0[3 * a + b];
            const double dl = dsub((double)uw_lo[3 * i + b], cc.t0[b]), dh = dsub((double)uw_hi[3 * i + b], cc.t0[b]);
            sl = dadd(sl, dmul(r, r >= 0 ? dl : dh));
            sh = dadd(sh, dmul(r, r >= 0 ? dh : dl));
        }
        o[a] = sl;
        o[3 + a] = sh;
    }
    mat3(cc.R0, Mw + 9 * i, o + 6);
    float *enc = reinterpret_cast<float *>(o + VN_ENC);
    for (int k = 0; k < VN_ENC; ++k) {
        enc[2 * k] = __double2float_rd(o[k]);
        enc[2 * k + 1] = __double2float_ru(o[k]);
    }
}

// The GParam of every Gaussian from its opacity and colour boxes.
__global__ void gparam_kernel(const float *__restrict__ o_lo, const float *__restrict__ o_hi,
                              const float *__restrict__ c_lo, const float *__restrict__ c_hi, int64_t n,
                              GParam *__restrict__ gp)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    GParam P;
    P.o_lo = o_lo[i];
    P.o_hi = o_hi[i];
    const double a = P.o_lo, b = P.o_hi;
    P.tau_lo = (a > 0) ? dmul(2.0, log(dmul(255.0, a))) : -INFINITY;
    P.tau_hi = (b > 0) ? dmul(2.0, log(dmul(255.0, b))) : -INFINITY;
    for (int k = 0; k < 3; ++k) {
        P.c_lo[k] = c_lo[3 * i + k];
        P.c_hi[k] = c_hi[3 * i + k];
    }
    gp[i] = P;
}

int launch_scene_prep(const float *logscale, const float *quat, const float *opacity, int64_t n, double *Mw,
                      double *tau, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int T = 128;
    scene_prep_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(logscale, quat, opacity, n, Mw, tau);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_pose_prep(const float *uw_lo, const float *uw_hi, const double *Mw, int64_t n, const CallConst &cc,
                     double *vN, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int T = 128;
    pose_prep_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(uw_lo, uw_hi, Mw, n, cc, vN);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_gparam(const float *o_lo, const float *o_hi, const float *c_lo, const float *c_hi, int64_t n, void *gp,
                  cudaStream_t st)
{
    if (n <= 0) return 0;
    const int T = 128;
    gparam_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(o_lo, o_hi, c_lo, c_hi, n, (GParam *)gp);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace ar
