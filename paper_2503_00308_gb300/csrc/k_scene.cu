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

// v = R_wc (uw - t), N = R_wc Mw for the call's nominal camera.
__global__ void pose_prep_kernel(const float *__restrict__ uw, const double *__restrict__ Mw, int64_t n,
                                 CallConst cc, double *__restrict__ vN)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *o = vN + 12 * i;
    for (int a = 0; a < 3; ++a) {
        double s = 0;
        for (int b = 0; b < 3; ++b) s = dadd(s, dmul(cc.R0[3 * a + b], dsub((double)uw[3 * i + b], cc.t0[b])));
        o[a] = s;
    }
    mat3(cc.R0, Mw + 9 * i, o + 3);
}

int launch_scene_prep(const float *logscale, const float *quat, const float *opacity, int64_t n, double *Mw,
                      double *tau, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int T = 128;
    scene_prep_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(logscale, quat, opacity, n, Mw, tau);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_pose_prep(const float *uw, const double *Mw, int64_t n, const CallConst &cc, double *vN, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int T = 128;
    pose_prep_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(uw, Mw, n, cc, vN);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace ar
