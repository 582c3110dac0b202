// fma_probe.cu -- FP32 FMA throughput of the current device, the measured
// companion of the nominal FP32 peak (SMs x 128 lanes x 2 flops x clock) that
// the render kernel's roofline is quoted against.  A benchmark helper built as
// its own library (libarprobe.so): it is not part of libar or of the
// rendering path.
//
// Every thread runs 16 independent FMA chains (scalar __fmaf_rn, or pairs
// through the packed __ffma2_rn of sm_100 and later), so the FMA pipe, not a
// dependency, sets the rate; a grid of 8 blocks of 256 threads per SM keeps
// every scheduler busy.
#include <cuda_runtime.h>
#include <stdint.h>

namespace arprobe {

template <bool PACKED>
__global__ void __launch_bounds__(256) fma_rate_kernel(float *out, float b, float c, int iters)
{
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
        if (PACKED) {
            const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float2 v = __ffma2_rn(make_float2(a[k], a[k + 1]), bb, cc);
                a[k] = v.x;
                a[k + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = __fmaf_rn(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

static int fma_rate(int packed, int iters, double *tflops, cudaStream_t st)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    const int blocks = sms * 8, threads = 256;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int r = 1;
    float ms = 0.f;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaEventRecord(e0, st);
        if (packed) fma_rate_kernel<true><<<blocks, threads, 0, st>>>(out, 0.999999f, 1e-3f, iters);
        else fma_rate_kernel<false><<<blocks, threads, 0, st>>>(out, 0.999999f, 1e-3f, iters);
        cudaEventRecord(e1, st);
        if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            *tflops = 2.0 * 16.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
            r = 0;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return r;
}

}  // namespace arprobe

// TFLOP/s (an FMA counts as 2 flops) of 16 independent FMA chains per thread
// over 8 blocks of 256 threads per SM, iters steps each, timed with CUDA
// events on stream; packed = 1 issues them in pairs.  Returns 0, or 1 for bad
// arguments or a CUDA error.  Synchronises with stream; allocates and frees a
// small device buffer.
extern "C" int arprobe_fp32_fma_rate(int32_t packed, int32_t iters, double *tflops, void *stream)
{
    if (!tflops || iters < 1) return 1;
    return arprobe::fma_rate(packed, iters, tflops, (cudaStream_t)stream);
}
