// k_union.cu -- union of the bounds of several pose cells.  Sec. 5 partitions
// the camera set into subsets, bounds each, and joins the bounds: the lower
// bound of the whole set is the elementwise minimum of the subsets' lower
// bounds, the upper bound the maximum of their upper bounds.
//
// HBM-bound: every element of every cell is read once, the joined images are
// written once.  Consecutive threads take consecutive 16-byte groups of one
// image position, looping over the cells, so every load instruction of a warp
// reads 512 contiguous bytes of one cell's image.
#include "ar_launch.h"

namespace ar {

// min and max that return NaN when either operand is NaN (fminf and fmaxf
// return the other operand): a NaN bound of any piece, which would mean an
// unsound piece, reaches the joined image instead of being hidden by the
// other pieces' finite bounds
__device__ __forceinline__ float min_nan(float a, float b) { return (a != a || b != b) ? __int_as_float(0x7fc00000) : fminf(a, b); }
__device__ __forceinline__ float max_nan(float a, float b) { return (a != a || b != b) ? __int_as_float(0x7fc00000) : fmaxf(a, b); }

__device__ __forceinline__ float4 min4(float4 a, float4 b)
{
    return make_float4(min_nan(a.x, b.x), min_nan(a.y, b.y), min_nan(a.z, b.z), min_nan(a.w, b.w));
}
__device__ __forceinline__ float4 max4(float4 a, float4 b)
{
    return make_float4(max_nan(a.x, b.x), max_nan(a.y, b.y), max_nan(a.z, b.z), max_nan(a.w, b.w));
}

// n4 groups of four floats per cell; acc: fold the current outputs in too
__global__ void __launch_bounds__(256) bounds_union4_kernel(const float4 *__restrict__ lo, const float4 *__restrict__ hi,
                                                            int n_cells, size_t n4, float4 *__restrict__ out_lo,
                                                            float4 *__restrict__ out_hi, int acc)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n4; j += stride) {
        float4 a = acc ? out_lo[j] : lo[j];
        float4 b = acc ? out_hi[j] : hi[j];
        int c = acc ? 0 : 1;
#pragma unroll 4
        for (; c < n_cells; ++c) {
            a = min4(a, lo[(size_t)c * n4 + j]);
            b = max4(b, hi[(size_t)c * n4 + j]);
        }
        out_lo[j] = a;
        out_hi[j] = b;
    }
}

// the same one float at a time (sizes or addresses not 16-byte multiples)
__global__ void __launch_bounds__(256) bounds_union1_kernel(const float *__restrict__ lo, const float *__restrict__ hi,
                                                            int n_cells, size_t n, float *__restrict__ out_lo,
                                                            float *__restrict__ out_hi, int acc)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        float a = acc ? out_lo[j] : lo[j];
        float b = acc ? out_hi[j] : hi[j];
        int c = acc ? 0 : 1;
#pragma unroll 4
        for (; c < n_cells; ++c) {
            a = min_nan(a, lo[(size_t)c * n + j]);
            b = max_nan(b, hi[(size_t)c * n + j]);
        }
        out_lo[j] = a;
        out_hi[j] = b;
    }
}

int launch_bounds_union(const float *lo, const float *hi, int n_cells, size_t n, float *out_lo, float *out_hi,
                        bool acc, cudaStream_t st)
{
    if (n == 0 || n_cells < 1) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    const bool vec = n % 4 == 0 && ((uintptr_t)lo | (uintptr_t)hi | (uintptr_t)out_lo | (uintptr_t)out_hi) % 16 == 0;
    const size_t units = vec ? n / 4 : n;
    const size_t want = (units + 255) / 256, cap = (size_t)sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (vec)
        bounds_union4_kernel<<<grid, 256, 0, st>>>((const float4 *)lo, (const float4 *)hi, n_cells, units,
                                                   (float4 *)out_lo, (float4 *)out_hi, acc ? 1 : 0);
    else
        bounds_union1_kernel<<<grid, 256, 0, st>>>(lo, hi, n_cells, n, out_lo, out_hi, acc ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// out = out intersected with [lo, hi]: the larger lower and the smaller upper bound
__global__ void __launch_bounds__(256) bounds_intersect_kernel(const float *__restrict__ lo,
                                                               const float *__restrict__ hi, size_t n,
                                                               float *__restrict__ out_lo, float *__restrict__ out_hi)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        out_lo[j] = max_nan(out_lo[j], lo[j]);
        out_hi[j] = min_nan(out_hi[j], hi[j]);
    }
}

// partial sums of (hi - lo) over each cell's n floats: block (b, c) sums the
// elements b, b + B, ... of cell c (B = gridDim.x blocks) into part[c B + b]
__global__ void __launch_bounds__(256) width_partials_kernel(const float *__restrict__ lo,
                                                             const float *__restrict__ hi, size_t n,
                                                             double *__restrict__ part)
{
    __shared__ double s_sum[256];
    const size_t c = blockIdx.y;
    const float *l = lo + c * n, *h = hi + c * n;
    double acc = 0.0;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
        acc += (double)h[j] - (double)l[j];
    s_sum[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = s_sum[0];
}

int launch_bounds_intersect(const float *lo, const float *hi, size_t n, float *out_lo, float *out_hi, cudaStream_t st)
{
    if (n == 0) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    const size_t want = (n + 255) / 256, cap = (size_t)sms * 8;
    bounds_intersect_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(lo, hi, n, out_lo, out_hi);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int launch_width_partials(const float *lo, const float *hi, int n_cells, size_t n, int blocks, double *part,
                          cudaStream_t st)
{
    if (n_cells < 1 || blocks < 1) return 0;
    width_partials_kernel<<<dim3((unsigned)blocks, (unsigned)n_cells), 256, 0, st>>>(lo, hi, n, part);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace ar
