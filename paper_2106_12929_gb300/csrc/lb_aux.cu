// Stencil-independent kernels of liblb: the second pass of the deterministic
// FP64 global sums, strided type-converting copies, and the Adam update.
#include "lb_ops.cuh"

namespace lb {

// Sum partials[b][k] over b for k < width, in block order per thread and a fixed
// tree across threads: the result depends only on the partials, not on timing.
__global__ void __launch_bounds__(256) k_reduce_final(const double* partials, int64_t nblocks, int width,
                                                      double* out)
{
    __shared__ double sh[256];
    for (int k = 0; k < width; ++k) {
        double s = 0.0;
        for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[b * width + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

cudaError_t reduce_final(const double* partials, int64_t nblocks, int width, double* out, cudaStream_t s)
{
    k_reduce_final<<<1, 256, 0, s>>>(partials, nblocks, width, out);
    return cudaGetLastError();
}

// dst[r * dst_stride + j] (+)= src[r * src_stride + j], j < n, r < rows, with
// FP64/FP32 conversion on the way.
__global__ void k_convert_copy(const void* src, int src_f64, void* dst, int dst_f64, int64_t n, int64_t ss,
                               int64_t ds, int accumulate)
{
    const int r = blockIdx.y;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double v = src_f64 ? ((const double*)src)[r * ss + j] : (double)((const float*)src)[r * ss + j];
        if (dst_f64) {
            double* d = (double*)dst + r * ds + j;
            *d = accumulate ? *d + v : v;
        } else {
            float* d = (float*)dst + r * ds + j;
            *d = accumulate ? *d + (float)v : (float)v;
        }
    }
}

cudaError_t convert_copy(const void* src, int src_f64, void* dst, int dst_f64, int64_t n, int64_t src_stride,
                         int64_t dst_stride, int rows, int accumulate, cudaStream_t s)
{
    if (n <= 0 || rows <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_convert_copy<<<dim3((unsigned)blocks, rows), 256, 0, s>>>(src, src_f64, dst, dst_f64, n, src_stride,
                                                                dst_stride, accumulate);
    return cudaGetLastError();
}

__global__ void k_adam(float* theta, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const float gj = g[j];
        const float mj = b1 * m[j] + (1.f - b1) * gj;
        const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
        m[j] = mj;
        v[j] = vj;
        theta[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
    }
}

cudaError_t adam_update(float* theta, float* m, float* v, const float* grad, int64_t n, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(theta, m, v, grad, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace lb
