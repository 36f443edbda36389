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

// Bandwidth reference: dst <- src in 16-byte vectors, four loads in flight per thread before
// their stores, over a grid-stride loop.
__global__ void __launch_bounds__(256) k_stream_copy(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

cudaError_t stream_copy(const void* src, void* dst, int64_t bytes, int sms, cudaStream_t s)
{
    const int64_t n = bytes / 16;
    int64_t blocks = (int64_t)(sms > 0 ? sms : 1) * 16;  // two rounds of resident blocks: measured best
    const int64_t need = (n + 255) / 256;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaSuccess;
    k_stream_copy<<<(unsigned)blocks, 256, 0, s>>>((const uint4*)src, (uint4*)dst, n);
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

// Block average by 2 in every axis of a grid with even extents: per coarse node the
// mean density and the mean momentum of its 2^d fine nodes; u_c = mean(rho u) / mean(rho).
// Fine and coarse arrays are FP64, component-major, x fastest.
__global__ void k_coarsen2(const double* rho_f, const double* u_f, int nxf, int nyf, int nzf, int d, double* rho_c,
                           double* u_c)
{
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf > 1 ? nzf / 2 : 1;
    const int64_t Nc = (int64_t)nxc * nyc * nzc, Nf = (int64_t)nxf * nyf * nzf;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nc; n += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(n % nxc), Y = (int)((n / nxc) % nyc), Z = (int)(n / ((int64_t)nxc * nyc));
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        const int zc = nzf > 1 ? 2 : 1;
        for (int c = 0; c < zc; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int64_t m = (2 * X + a) + (int64_t)nxf * ((2 * Y + b) + (int64_t)nyf * (zc * Z + c));
                    const double rf = rho_f[m];
                    r += rf;
                    for (int k = 0; k < d; ++k) j[k] += rf * u_f[k * Nf + m];
                }
        rho_c[n] = r / (double)(4 * zc);
        for (int k = 0; k < d; ++k) u_c[k * Nc + n] = j[k] / r;
    }
}

cudaError_t coarsen2(const double* rho_f, const double* u_f, int nxf, int nyf, int nzf, int d, double* rho_c,
                     double* u_c, cudaStream_t s)
{
    const int64_t Nc = (int64_t)(nxf / 2) * (nyf / 2) * (nzf > 1 ? nzf / 2 : 1);
    int64_t blocks = (Nc + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_coarsen2<<<(unsigned)blocks, 256, 0, s>>>(rho_f, u_f, nxf, nyf, nzf, d, rho_c, u_c);
    return cudaGetLastError();
}

// 2D vorticity w = (v(x+1) - v(x-1))/2 - (u(y+1) - u(y-1))/2 of a velocity field u[2][N]
// (FP64) on a periodic nx x ny grid, written as FP64 or FP32.
__global__ void k_vorticity2d(const double* u, int nx, int ny, void* w, int w_f64)
{
    const int64_t N = (int64_t)nx * ny;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)(n / nx);
        const int xp = x == nx - 1 ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
        const int yp = y == ny - 1 ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
        const double v = 0.5 * (u[N + xp + (int64_t)nx * y] - u[N + xm + (int64_t)nx * y]) -
                         0.5 * (u[x + (int64_t)nx * yp] - u[x + (int64_t)nx * ym]);
        if (w_f64) ((double*)w)[n] = v;
        else ((float*)w)[n] = (float)v;
    }
}

cudaError_t vorticity2d(const double* u, int nx, int ny, void* w, int w_f64, cudaStream_t s)
{
    const int64_t N = (int64_t)nx * ny;
    int64_t blocks = (N + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_vorticity2d<<<(unsigned)blocks, 256, 0, s>>>(u, nx, ny, w, w_f64);
    return cudaGetLastError();
}

}  // namespace lb
