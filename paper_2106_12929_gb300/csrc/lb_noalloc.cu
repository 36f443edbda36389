// lb_reduce_noalloc: the global FP64 sums of lb_reduce for a caller-owned
// population array, with no device allocation of any kind.
//
// Some callers cannot allocate device memory at the point where they need these
// sums: code that has handed the whole device to another framework's caching
// allocator (a foreign cudaMalloc may fail or fragment its pool), and
// latency-critical loops where cudaMalloc / cudaFree are not acceptable because
// they can synchronise the whole device. This entry point needs no context and
// allocates nothing: the inputs and the host output belong to the caller, and the
// per-block partial sums live in a fixed file-scope device array.
//
// The scratch array is static device memory of this library: every GPU that loads
// the library holds it (kScratchDoubles doubles, about 385 KB) until the process
// exits. Its address is looked up once per device (cudaGetSymbolAddress) by the
// first call on that device, with that device current; make that first call before
// any stream capture. The looked-up address is kept for the life of the process, so
// it does not survive a cudaDeviceReset of that device: do not call this entry point
// on a device after resetting it. All calls share the array and it keeps the last call's
// contents; every word a call reads was written earlier in the same call (each
// block overwrites its partial slot, the final pass overwrites the result slot), so
// nothing has to be cleared. Calls whose work overlaps on the GPU (different
// streams, or different host threads on the same device) race on the array; the
// caller must order them.
#include <cuda_runtime.h>

#include <mutex>

#include "lb.h"
#include "lb_collide.cuh"
#include "lb_ops.cuh"

namespace lb {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNodesPerThread = 16;
constexpr int64_t kNodesPerBlock = (int64_t)kNoallocThreads * kNodesPerThread;  // 4096
constexpr int64_t kMaxBlocks = 8192;
constexpr int64_t kMaxNodes = kMaxBlocks * kNodesPerBlock;  // 33,554,432 nodes (e.g. 320^3)
constexpr int kWidth = 6;
constexpr int64_t kScratchDoubles = kMaxBlocks * kWidth + 8;  // partials + final sums

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Pass 1: block b sums the moments of nodes [b * 4096, (b + 1) * 4096) into
// scratch[b * 6 .. b * 6 + 5]; populations are in natural layout f[i][n], n < N.
template <class St, class T, bool FORCE>
__global__ void __launch_bounds__(kNoallocThreads) k_noalloc_partial(const T* f, const T* F, Geom g, int64_t N,
                                                                     double* scratch)
{
    using R = typename Store<T>::Real;
    double v[kWidth] = {0, 0, 0, 0, 0, 0};
    const int64_t first = (int64_t)blockIdx.x * kNodesPerBlock;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const int64_t n = first + (int64_t)k * kNoallocThreads + threadIdx.x;
        if (n >= N) break;
        R d[St::Q];
#pragma unroll
        for (int i = 0; i < St::Q; ++i) d[i] = (R)f[(int64_t)i * N + n] - R(St::w(i));  // caller's f, unshifted
        R Fl[3] = {R(0), R(0), R(0)};
        if constexpr (FORCE) {
            Fl[0] = F[n];
            Fl[1] = F[N + n];
            if (St::D == 3) Fl[2] = F[2 * N + n];
        }
        const NodeMoments<St, R> m = node_moments<St, FORCE>(d, Fl);
        const double r = m.rho, ux = m.ux, uy = m.uy, uz = m.uz, uu = ux * ux + uy * uy + uz * uz;
        v[0] += r;
        v[1] += r * ux;
        v[2] += r * uy;
        v[3] += r * uz;
        v[4] += uu;
        v[5] += r * uu;
    }
    __shared__ double sh[kWidth][kNoallocThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < kWidth; ++w) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[w] += __shfl_down_sync(0xffffffffu, v[w], o);
        if (lane == 0) sh[w][warp] = v[w];
    }
    __syncthreads();
    if (threadIdx.x < kWidth) {
        double s = 0.0;
        for (int w = 0; w < kNoallocThreads / 32; ++w) s += sh[threadIdx.x][w];
        scratch[(int64_t)blockIdx.x * kWidth + threadIdx.x] = s;
    }
}

// Pass 2: one block adds the partials in block order and writes the six results
// to scratch[kMaxBlocks * 6 ..], scaled like lb_reduce.
__global__ void __launch_bounds__(kNoallocThreads) k_noalloc_final(double* scratch, int64_t nblocks, int64_t N)
{
    __shared__ double sh[kNoallocThreads];
    for (int w = 0; w < kWidth; ++w) {
        double s = 0.0;
        for (int64_t b = threadIdx.x; b < nblocks; b += kNoallocThreads) s += scratch[b * kWidth + w];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = kNoallocThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[kMaxBlocks * kWidth + w] = (w >= 4) ? 0.5 * sh[0] / (double)N : sh[0];
        __syncthreads();
    }
}

template <class St, class T>
cudaError_t launch_noalloc(const void* f, const void* F, const Geom& g, int64_t N, double* scratch, cudaStream_t s)
{
    const int64_t nblocks = (N + kNodesPerBlock - 1) / kNodesPerBlock;
    if (F)
        k_noalloc_partial<St, T, true><<<(unsigned)nblocks, kNoallocThreads, 0, s>>>((const T*)f, (const T*)F, g, N,
                                                                                      scratch);
    else
        k_noalloc_partial<St, T, false><<<(unsigned)nblocks, kNoallocThreads, 0, s>>>((const T*)f, nullptr, g, N,
                                                                                       scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_noalloc_final<<<1, kNoallocThreads, 0, s>>>(scratch, nblocks, N);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lb

extern "C" lb_status lb_reduce_noalloc(lb_stencil stencil, const int64_t dims[3], const void* f, const void* F,
                                       lb_mem mem, double out[6], void* cuda_stream)
{
    using namespace lb;
    auto reject = [](lb_status st, const char* msg) {
        set_last_error(msg);
        return st;
    };
    if (!dims || !f || !out) return reject(LB_ERR_ARG, "lb_reduce_noalloc: dims, f and out are required");
    if ((int)stencil < 0 || (int)stencil > 2) return reject(LB_ERR_ARG, "lb_reduce_noalloc: unknown stencil");
    if (mem != LB_DEVICE_F64 && mem != LB_DEVICE_F32)
        return reject(LB_ERR_ARG, "lb_reduce_noalloc: f (and F) must be device arrays (LB_DEVICE_F64 or LB_DEVICE_F32)");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > 65535) return reject(LB_ERR_ARG, "lb_reduce_noalloc: dims out of [1, 65535]");
    if (stencil == LB_D2Q9 && dims[2] != 1) return reject(LB_ERR_ARG, "lb_reduce_noalloc: 2D stencil needs dims[2] == 1");
    const int64_t N = dims[0] * dims[1] * dims[2];
    if (N > kMaxNodes)  // the scratch array holds the partials of at most 8192 blocks of 4096 nodes
        return reject(LB_ERR_ARG, "lb_reduce_noalloc: more than 33,554,432 nodes (its fixed scratch array holds the "
                                  "partial sums of at most 8192 blocks of 4096 nodes)");
    // f and F must be memory the current device can read: a host pointer or another
    // device's allocation passed with a device code would make the kernel fault.
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return reject(LB_ERR_CUDA, "lb_reduce_noalloc: cudaGetDevice failed");
    for (const void* p : {f, F}) {
        if (!p) continue;
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
            cudaGetLastError();  // clear the (non-sticky) error the failed query recorded
            return reject(LB_ERR_ARG, "lb_reduce_noalloc: f or F is not a CUDA pointer");
        }
        const bool readable = (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) &&
                              attr.device == cur;
        if (!readable)
            return reject(LB_ERR_ARG, "lb_reduce_noalloc: f and F must be device (or managed) memory of the current "
                                      "device");
    }
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess)
        return reject(LB_ERR_CUDA, "lb_reduce_noalloc: cudaGetSymbolAddress of the scratch array failed");
    Geom g;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = (int)dims[2];
    g.plane = N;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e;
    const bool f64 = mem == LB_DEVICE_F64;
    switch (stencil) {
    case LB_D2Q9: e = f64 ? launch_noalloc<D2Q9, double>(f, F, g, N, scratch, s) : launch_noalloc<D2Q9, float>(f, F, g, N, scratch, s); break;
    case LB_D3Q19: e = f64 ? launch_noalloc<D3Q19, double>(f, F, g, N, scratch, s) : launch_noalloc<D3Q19, float>(f, F, g, N, scratch, s); break;
    default: e = f64 ? launch_noalloc<D3Q27, double>(f, F, g, N, scratch, s) : launch_noalloc<D3Q27, float>(f, F, g, N, scratch, s); break;
    }
    if (e != cudaSuccess) return reject(LB_ERR_CUDA, "lb_reduce_noalloc: kernel launch failed");
    e = cudaMemcpyAsync(out, scratch + kMaxBlocks * kWidth, kWidth * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return reject(LB_ERR_CUDA, "lb_reduce_noalloc: copying the sums to the host failed");
    return LB_OK;
}
