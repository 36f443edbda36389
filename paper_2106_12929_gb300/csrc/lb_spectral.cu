// Spectral flow control (Sec. 3.2) on a periodic n x n D2Q9 grid, n = 2^logn.
//
// Every controlled step keeps the flow's energy spectrum near a target sigma_0 with the cost
//   R(u) = || ln max(sigma(u), c) - ln max(sigma_0, c) ||^2
// and collides with the equilibrium at the shifted velocity u + du, du = -kappa grad_u R.
// With U_a = sum_x u_a(x) exp(-2 pi i k.x / n) (unnormalised DFT), the spectrum is
//   sigma_s = sum over the modes k with round(|k|) = s < n/2 of (|U_x|^2 + |U_y|^2) / (2 N^2),
// and the chain rule through sigma and the DFT gives grad_u R as a spectral filter:
//   grad_u_a R(x) = Re sum_k G(k) U_a(k) exp(+2 pi i k.x / n) / N^2,
//   G(k) = dR/dsigma_s of k's shell s (0 outside the kept shells),
//   dR/dsigma_s = 2 (ln sigma_s - ln max(sigma0_s, c)) / sigma_s if sigma_s > c, else 0.
// A controlled step is five launches: rows (moments + forward DFT along x), columns (forward
// DFT along y, modal energies and per-column shell sums), shells (sigma and dR/dsigma, one
// warp per shell), columns (filter by G, inverse DFT along y; the cost R), rows (inverse DFT
// along x: du, then the shifted BGK step of the row's nodes). lb_spectral_shift writes du
// instead of stepping. Each DFT is an in-place radix-2 FFT of one grid line in shared
// memory, one block per line, in passes of three radix-2 stages held in registers (a padded
// layout keeps the passes free of bank conflicts), with a per-block twiddle table; both velocity
// components go through the same passes. Every sum runs in a fixed order (deterministic).
#include "lb_collide.cuh"
#include "lb_spectral.cuh"

namespace lb {

template <class R>
struct Cx {
    R re, im;
};

LB_DEV void sincos_pi(float x, float* s, float* c) { sincospif(x, s, c); }
LB_DEV void sincos_pi(double x, double* s, double* c) { sincospi(x, s, c); }

LB_DEV int bitrev(int v, int logn) { return (int)(__brev((unsigned)v) >> (32 - logn)); }

// Twiddle table tw[k] = exp(sign i 2 pi k / n), k < n/2 (block-wide; the caller syncs).
template <class R>
LB_DEV void twiddles(Cx<R>* tw, int n, R sign)
{
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        R s, c;
        sincos_pi(sign * R(2 * k) / R(n), &s, &c);
        tw[k] = {c, s};
    }
}

// Shared-memory position of element i of a line: one spare slot after every eight elements, so
// that the threads of a half-warp reading the sets of the first passes hit distinct banks.
LB_HD int pz(int i) { return i + (i >> 3); }
LB_HD int line_stride(int n) { return n + (n >> 3); }

// One pass of the in-place decimation-in-time FFT over the stages s .. s + RB - 1 of the two
// n-point lines z[0 ..) and z[line_stride(n) ..) (bit-reversed input order): those stages
// only combine elements within the sets {base + k h : k < 2^RB}, h = 2^s, so each thread loads
// whole sets, runs the RB stages in registers and stores them back (one shared-memory round
// trip and one barrier for RB stages). tw from twiddles(); unnormalised.
template <class R, int RB>
LB_DEV void fft_pass(Cx<R>* z, const Cx<R>* tw, int n, int logn, int s)
{
    constexpr int RR = 1 << RB;
    const int h = 1 << s, sets = n >> RB, ls = line_stride(n);
    for (int t = threadIdx.x; t < 2 * sets; t += blockDim.x) {
        Cx<R>* line = z + (t >= sets ? ls : 0);
        const int q = t >= sets ? t - sets : t;
        const int j = q & (h - 1);
        const int base = (q - j) * RR + j;  // (q / h) RR h + j
        Cx<R> v[RR];
#pragma unroll
        for (int k = 0; k < RR; ++k) v[k] = line[pz(base + k * h)];
#pragma unroll
        for (int l = 0; l < RB; ++l) {  // stage s + l: half H = h 2^l, pairs (k, k + 2^l)
#pragma unroll
            for (int k = 0; k < RR; ++k) {
                if (k & (1 << l)) continue;
                const int m = j + (k & ((1 << l) - 1)) * h;  // position of the pair within its half
                const Cx<R> w = tw[m << (logn - 1 - s - l)];   // exp(sign i pi m / H)
                const Cx<R> p = v[k], qv = v[k | (1 << l)];
                const R tr = w.re * qv.re - w.im * qv.im, ti = w.re * qv.im + w.im * qv.re;
                v[k] = {p.re + tr, p.im + ti};
                v[k | (1 << l)] = {p.re - tr, p.im - ti};
            }
        }
#pragma unroll
        for (int k = 0; k < RR; ++k) line[pz(base + k * h)] = v[k];
    }
    __syncthreads();
}

// FFT of the two lines (bit-reversed input order, loaded and synchronised by the caller):
// passes of three stages, the last one of one or two.
template <class R>
LB_DEV void fft2_lines(Cx<R>* z, const Cx<R>* tw, int n, int logn)
{
    int s = 0;
    for (; s + 3 <= logn; s += 3) fft_pass<R, 3>(z, tw, n, logn, s);
    if (logn - s == 2) fft_pass<R, 2>(z, tw, n, logn, s);
    else if (logn - s == 1) fft_pass<R, 1>(z, tw, n, logn, s);
}

// round(|k|) of the mode (kx, ky) (signed wavenumbers), in exact integer arithmetic: an FP32
// square root of m = kx^2 + ky^2 <= 2 * 2048^2 (exact in FP32) is off by at most one, which
// the integer corrections remove
LB_DEV int shell_of(int kx, int ky)
{
    const int m = kx * kx + ky * ky;
    int r = (int)sqrtf((float)m);
    if (r * r > m) --r;
    if ((r + 1) * (r + 1) <= m) ++r;
    return 4 * m >= (2 * r + 1) * (2 * r + 1) ? r + 1 : r;
}

LB_DEV int signed_k(int k, int n) { return k < n / 2 ? k : k - n; }

// rows, forward: moments of every node of row y, DFT along x -> spec[a][y][kx]
template <class T, int MODE>
__global__ void __launch_bounds__(256) k_sc_rows_fwd(const T* buf, Geom g, int logn,
                                                     Cx<typename Store<T>::Real>* spec)
{
    using R = typename Store<T>::Real;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    const int n = g.nx, y = blockIdx.x;
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n);
    Cx<R>* tw = z + 2 * ls;
    twiddles(tw, n, R(-1));
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        Nbr nb = make_nbr<sizeof(T)>(g, x, y, 0);
        R f[9], Fz[3] = {R(0), R(0), R(0)};
        load_node<D2Q9, MODE>(buf, g, nb, x + n * y, f);
        const NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f, Fz);
        const int r = bitrev(x, logn);
        z[pz(r)] = {m.ux, R(0)};
        z[ls + pz(r)] = {m.uy, R(0)};
    }
    __syncthreads();
    fft2_lines(z, tw, n, logn);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        spec[(int64_t)y * n + k] = z[pz(k)];
        spec[((int64_t)n + y) * n + k] = z[ls + pz(k)];
    }
}

// first |ky| in [0, n/2] whose mode (kx, ky) lies in shell s or above (the shell grows with |ky|)
LB_DEV int first_m(int kxs, int s, int n)
{
    int lo = 0, hi = n / 2 + 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (shell_of(kxs, mid) >= s) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// columns, forward: DFT along y of column kx, modal energies, shell sums of the column into
// partials[s][kx] (the modes of shell s in this column are one run of |ky|; summed in order
// of |ky|, +ky before -ky)
template <class R>
__global__ void __launch_bounds__(256) k_sc_cols_fwd(Cx<R>* spec, int n, int logn, double* partials)
{
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n);
    Cx<R>* tw = z + 2 * ls;
    double* e = reinterpret_cast<double*>(tw + n / 2);
    const int kx = blockIdx.x, K = n / 2;
    twiddles(tw, n, R(-1));
    for (int y = threadIdx.x; y < n; y += blockDim.x) {
        const int r = bitrev(y, logn);
        z[pz(r)] = spec[(int64_t)y * n + kx];
        z[ls + pz(r)] = spec[((int64_t)n + y) * n + kx];
    }
    __syncthreads();
    fft2_lines(z, tw, n, logn);
    const double inv_n4 = 1.0 / ((double)n * n * (double)n * n);
    for (int ky = threadIdx.x; ky < n; ky += blockDim.x) {
        const Cx<R> a = z[pz(ky)], b = z[ls + pz(ky)];
        spec[(int64_t)ky * n + kx] = a;
        spec[((int64_t)n + ky) * n + kx] = b;
        e[ky] = 0.5 * ((double)a.re * a.re + (double)a.im * a.im + (double)b.re * b.re + (double)b.im * b.im) * inv_n4;
    }
    __syncthreads();
    const int kxs = signed_k(kx, n);
    for (int s = threadIdx.x; s < K; s += blockDim.x) {
        const int m0 = first_m(kxs, s, n), m1 = first_m(kxs, s + 1, n);
        double acc = 0.0;
        for (int m = m0; m < m1; ++m) {
            acc += e[m];
            if (m > 0 && m < n / 2) acc += e[n - m];
        }
        partials[(int64_t)s * n + kx] = acc;
    }
}

// shells: sigma_s = sum over the columns (one warp per shell: lane l takes kx = l, l + 32, ...
// into four running sums in a fixed order, then a fixed shuffle tree), dR/dsigma_s and the
// shell's term of R
__global__ void __launch_bounds__(256) k_sc_shells(const double* partials, int n, const double* sigma0, double c,
                                                   double* sigma, double* grad, double* r2)
{
    const int K = n / 2, lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= K) return;
    // four independent running sums per lane keep four loads in flight
    const double* p = partials + (int64_t)s * n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int kx = lane;
    for (; kx + 96 < n; kx += 128) {
        a0 += p[kx];
        a1 += p[kx + 32];
        a2 += p[kx + 64];
        a3 += p[kx + 96];
    }
    for (; kx < n; kx += 32) a0 += p[kx];
    double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane != 0) return;
    sigma[s] = acc;
    if (sigma0) {
        const double l0 = log(fmax(sigma0[s], c));
        const double d = log(fmax(acc, c)) - l0;
        r2[s] = d * d;
        grad[s] = acc > c ? 2.0 * (log(acc) - l0) / acc : 0.0;
    }
}

// R = sum_s r2[s] by one warp in a fixed order
LB_DEV void sum_cost(const double* r2, int K, double* cost)
{
    double acc = 0.0;
    for (int s = threadIdx.x; s < K; s += 32) acc += r2[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) cost[0] = acc;
}

// cost R = sum_s r2[s] (one warp, fixed order)
__global__ void __launch_bounds__(32) k_sc_cost(const double* r2, int K, double* cost) { sum_cost(r2, K, cost); }

// columns, inverse: multiply by G(k), inverse DFT along y; block 0's first warp also totals
// the cost R (cost non-null)
template <class R>
__global__ void __launch_bounds__(256) k_sc_cols_inv(Cx<R>* spec, int n, int logn, const double* grad,
                                                     const double* r2, double* cost)
{
    if (cost && blockIdx.x == 0 && threadIdx.x < 32) sum_cost(r2, n / 2, cost);
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n);
    Cx<R>* tw = z + 2 * ls;
    const int kx = blockIdx.x, K = n / 2, kxs = signed_k(kx, n);
    twiddles(tw, n, R(1));
    for (int ky = threadIdx.x; ky < n; ky += blockDim.x) {
        const int sh = shell_of(kxs, signed_k(ky, n));
        const R G = sh < K ? (R)grad[sh] : R(0);
        const int r = bitrev(ky, logn);
        const Cx<R> a = spec[(int64_t)ky * n + kx], b = spec[((int64_t)n + ky) * n + kx];
        z[pz(r)] = {G * a.re, G * a.im};
        z[ls + pz(r)] = {G * b.re, G * b.im};
    }
    __syncthreads();
    fft2_lines(z, tw, n, logn);
    for (int y = threadIdx.x; y < n; y += blockDim.x) {
        spec[(int64_t)y * n + kx] = z[pz(y)];
        spec[((int64_t)n + y) * n + kx] = z[ls + pz(y)];
    }
}

// rows, inverse: inverse DFT along x, du_a = scale Re(.), scale = -kappa / N^2
template <class R>
__global__ void __launch_bounds__(256) k_sc_rows_inv(const Cx<R>* spec, int n, int logn, R scale, R* du,
                                                     int64_t plane)
{
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n);
    Cx<R>* tw = z + 2 * ls;
    const int y = blockIdx.x;
    twiddles(tw, n, R(1));
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = bitrev(k, logn);
        z[pz(r)] = spec[(int64_t)y * n + k];
        z[ls + pz(r)] = spec[((int64_t)n + y) * n + k];
    }
    __syncthreads();
    fft2_lines(z, tw, n, logn);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        du[(int64_t)y * n + x] = scale * z[pz(x)].re;
        du[plane + (int64_t)y * n + x] = scale * z[ls + pz(x)].re;
    }
}

// one BGK step of node (x, y) with the equilibrium at u + du
template <class T, int MODE>
LB_DEV void shifted_bgk_node(const T* src, T* dst, const Geom& g, typename Store<T>::Real omega, int x, int y,
                             typename Store<T>::Real dux, typename Store<T>::Real duy, unsigned* status)
{
    using R = typename Store<T>::Real;
    Nbr nb = make_nbr<sizeof(T)>(g, x, y, 0);
    const int n = x + g.nx * y;
    R f[9], feq[9], Fz[3] = {R(0), R(0), R(0)};
    load_node<D2Q9, MODE>(src, g, nb, n, f);
    NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f, Fz);
    const R rho = m.rho;
    m.ux += dux;
    m.uy += duy;
    equilibrium<D2Q9>(m, feq);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
    store_node<D2Q9, MODE>(dst, g, nb, n, f);
    if (!(rho > R(0) && rho < R(1e30))) atomicOr(status, 1u);
}

// rows, inverse, fused with the step: the inverse DFT of row y gives du of the row in shared
// memory, and the block then steps the row's nodes (the step reads only the pre-step state,
// which no kernel of this step writes; every node is stepped by exactly one thread, as in the
// one-kernel AA update)
template <class T, int MODE>
__global__ void __launch_bounds__(256) k_sc_rows_inv_step(const Cx<typename Store<T>::Real>* spec, int logn,
                                                          typename Store<T>::Real scale, const T* src, T* dst,
                                                          Geom g, typename Store<T>::Real omega, unsigned* status)
{
    using R = typename Store<T>::Real;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int n = g.nx, ls = line_stride(n);
    Cx<R>* tw = z + 2 * ls;
    const int y = blockIdx.x;
    twiddles(tw, n, R(1));
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = bitrev(k, logn);
        z[pz(r)] = spec[(int64_t)y * n + k];
        z[ls + pz(r)] = spec[((int64_t)n + y) * n + k];
    }
    __syncthreads();
    fft2_lines(z, tw, n, logn);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const R dux = scale * z[pz(x)].re, duy = scale * z[ls + pz(x)].re;
        shifted_bgk_node<T, MODE>(src, dst, g, omega, x, y, dux, duy, status);
    }
}

static int line_threads(int n) { return n < 256 ? n : 256; }

template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// step = true: the controlled step itself (a.dst, a.status, a.omega of s.a), du stays on chip
template <class T>
static cudaError_t shift_typed(const SpectralArgs& s, int* launches, bool step)
{
    using R = typename Store<T>::Real;
    const OpArgs& a = s.a;
    const int n = s.n, logn = s.logn, th = line_threads(n), K = n / 2;
    Cx<R>* spec = (Cx<R>*)s.spec;
    const size_t lines = (2 * (size_t)line_stride(n) + (size_t)K) * sizeof(Cx<R>);  // two lines + twiddles
    cudaError_t e;
    const T* buf = (const T*)a.src;
    if (a.mode == AB) {
        if ((e = smem_attr(k_sc_rows_fwd<T, AB>, lines)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AB><<<n, th, lines, a.stream>>>(buf, a.g, logn, spec);
    } else if (a.mode == AA_EVEN) {
        if ((e = smem_attr(k_sc_rows_fwd<T, AA_EVEN>, lines)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AA_EVEN><<<n, th, lines, a.stream>>>(buf, a.g, logn, spec);
    } else {
        if ((e = smem_attr(k_sc_rows_fwd<T, AA_ODD>, lines)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AA_ODD><<<n, th, lines, a.stream>>>(buf, a.g, logn, spec);
    }
    const size_t cols = lines + (size_t)n * sizeof(double);
    if ((e = smem_attr(k_sc_cols_fwd<R>, cols)) != cudaSuccess) return e;
    k_sc_cols_fwd<R><<<n, th, cols, a.stream>>>(spec, n, logn, s.partials);
    k_sc_shells<<<(K + 7) / 8, 256, 0, a.stream>>>(s.partials, n, s.sigma0, s.cutoff, s.sigma, s.grad, s.r2);
    *launches += 3;
    if (!s.sigma0) return cudaGetLastError();
    if (!s.du && !step) {
        k_sc_cost<<<1, 32, 0, a.stream>>>(s.r2, K, s.cost);
        *launches += 1;
        return cudaGetLastError();
    }
    if ((e = smem_attr(k_sc_cols_inv<R>, lines)) != cudaSuccess) return e;
    k_sc_cols_inv<R><<<n, th, lines, a.stream>>>(spec, n, logn, s.grad, s.r2, s.cost);
    const R scale = (R)(-s.kappa / ((double)n * n * (double)n * n));
    if (step) {  // inverse rows fused with the step
        const T* src = (const T*)a.src;
        T* dst = (T*)a.dst;
        const R om = (R)a.omega;
        if (a.mode == AB) {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AB>, lines)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AB><<<n, th, lines, a.stream>>>(spec, logn, scale, src, dst, a.g, om, a.status);
        } else if (a.mode == AA_EVEN) {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AA_EVEN>, lines)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AA_EVEN><<<n, th, lines, a.stream>>>(spec, logn, scale, src, dst, a.g, om,
                                                                       a.status);
        } else {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AA_ODD>, lines)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AA_ODD><<<n, th, lines, a.stream>>>(spec, logn, scale, src, dst, a.g, om,
                                                                      a.status);
        }
        *launches += 2;
        return cudaGetLastError();
    }
    if ((e = smem_attr(k_sc_rows_inv<R>, lines)) != cudaSuccess) return e;
    k_sc_rows_inv<R><<<n, th, lines, a.stream>>>(spec, n, logn, scale, (R*)s.du, a.g.plane);
    *launches += 2;
    return cudaGetLastError();
}

static cudaError_t shift_or_step(const SpectralArgs& s, int* launches, bool step)
{
    if (s.a.g.nx != s.n || s.a.g.ny != s.n || s.a.g.nz != 1 || s.n < 4 || s.n > kSpecMaxN || (1 << s.logn) != s.n)
        return cudaErrorInvalidValue;
    if (step && !s.sigma0) return cudaErrorInvalidValue;
    switch (s.a.storage) {
    case S_F64: return shift_typed<double>(s, launches, step);
    case S_F32: return shift_typed<float>(s, launches, step);
    case S_F16: return shift_typed<__half>(s, launches, step);
    case S_BF16: return shift_typed<__nv_bfloat16>(s, launches, step);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t spectral_shift(const SpectralArgs& s, int* launches) { return shift_or_step(s, launches, false); }

cudaError_t spectral_step(const SpectralArgs& s, int* launches) { return shift_or_step(s, launches, true); }

}  // namespace lb
