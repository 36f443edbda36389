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
// Both velocity components travel as one complex field w = u_x + i u_y: its transform is
// W = U_x + i U_y, and since k and -k lie in the same shell, the shell sums of
// |U_x|^2 + |U_y|^2 equal those of |W|^2 (|U_x(k)|^2 + |U_y(k)|^2 = (|W(k)|^2 + |W(-k)|^2) / 2);
// G is real and even, so the inverse transform of G W has the real part grad_u_x R N^2 and
// the imaginary part grad_u_y R N^2. One complex 2D FFT each way instead of two.
//
// A controlled step is five launches: rows (moments + forward DFT along x, lb_spectral_fft.cuh),
// columns (forward DFT along y and the shell sums of |W|^2 over the block's columns), shells
// (sigma and dR/dsigma, one warp per shell), columns (filter by G, inverse DFT along y), rows
// (inverse DFT along x: du, then the shifted BGK step of the row's nodes, and the cost R).
// lb_spectral_shift writes du instead of stepping. The line transforms hold their values in
// registers (lb_spectral_fft.cuh); the tables they use (twiddle factors per level, the shell of
// every mode, the first |ky| of every shell per column) are computed once per context. A
// column block takes several adjacent columns, so that its loads and stores of a grid row are
// whole 32-byte sectors. Every sum runs in a fixed order (deterministic).
#include "lb_spectral_fft.cuh"

namespace lb {
namespace sc {

LB_DEV void sincos_pi(double x, double* s, double* c) { sincospi(x, s, c); }

// Level twiddles exp(-2 pi i m r / (Ns R)) in the layout of Plan<L> (level 1: Ns = P, radix R1;
// level 2: Ns = P R1, radix R2), computed in FP64 and rounded once
template <class R>
__global__ void k_sc_twiddles(Cx<R>* tw, int P, int R1, int R2, int nlev)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int tw2 = nlev >= 2 ? (R1 - 1) * P : 0;
    const int twn = tw2 + (nlev == 3 ? (R2 - 1) * P * R1 : 0);
    if (e >= twn) return;
    int ns, rad, r, m;
    if (e < tw2) {
        ns = P, rad = R1, r = e / P + 1, m = e % P;
    } else {
        ns = P * R1, rad = R2, r = (e - tw2) / ns + 1, m = (e - tw2) % ns;
    }
    double s, c;
    sincos_pi(-2.0 * (double)m * r / ((double)ns * rad), &s, &c);
    tw[e] = {(R)c, (R)s};
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

// round(|k|) of every mode, in the order the column transforms load them: entry
// (kx M + t) P + r is the mode (kx, ky = t + r M) of thread t of column kx (P values per
// thread, M threads per column), so that a thread reads its P entries in one or two vectors
__global__ void k_sc_shell_table(short* shell, int n, int P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n) return;
    const int kx = (int)(i / n), rem = (int)(i % n), t = rem / P, r = rem % P, M = n / P;
    shell[i] = (short)shell_of(signed_k(kx, n), signed_k(t + r * M, n));
}

// first |ky| in [0, n/2 + 1] whose mode (kx, ky) lies in shell s or above (the shell grows
// with |ky|): shell_of is floor(sqrt(m) + 1/2), so for s >= 1 the condition is
// 4 (kx^2 + ky^2) >= (2s - 1)^2, solved for ky in integers (an FP32 square root, then exact
// corrections)
LB_DEV int first_m(int kxs, int s, int n)
{
    if (s <= 0) return 0;
    const int d = (2 * s - 1) * (2 * s - 1) - 4 * kxs * kxs;  // need 4 ky^2 >= d
    if (d <= 0) return 0;
    int ky = (int)ceilf(0.5f * sqrtf((float)d));
    while (ky > 0 && 4 * (ky - 1) * (ky - 1) >= d) --ky;
    while (4 * ky * ky < d) ++ky;
    return ky < n / 2 + 1 ? ky : n / 2 + 1;
}

// first[a][s] = first_m(a, s) for |kx| = a in [0, n/2] and s in [0, n/2]: in a column the modes
// of shell s are the |ky| in [first[a][s], first[a][s + 1])
__global__ void k_sc_first_table(short* first, int n)
{
    const int K = n / 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(K + 1) * (K + 1)) return;
    const int a = (int)(i / (K + 1)), s = (int)(i % (K + 1));
    first[i] = (short)first_m(a, s, n);
}

// columns per block: 32-byte runs of a grid row (four FP32 or two FP64 complex values), at most
// 512 threads per block
constexpr int col_c(int L, int rbytes)
{
    const int c0 = rbytes == 4 ? 4 : 2, m = (1 << L) / Plan_P(L);
    return c0 * m <= 512 ? c0 : 512 / m;
}
template <class R, int L>
struct ColShape {
    static constexpr int C = col_c(L, (int)sizeof(R));
};
template <class R, int L>
constexpr int col_threads() { return ColShape<R, L>::C * Plan<L>::M; }

// columns, forward: DFT along y of the block's C columns, then the shell sums of
// |W|^2 / (2 N^2) over those columns into partials[s][block] (per column the modes of shell s
// are one run of |ky|, summed in order of |ky|, +ky before -ky; the columns in order; the
// sums in the arithmetic type, scaled into FP64 once per shell)
template <class R, int L>
__global__ void __launch_bounds__(col_threads<R, L>()) k_sc_cols_fwd(Cx<R>* spec, const Cx<R>* __restrict__ tw,
                                                     const short* __restrict__ first, double* partials)
{
    using PL = Plan<L>;
    constexpr int C = ColShape<R, L>::C, n = PL::N, K = n / 2;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* zs = reinterpret_cast<Cx<R>*>(sc_smem);
    const int c = threadIdx.x % C, t = threadIdx.x / C, kx = blockIdx.x * C + c;
    // after the lines: the twiddles, then the shell runs of the block's columns,
    // first[|kx|][0 .. K] (read after the barriers below)
    Cx<R>* tws = zs + C * PL::LS;
    stage_twiddles<R, L>(tws, tw);
    short* fs = reinterpret_cast<short*>(tws + PL::TWN);
    for (int i = threadIdx.x; i < C * (K + 1); i += blockDim.x) {
        const int cc = i / (K + 1), kxc = blockIdx.x * C + cc;
        fs[i] = first[(kxc <= K ? kxc : n - kxc) * (K + 1) + i % (K + 1)];
    }
    pdl_wait();  // the row transforms of the previous launch
    pdl_trigger();
    Cx<R> a[PL::P];
#pragma unroll
    for (int r = 0; r < PL::P; ++r) a[r] = spec[(t + r * PL::M) * n + kx];
    line_fft<R, L, false>(a, zs + c * PL::LS, tws, t);
#pragma unroll
    for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
        for (int k = 0; k < PL::RL; ++k) spec[PL::out_index(t, s, k) * n + kx] = a[s * PL::RL + k];
    __syncthreads();  // the shared lines are free again
    R* e = reinterpret_cast<R*>(zs + c * PL::LS);
#pragma unroll
    for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
        for (int k = 0; k < PL::RL; ++k) {
            const Cx<R> v = a[s * PL::RL + k];
            e[PL::out_index(t, s, k)] = v.re * v.re + v.im * v.im;
        }
    __syncthreads();
    const double scale = 0.5 / ((double)n * n * (double)n * n);
    for (int sh = threadIdx.x; sh < K; sh += blockDim.x) {
        R acc = R(0);
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
            const R* ec = reinterpret_cast<const R*>(zs + cc * PL::LS);
            const short* fr = fs + cc * (K + 1);
            const int m0 = fr[sh], m1 = fr[sh + 1];
            R run = R(0);
            for (int m = m0; m < m1; ++m) {
                run += ec[m];
                if (m > 0 && m < K) run += ec[n - m];
            }
            acc += run;
        }
        partials[(int64_t)sh * gridDim.x + blockIdx.x] = (double)acc * scale;
    }
}

// columns, inverse: multiply by G(k) of the mode's shell, inverse DFT along y of the block's
// C columns (the twiddles and G of every kept shell staged in shared memory after the lines)
template <class R, int L>
__global__ void __launch_bounds__(col_threads<R, L>()) k_sc_cols_inv(Cx<R>* spec, const Cx<R>* __restrict__ tw,
                                                     const short* __restrict__ shell, const double* __restrict__ grad)
{
    using PL = Plan<L>;
    constexpr int C = ColShape<R, L>::C, n = PL::N, K = n / 2;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* zs = reinterpret_cast<Cx<R>*>(sc_smem);
    Cx<R>* tws = zs + C * PL::LS;
    R* gs = reinterpret_cast<R*>(tws + PL::TWN);
    stage_twiddles<R, L>(tws, tw);
    const int c = threadIdx.x % C, t = threadIdx.x / C, kx = blockIdx.x * C + c;
    // the thread's P shell indices are contiguous (k_sc_shell_table's order)
    short shv[PL::P];
    const short* sp = shell + (kx * PL::M + t) * PL::P;
    if constexpr (PL::P % 8 == 0) {
#pragma unroll
        for (int q = 0; q < PL::P / 8; ++q) {
            const uint4 v = reinterpret_cast<const uint4*>(sp)[q];
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                shv[8 * q + 2 * e] = (short)(w[e] & 0xffffu);
                shv[8 * q + 2 * e + 1] = (short)(w[e] >> 16);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < PL::P; ++r) shv[r] = sp[r];
    }
    pdl_wait();  // dR/dsigma of the previous launch (and the columns of the one before)
    pdl_trigger();
    for (int i = threadIdx.x; i < K; i += blockDim.x) gs[i] = (R)grad[i];
    Cx<R> a[PL::P];
#pragma unroll
    for (int r = 0; r < PL::P; ++r) a[r] = spec[(t + r * PL::M) * n + kx];
    __syncthreads();  // G staged
#pragma unroll
    for (int r = 0; r < PL::P; ++r) {
        const R G = shv[r] < K ? gs[shv[r]] : R(0);
        a[r] = {G * a[r].re, G * a[r].im};
    }
    line_fft<R, L, true>(a, zs + c * PL::LS, tws, t);
#pragma unroll
    for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
        for (int k = 0; k < PL::RL; ++k) spec[PL::out_index(t, s, k) * n + kx] = a[s * PL::RL + k];
}

// rows, inverse: inverse DFT along x, du_x = scale Re(.), du_y = scale Im(.), scale = -kappa / N^2,
// written by the transform's threads; the first warp of block 0 also totals the cost R
template <class R, int L>
__global__ void __launch_bounds__(RowShape<L>::THREADS) k_sc_rows_inv(const Cx<R>* __restrict__ spec,
                                                                      const Cx<R>* __restrict__ tw, R scale, R* du,
                                                                      int plane, const double* r2, double* cost)
{
    using PL = Plan<L>;
    using RS = RowShape<L>;
    constexpr int n = PL::N;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* tws = reinterpret_cast<Cx<R>*>(sc_smem) + RS::LPB * PL::LS;
    stage_twiddles<R, L>(tws, tw);
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x == 0 && threadIdx.x < 32) sum_cost(r2, n / 2, cost);
    const int l = threadIdx.x / PL::M, t = threadIdx.x % PL::M, y = blockIdx.x * RS::LPB + l;
    const bool act = threadIdx.x < RS::FFT_T && y < n;
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem) + (act ? l : 0) * PL::LS;
    Cx<R> a[PL::P];
    if (act) {
#pragma unroll
        for (int r = 0; r < PL::P; ++r) a[r] = spec[y * n + t + r * PL::M];
    }
    line_fft<R, L, true>(a, z, tws, t, act);
    if (!act) return;
#pragma unroll
    for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
        for (int k = 0; k < PL::RL; ++k) {
            const int x = PL::out_index(t, s, k);
            du[y * n + x] = scale * a[s * PL::RL + k].re;
            du[plane + y * n + x] = scale * a[s * PL::RL + k].im;
        }
}

// shells: sigma_s = sum over the column blocks (one warp per shell: lane l takes blocks l, l + 32,
// ... into four running sums in a fixed order, then a fixed shuffle tree), dR/dsigma_s and the
// shell's term of R. l0_s = ln max(sigma0_s, c) comes from the host; the logarithm of sigma and
// the gradient run in the arithmetic type R (the FP64 pipe is slow on this part, and FP32
// storage needs no more).
template <class R>
__global__ void __launch_bounds__(256) k_sc_shells(const double* partials, int n, int nblk, const double* l0,
                                                   double c, double* sigma, double* grad, double* r2)
{
    pdl_wait();  // the column blocks' partial sums
    pdl_trigger();
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n / 2) return;
    const int lane = threadIdx.x & 31;
    const double* p = partials + (int64_t)s * nblk;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nblk; b += 128) {
        a0 += p[b];
        a1 += p[b + 32];
        a2 += p[b + 64];
        a3 += p[b + 96];
    }
    for (; b < nblk; b += 32) a0 += p[b];
    double acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane != 0) return;
    sigma[s] = acc;
    if (l0) {
        const R d = log((R)fmax(acc, c)) - (R)l0[s];
        r2[s] = (double)d * (double)d;
        grad[s] = acc > c ? (double)(R(2) * d / (R)acc) : 0.0;
    }
}

// cost R = sum_s r2[s] (one warp, fixed order)
__global__ void __launch_bounds__(32) k_sc_cost(const double* r2, int K, double* cost)
{
    pdl_wait();
    pdl_trigger();
    sum_cost(r2, K, cost);
}

template <class R, int L>
static size_t col_smem_bytes()  // the lines, the twiddles, then G (inverse) or the shell runs (forward)
{
    constexpr int C = ColShape<R, L>::C, K = Plan<L>::N / 2;
    const size_t g = (size_t)K * sizeof(R), f = (size_t)C * (K + 1) * sizeof(short);
    return ((size_t)C * Plan<L>::LS + Plan<L>::TWN) * sizeof(Cx<R>) + (g > f ? g : f);
}

// the column passes of grid edge 2^L: forward DFT and shell sums (inv = false), or the filter
// by G and the inverse DFT
template <class R, int L>
static cudaError_t cols_sized(const SpectralArgs& s, bool inv)
{
    const int nblk = Plan<L>::N / ColShape<R, L>::C, th = col_threads<R, L>();
    const size_t smem = col_smem_bytes<R, L>();
    Cx<R>* spec = (Cx<R>*)s.spec;
    const Cx<R>* tw = (const Cx<R>*)s.tw;
    cudaError_t e;
    if (!inv) {
        if ((e = sc_smem_attr(k_sc_cols_fwd<R, L>, smem)) != cudaSuccess) return e;
        return launch_pdl(s.n <= kPdlMaxN, k_sc_cols_fwd<R, L>, nblk, th, smem, s.a.stream, spec, tw, (const short*)s.first, s.partials);
    } else {
        if ((e = sc_smem_attr(k_sc_cols_inv<R, L>, smem)) != cudaSuccess) return e;
        return launch_pdl(s.n <= kPdlMaxN, k_sc_cols_inv<R, L>, nblk, th, smem, s.a.stream, spec, tw, (const short*)s.shell,
                          (const double*)s.grad);
    }
}

// inverse rows writing du (no step)
template <class R, int L>
static cudaError_t rows_inv_sized(const SpectralArgs& s)
{
    const int blocks = (Plan<L>::N + RowShape<L>::LPB - 1) / RowShape<L>::LPB;
    const size_t smem = row_smem_bytes<R, L>();
    const R scale = (R)(-s.kappa / ((double)s.n * s.n * (double)s.n * s.n));
    cudaError_t e;
    if ((e = sc_smem_attr(k_sc_rows_inv<R, L>, smem)) != cudaSuccess) return e;
    return launch_pdl(s.n <= kPdlMaxN, k_sc_rows_inv<R, L>, blocks, RowShape<L>::THREADS, smem, s.a.stream, (const Cx<R>*)s.spec,
                      (const Cx<R>*)s.tw, scale, (R*)s.du, (int)s.a.g.plane, (const double*)s.r2, s.cost);
}

template <class R>
static cudaError_t cols(const SpectralArgs& s, bool inv)
{
    switch (s.logn) {
    case 2: return cols_sized<R, 2>(s, inv);
    case 3: return cols_sized<R, 3>(s, inv);
    case 4: return cols_sized<R, 4>(s, inv);
    case 5: return cols_sized<R, 5>(s, inv);
    case 6: return cols_sized<R, 6>(s, inv);
    case 7: return cols_sized<R, 7>(s, inv);
    case 8: return cols_sized<R, 8>(s, inv);
    case 9: return cols_sized<R, 9>(s, inv);
    case 10: return cols_sized<R, 10>(s, inv);
    case 11: return cols_sized<R, 11>(s, inv);
    case 12: return cols_sized<R, 12>(s, inv);
    default: return cudaErrorInvalidValue;
    }
}

template <class R>
static cudaError_t rows_inv(const SpectralArgs& s)
{
    switch (s.logn) {
    case 2: return rows_inv_sized<R, 2>(s);
    case 3: return rows_inv_sized<R, 3>(s);
    case 4: return rows_inv_sized<R, 4>(s);
    case 5: return rows_inv_sized<R, 5>(s);
    case 6: return rows_inv_sized<R, 6>(s);
    case 7: return rows_inv_sized<R, 7>(s);
    case 8: return rows_inv_sized<R, 8>(s);
    case 9: return rows_inv_sized<R, 9>(s);
    case 10: return rows_inv_sized<R, 10>(s);
    case 11: return rows_inv_sized<R, 11>(s);
    case 12: return rows_inv_sized<R, 12>(s);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t rows(const SpectralArgs& s, bool step)
{
    switch (s.a.storage) {
    case S_F64: return spectral_rows_f64(s, step);
    case S_F32: return spectral_rows_f32(s, step);
    case S_F16: return spectral_rows_f16(s, step);
    case S_BF16: return spectral_rows_bf16(s, step);
    default: return cudaErrorInvalidValue;
    }
}

// step = true: the controlled step itself (a.dst, a.status, a.omega of s.a), du stays on chip
template <class R>
static cudaError_t shift_typed(const SpectralArgs& s, int* launches, bool step)
{
    const OpArgs& a = s.a;
    const int n = s.n, K = n / 2, nblk = n / col_c(s.logn, (int)sizeof(R));
    cudaError_t e;
    if ((e = rows(s, false)) != cudaSuccess) return e;
    if ((e = cols<R>(s, false)) != cudaSuccess) return e;
    if ((e = launch_pdl(n <= kPdlMaxN, k_sc_shells<R>, (K + 7) / 8, 256, 0, a.stream, (const double*)s.partials, n, nblk,
                        s.sigma0 ? s.l0 : nullptr, s.cutoff, s.sigma, s.grad, s.r2)) != cudaSuccess)
        return e;
    *launches += 3;
    if (!s.sigma0) return cudaGetLastError();
    if (!s.du && !step) {
        if ((e = launch_pdl(n <= kPdlMaxN, k_sc_cost, 1, 32, 0, a.stream, (const double*)s.r2, K, s.cost)) != cudaSuccess) return e;
        *launches += 1;
        return cudaGetLastError();
    }
    if ((e = cols<R>(s, true)) != cudaSuccess) return e;
    e = step ? rows(s, true) : rows_inv<R>(s);
    *launches += 2;
    return e != cudaSuccess ? e : cudaGetLastError();
}

static cudaError_t shift_or_step(const SpectralArgs& s, int* launches, bool step)
{
    if (s.a.g.nx != s.n || s.a.g.ny != s.n || s.a.g.nz != 1 || s.n < 4 || s.n > kSpecMaxN || (1 << s.logn) != s.n)
        return cudaErrorInvalidValue;
    if (step && !s.sigma0) return cudaErrorInvalidValue;
    if (!s.tw || !s.shell || !s.first) return cudaErrorInvalidValue;
    return s.a.storage == S_F64 ? shift_typed<double>(s, launches, step) : shift_typed<float>(s, launches, step);
}

template <int L>
static void plan_of(int* P, int* R1, int* R2, int* nlev)
{
    *P = Plan<L>::P;
    *R1 = Plan<L>::R1;
    *R2 = Plan<L>::R2;
    *nlev = Plan<L>::NLEV;
}

}  // namespace sc

cudaError_t spectral_shift(const SpectralArgs& s, int* launches) { return sc::shift_or_step(s, launches, false); }

cudaError_t spectral_step(const SpectralArgs& s, int* launches) { return sc::shift_or_step(s, launches, true); }

size_t spectral_twiddle_count(int n)
{
    switch (n) {
    case 4: return sc::Plan<2>::TWN;
    case 8: return sc::Plan<3>::TWN;
    case 16: return sc::Plan<4>::TWN;
    case 32: return sc::Plan<5>::TWN;
    case 64: return sc::Plan<6>::TWN;
    case 128: return sc::Plan<7>::TWN;
    case 256: return sc::Plan<8>::TWN;
    case 512: return sc::Plan<9>::TWN;
    case 1024: return sc::Plan<10>::TWN;
    case 2048: return sc::Plan<11>::TWN;
    case 4096: return sc::Plan<12>::TWN;
    default: return 0;
    }
}

cudaError_t spectral_tables(void* tw, void* shell, void* first, int n, int storage, cudaStream_t st, int* launches)
{
    if (n < 4 || n > kSpecMaxN || (n & (n - 1))) return cudaErrorInvalidValue;
    int P = 0, R1 = 0, R2 = 0, nlev = 0;
    switch (n) {
    case 4: sc::plan_of<2>(&P, &R1, &R2, &nlev); break;
    case 8: sc::plan_of<3>(&P, &R1, &R2, &nlev); break;
    case 16: sc::plan_of<4>(&P, &R1, &R2, &nlev); break;
    case 32: sc::plan_of<5>(&P, &R1, &R2, &nlev); break;
    case 64: sc::plan_of<6>(&P, &R1, &R2, &nlev); break;
    case 128: sc::plan_of<7>(&P, &R1, &R2, &nlev); break;
    case 256: sc::plan_of<8>(&P, &R1, &R2, &nlev); break;
    case 512: sc::plan_of<9>(&P, &R1, &R2, &nlev); break;
    case 1024: sc::plan_of<10>(&P, &R1, &R2, &nlev); break;
    case 2048: sc::plan_of<11>(&P, &R1, &R2, &nlev); break;
    default: sc::plan_of<12>(&P, &R1, &R2, &nlev); break;
    }
    const int twn = (int)spectral_twiddle_count(n);
    if (twn > 0) {
        const int blocks = (twn + 127) / 128;
        if (storage == S_F64) sc::k_sc_twiddles<double><<<blocks, 128, 0, st>>>((sc::Cx<double>*)tw, P, R1, R2, nlev);
        else sc::k_sc_twiddles<float><<<blocks, 128, 0, st>>>((sc::Cx<float>*)tw, P, R1, R2, nlev);
        *launches += 1;
    }
    const int64_t nn = (int64_t)n * n, K = n / 2, nf = (K + 1) * (K + 1);
    sc::k_sc_shell_table<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>((short*)shell, n, P);
    sc::k_sc_first_table<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>((short*)first, n);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace lb
