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
// A controlled step is five launches: rows (moments + forward DFT along x), columns (forward
// DFT along y and the shell sums of |W|^2 over the block's columns), shells (sigma and
// dR/dsigma, one warp per shell), columns (filter by G, inverse DFT along y; the cost R), rows
// (inverse DFT along x: du, then the shifted BGK step of the row's nodes). lb_spectral_shift
// writes du instead of stepping. Each DFT is an in-place radix-2 FFT of grid lines in shared
// memory, in passes of three radix-2 stages held in registers (three twiddle-table entries per
// set of eight, the rest fixed rotations; a padded layout keeps the passes free of bank
// conflicts), with the twiddle table computed once per context. A row block takes one grid
// line; a column block takes several adjacent columns, so that its loads and stores of a grid
// row are contiguous runs of whole 32-byte sectors. Every sum runs in a fixed order
// (deterministic).
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

// twiddle table tw[k] = exp(-i 2 pi k / n), k < n/2
template <class R>
__global__ void k_sc_twiddles(Cx<R>* tw, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n / 2) return;
    R s, c;
    sincos_pi(R(-2 * k) / R(n), &s, &c);
    tw[k] = {c, s};
}

// the table into shared memory (block-wide; the caller syncs)
template <class R>
LB_DEV void load_twiddles(Cx<R>* tws, const Cx<R>* tw, int n)
{
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) tws[k] = tw[k];
}

// Shared-memory position of element i of a line: one spare slot after every eight elements, so
// that the threads of a half-warp reading the sets of the first passes hit distinct banks.
LB_HD int pz(int i) { return i + (i >> 3); }
// (one more slot per line, so that the lines of a column block start on different banks)
LB_HD int line_stride(int n) { return n + (n >> 3) + 1; }

// One pass of the in-place decimation-in-time FFT over the stages s .. s + RB - 1 (RB <= 3) of
// `lines` n-point lines z[l line_stride(n) ..) (bit-reversed input order): those stages only
// combine elements within the sets {base + k h : k < 2^RB}, h = 2^s, so each thread loads whole
// sets, runs the RB stages in registers and stores them back (one shared-memory round trip and
// one barrier for RB stages). Element k of a set sits at position j + k h of its 2^RB h block
// (j = its offset in the first h), so the stages' twiddles are
//   stage s:     w1 = exp(-i pi j / h)                              for every pair,
//   stage s + 1: w2 = exp(-i pi j / 2h), times -i for the pairs with odd k,
//   stage s + 2: w4 = exp(-i pi j / 4h), times exp(-i pi (k mod 4) / 4),
// three table entries per set and fixed rotations (the conjugates for INV); unnormalised.
template <class R, bool INV>
LB_DEV Cx<R> cmul(Cx<R> w, Cx<R> q)
{
    return {w.re * q.re - w.im * q.im, w.re * q.im + w.im * q.re};
}
// t times -i (forward) or +i (inverse)
template <class R, bool INV>
LB_DEV Cx<R> rot90(Cx<R> t)
{
    return INV ? Cx<R>{-t.im, t.re} : Cx<R>{t.im, -t.re};
}
template <class R>
LB_DEV void bfly(Cx<R>& p, Cx<R>& q, Cx<R> t)  // p, q <- p + t, p - t
{
    const Cx<R> a = p;
    p = {a.re + t.re, a.im + t.im};
    q = {a.re - t.re, a.im - t.im};
}

template <class R, int RB, bool INV>
LB_DEV void fft_pass(Cx<R>* z, const Cx<R>* tw, int n, int logn, int s, int lines)
{
    constexpr int RR = 1 << RB;
    const int h = 1 << s, lsets = logn - RB, ls = line_stride(n);
    for (int t = threadIdx.x; t < (lines << lsets); t += blockDim.x) {
        const int l = t >> lsets, q = t & ((1 << lsets) - 1);
        Cx<R>* line = z + l * ls;
        const int j = q & (h - 1);
        const int base = ((q - j) << RB) + j;
        Cx<R> v[RR];
#pragma unroll
        for (int k = 0; k < RR; ++k) v[k] = line[pz(base + k * h)];
        auto twid = [&](int sh) {
            Cx<R> w = tw[j << sh];
            if (INV) w.im = -w.im;
            return w;
        };
        {
            const Cx<R> w1 = twid(logn - 1 - s);
#pragma unroll
            for (int k = 0; k < RR; k += 2) bfly(v[k], v[k + 1], cmul<R, INV>(w1, v[k + 1]));
        }
        if constexpr (RB >= 2) {
            const Cx<R> w2 = twid(logn - 2 - s);
#pragma unroll
            for (int k0 = 0; k0 < RR; k0 += 4) {
                bfly(v[k0], v[k0 + 2], cmul<R, INV>(w2, v[k0 + 2]));
                bfly(v[k0 + 1], v[k0 + 3], rot90<R, INV>(cmul<R, INV>(w2, v[k0 + 3])));
            }
        }
        if constexpr (RB >= 3) {
            const Cx<R> w4 = twid(logn - 3 - s);
            // exp(-+ i pi / 4) = (1 -+ i) / sqrt 2
            const R r = R(0.70710678118654752440);
            const Cx<R> c8 = {r, INV ? r : -r};
            const Cx<R> w4c = cmul<R, INV>(c8, w4);
            bfly(v[0], v[4], cmul<R, INV>(w4, v[4]));
            bfly(v[1], v[5], cmul<R, INV>(w4c, v[5]));
            bfly(v[2], v[6], rot90<R, INV>(cmul<R, INV>(w4, v[6])));
            bfly(v[3], v[7], rot90<R, INV>(cmul<R, INV>(w4c, v[7])));
        }
#pragma unroll
        for (int k = 0; k < RR; ++k) line[pz(base + k * h)] = v[k];
    }
    __syncthreads();
}

// FFT of `lines` lines (bit-reversed input order, loaded and synchronised by the caller):
// passes of three stages, the last one of one or two.
template <class R, bool INV>
LB_DEV void fft_lines(Cx<R>* z, const Cx<R>* tw, int n, int logn, int lines)
{
    int s = 0;
    for (; s + 3 <= logn; s += 3) fft_pass<R, 3, INV>(z, tw, n, logn, s, lines);
    if (logn - s == 2) fft_pass<R, 2, INV>(z, tw, n, logn, s, lines);
    else if (logn - s == 1) fft_pass<R, 1, INV>(z, tw, n, logn, s, lines);
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

// Population access of node x of row y with 32-bit element offsets (9 x plane < 2^31 for every
// grid the spectral calls accept): the three columns x - 1, x, x + 1 and the three row offsets
// (y - 1) n, y n, (y + 1) n, periodic; access modes as in lb_device.cuh.
struct ScRows {
    int r[3];
};
LB_DEV ScRows sc_rows(int y, int n)
{
    return {{(y == 0 ? n - 1 : y - 1) * n, y * n, (y == n - 1 ? 0 : y + 1) * n}};
}
template <class T, int MODE>
LB_DEV void sc_load(const T* buf, int plane, const ScRows& rw, int x, int n, typename Store<T>::Real* f)
{
    const int col[3] = {x == 0 ? n - 1 : x - 1, x, x == n - 1 ? 0 : x + 1};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int sg = (MODE == AA_EVEN) ? 0 : -1;
        f[i] = load_pop<D2Q9>(buf + (slot * plane + rw.r[1 + sg * c2(i, 1)] + col[1 + sg * c2(i, 0)]), slot);
    }
}
template <class T, int MODE>
LB_DEV void sc_store(T* buf, int plane, const ScRows& rw, int x, int n, const typename Store<T>::Real* f)
{
    const int col[3] = {x == 0 ? n - 1 : x - 1, x, x == n - 1 ? 0 : x + 1};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int slot = (MODE == AA_EVEN) ? opp(i) : i;
        const int sg = (MODE == AA_ODD) ? 1 : 0;
        store_pop<D2Q9>(buf + (slot * plane + rw.r[1 + sg * c2(i, 1)] + col[1 + sg * c2(i, 0)]), slot, f[i]);
    }
}

constexpr int kRowBatch = 4;

// rows, forward: moments of every node of row y, w = u_x + i u_y, DFT along x -> spec[y][kx]
template <class T, int MODE>
__global__ void __launch_bounds__(256) k_sc_rows_fwd(const T* buf, Geom g, int logn,
                                                     const Cx<typename Store<T>::Real>* tw,
                                                     Cx<typename Store<T>::Real>* spec)
{
    using R = typename Store<T>::Real;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    const int n = g.nx, y = blockIdx.x, plane = (int)g.plane;
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    Cx<R>* tws = z + line_stride(n);
    load_twiddles(tws, tw, n);
    const ScRows rw = sc_rows(y, n);
    // kRowBatch nodes per thread at a time: all their loads are issued before the first
    // shared-memory store (which the compiler would not move loads across)
    for (int x0 = threadIdx.x; x0 < n; x0 += kRowBatch * blockDim.x) {
        R f[kRowBatch][9];
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b) {
            const int x = x0 + b * blockDim.x;
            if (x < n) sc_load<T, MODE>(buf, plane, rw, x, n, f[b]);
        }
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b) {
            const int x = x0 + b * blockDim.x;
            if (x < n) {
                const R Fz[3] = {R(0), R(0), R(0)};
                const NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f[b], Fz);
                z[pz(bitrev(x, logn))] = {m.ux, m.uy};
            }
        }
    }
    __syncthreads();
    fft_lines<R, false>(z, tws, n, logn, 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) spec[(int64_t)y * n + k] = z[pz(k)];
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

// load the C columns kx0 .. kx0 + C - 1 of spec into lines 0 .. C - 1 (bit-reversed order along
// y), each value times G of its shell if grad is given: thread t takes row t / C, column t % C,
// so the threads of a warp read runs of C adjacent values of a row
template <class R, int C>
LB_DEV void load_columns(Cx<R>* z, const Cx<R>* spec, int n, int logn, int kx0, const double* grad)
{
    const int ls = line_stride(n), K = n / 2, total = n * C;
    constexpr int U = 4;  // loads in flight per thread
    for (int t0 = threadIdx.x; t0 < total; t0 += U * blockDim.x) {
        Cx<R> v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < total) {
                const int y = t / C, c = t - y * C;
                v[u] = spec[(int64_t)y * n + kx0 + c];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < total) {
                const int y = t / C, c = t - y * C;
                if (grad) {
                    const int sh = shell_of(signed_k(kx0 + c, n), signed_k(y, n));
                    const R G = sh < K ? (R)__ldg(grad + sh) : R(0);
                    v[u].re *= G;
                    v[u].im *= G;
                }
                z[c * ls + pz(bitrev(y, logn))] = v[u];
            }
        }
    }
}

template <class R, int C>
LB_DEV void store_columns(const Cx<R>* z, Cx<R>* spec, int n, int kx0)
{
    const int ls = line_stride(n);
    for (int t = threadIdx.x; t < n * C; t += blockDim.x) {
        const int y = t / C, c = t - y * C;
        spec[(int64_t)y * n + kx0 + c] = z[c * ls + pz(y)];
    }
}

// the shell sums of |W|^2 / (2 N^2) over the block's C transformed columns (natural order)
// into partials[s][block]: per column the modes of shell s are one run of |ky|, summed in order
// of |ky|, +ky before -ky; the runs' sums and the columns in the arithmetic type (a few to a
// few hundred terms; FP64 is a slow pipe on this part), scaled into FP64 once per shell
template <class R, int C>
LB_DEV void column_shell_sums(const Cx<R>* z, int n, int kx0, int nblk, double* partials)
{
    const int ls = line_stride(n), K = n / 2;
    const double scale = 0.5 / ((double)n * n * (double)n * n);
    for (int s = threadIdx.x; s < K; s += blockDim.x) {
        R acc = R(0);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const Cx<R>* line = z + c * ls;
            const int kxs = signed_k(kx0 + c, n);
            const int m0 = first_m(kxs, s, n), m1 = first_m(kxs, s + 1, n);
            R run = R(0);
            for (int m = m0; m < m1; ++m) {
                const Cx<R> a = line[pz(m)];
                run += a.re * a.re + a.im * a.im;
                if (m > 0 && m < n / 2) {
                    const Cx<R> b = line[pz(n - m)];
                    run += b.re * b.re + b.im * b.im;
                }
            }
            acc += run;
        }
        partials[(int64_t)s * nblk + blockIdx.x] = (double)acc * scale;
    }
}

// columns, forward: DFT along y of the block's C columns, then the shell sums of |W|^2 / (2 N^2)
// over those columns into partials[s][block] (per column the modes of shell s are one run of
// |ky|, summed in order of |ky|, +ky before -ky; the columns in order)
template <class R, int C>
__global__ void __launch_bounds__(512) k_sc_cols_fwd(Cx<R>* spec, int n, int logn, const Cx<R>* tw,
                                                     double* partials)
{
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n), kx0 = blockIdx.x * C, nblk = gridDim.x;
    Cx<R>* tws = z + C * ls;
    load_twiddles(tws, tw, n);
    load_columns<R, C>(z, spec, n, logn, kx0, nullptr);
    __syncthreads();
    fft_lines<R, false>(z, tws, n, logn, C);
    store_columns<R, C>(z, spec, n, kx0);
    column_shell_sums<R, C>(z, n, kx0, nblk, partials);
}

// shells: sigma_s = sum over the column blocks (one warp per shell: lane l takes blocks l, l + 32,
// ... into four running sums in a fixed order, then a fixed shuffle tree), dR/dsigma_s and the
// shell's term of R. l0_s = ln max(sigma0_s, c) comes from the host; the logarithm of sigma and
// the gradient run in the arithmetic type R (the FP64 pipe is slow on this part, and FP32
// storage needs no more).
template <class R>
LB_DEV void shell_reduce(const double* partials, int nblk, int s, int lane, const double* l0, double c,
                         double* sigma, double* grad, double* r2)
{
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

template <class R>
__global__ void __launch_bounds__(256) k_sc_shells(const double* partials, int n, int nblk, const double* l0,
                                                   double c, double* sigma, double* grad, double* r2)
{
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n / 2) return;
    shell_reduce<R>(partials, nblk, s, threadIdx.x & 31, l0, c, sigma, grad, r2);
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

// columns, inverse: multiply by G(k), inverse DFT along y of the block's C columns; block 0's
// first warp also totals the cost R (cost non-null)
template <class R, int C>
__global__ void __launch_bounds__(512) k_sc_cols_inv(Cx<R>* spec, int n, int logn, const Cx<R>* tw,
                                                     const double* grad, const double* r2, double* cost)
{
    if (cost && blockIdx.x == 0 && threadIdx.x < 32) sum_cost(r2, n / 2, cost);
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int ls = line_stride(n), kx0 = blockIdx.x * C;
    Cx<R>* tws = z + C * ls;
    load_twiddles(tws, tw, n);
    load_columns<R, C>(z, spec, n, logn, kx0, grad);
    __syncthreads();
    fft_lines<R, true>(z, tws, n, logn, C);
    store_columns<R, C>(z, spec, n, kx0);
}

// rows, inverse: inverse DFT along x, du_x = scale Re(.), du_y = scale Im(.), scale = -kappa / N^2
template <class R>
__global__ void __launch_bounds__(256) k_sc_rows_inv(const Cx<R>* spec, int n, int logn, const Cx<R>* tw, R scale,
                                                     R* du, int64_t plane)
{
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    Cx<R>* tws = z + line_stride(n);
    const int y = blockIdx.x;
    load_twiddles(tws, tw, n);
    for (int k = threadIdx.x; k < n; k += blockDim.x) z[pz(bitrev(k, logn))] = spec[(int64_t)y * n + k];
    __syncthreads();
    fft_lines<R, true>(z, tws, n, logn, 1);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        du[(int64_t)y * n + x] = scale * z[pz(x)].re;
        du[plane + (int64_t)y * n + x] = scale * z[pz(x)].im;
    }
}

// one BGK step of a node from its pre-collision deviations f (loaded by the caller) with the
// equilibrium at u + du
template <class T, int MODE>
LB_DEV void shifted_bgk_node(typename Store<T>::Real* f, T* dst, int plane, const ScRows& rw, int n,
                             typename Store<T>::Real omega, int x, typename Store<T>::Real dux,
                             typename Store<T>::Real duy, unsigned* status)
{
    using R = typename Store<T>::Real;
    R feq[9];
    const R Fz[3] = {R(0), R(0), R(0)};
    NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f, Fz);
    const R rho = m.rho;
    m.ux += dux;
    m.uy += duy;
    equilibrium<D2Q9>(m, feq);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = f[i] - omega * (f[i] - feq[i]);
    sc_store<T, MODE>(dst, plane, rw, x, n, f);
    if (!(rho > R(0) && rho < R(1e30))) atomicOr(status, 1u);
}

// rows, inverse, fused with the step: the inverse DFT of row y gives du of the row in shared
// memory, and the block then steps the row's nodes (the step reads only the pre-step state,
// which no kernel of this step writes; every node is stepped by exactly one thread, as in the
// one-kernel AA update)
template <class T, int MODE>
__global__ void __launch_bounds__(256) k_sc_rows_inv_step(const Cx<typename Store<T>::Real>* spec, int logn,
                                                          const Cx<typename Store<T>::Real>* tw,
                                                          typename Store<T>::Real scale, const T* src, T* dst,
                                                          Geom g, typename Store<T>::Real omega, unsigned* status)
{
    using R = typename Store<T>::Real;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* z = reinterpret_cast<Cx<R>*>(sc_smem);
    const int n = g.nx;
    Cx<R>* tws = z + line_stride(n);
    const int y = blockIdx.x;
    load_twiddles(tws, tw, n);
    for (int k = threadIdx.x; k < n; k += blockDim.x) z[pz(bitrev(k, logn))] = spec[(int64_t)y * n + k];
    __syncthreads();
    fft_lines<R, true>(z, tws, n, logn, 1);
    const ScRows rw = sc_rows(y, n);
    const int plane = (int)g.plane;
    // every node is read and written by its own thread only (AB: other buffer; AA: its own
    // slots), so the loads of a batch may precede the stores of the nodes before it
    for (int x0 = threadIdx.x; x0 < n; x0 += kRowBatch * blockDim.x) {
        R f[kRowBatch][9];
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b) {
            const int x = x0 + b * blockDim.x;
            if (x < n) sc_load<T, MODE>(src, plane, rw, x, n, f[b]);
        }
#pragma unroll
        for (int b = 0; b < kRowBatch; ++b) {
            const int x = x0 + b * blockDim.x;
            if (x < n) {
                const Cx<R> d = z[pz(x)];
                shifted_bgk_node<T, MODE>(f[b], dst, plane, rw, n, omega, x, scale * d.re, scale * d.im, status);
            }
        }
    }
}

// threads of a block that FFTs `lines` lines of n points (passes of three stages: n / 8 sets
// per line, one per thread, 32 to `cap`)
static int fft_threads(int n, int lines, int cap)
{
    const int t = lines * n / 8;
    return t < 32 ? 32 : (t > cap ? cap : t);
}

// columns per column block: four (whole 32-byte sectors of FP32 values, two of FP64), fewer
// where four lines would not fit in shared memory
template <class R>
static int column_block(int n)
{
    int C = 4;
    while (C > 1 && (size_t)C * line_stride(n) * sizeof(Cx<R>) > 160 * 1024) C >>= 1;
    return C < n ? C : n;
}

template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// the column passes with C columns per block: forward DFT and shell sums (inv = false), or
// the filter by G and the inverse DFT
template <class R, int C>
static cudaError_t launch_columns(const SpectralArgs& s, bool inv)
{
    const int n = s.n, logn = s.logn, K = n / 2, nblk = n / C, th = fft_threads(n, C, 512);
    const size_t smem = ((size_t)C * line_stride(n) + (size_t)K) * sizeof(Cx<R>);
    Cx<R>* spec = (Cx<R>*)s.spec;
    const Cx<R>* tw = (const Cx<R>*)s.tw;
    cudaError_t e;
    if (!inv) {
        if ((e = smem_attr(k_sc_cols_fwd<R, C>, smem)) != cudaSuccess) return e;
        k_sc_cols_fwd<R, C><<<nblk, th, smem, s.a.stream>>>(spec, n, logn, tw, s.partials);
    } else {
        if ((e = smem_attr(k_sc_cols_inv<R, C>, smem)) != cudaSuccess) return e;
        k_sc_cols_inv<R, C><<<nblk, th, smem, s.a.stream>>>(spec, n, logn, tw, s.grad, s.r2, s.cost);
    }
    return cudaGetLastError();
}
template <class R>
static cudaError_t columns(const SpectralArgs& s, bool inv)
{
    switch (column_block<R>(s.n)) {
    case 4: return launch_columns<R, 4>(s, inv);
    case 2: return launch_columns<R, 2>(s, inv);
    default: return launch_columns<R, 1>(s, inv);
    }
}

// step = true: the controlled step itself (a.dst, a.status, a.omega of s.a), du stays on chip
template <class T>
static cudaError_t shift_typed(const SpectralArgs& s, int* launches, bool step)
{
    using R = typename Store<T>::Real;
    const OpArgs& a = s.a;
    const int n = s.n, logn = s.logn, K = n / 2;
    const int nblk = n / column_block<R>(n);
    // a row block: one thread per set of the FFT passes (n / 8, 32 to 256), each loading and
    // stepping n / threads nodes of the row
    const int th_row = fft_threads(n, 1, 256);
    Cx<R>* spec = (Cx<R>*)s.spec;
    const Cx<R>* tw = (const Cx<R>*)s.tw;
    const size_t row_smem = ((size_t)line_stride(n) + (size_t)K) * sizeof(Cx<R>);  // one line + twiddles
    cudaError_t e;
    const T* buf = (const T*)a.src;
    if (a.mode == AB) {
        if ((e = smem_attr(k_sc_rows_fwd<T, AB>, row_smem)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AB><<<n, th_row, row_smem, a.stream>>>(buf, a.g, logn, tw, spec);
    } else if (a.mode == AA_EVEN) {
        if ((e = smem_attr(k_sc_rows_fwd<T, AA_EVEN>, row_smem)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AA_EVEN><<<n, th_row, row_smem, a.stream>>>(buf, a.g, logn, tw, spec);
    } else {
        if ((e = smem_attr(k_sc_rows_fwd<T, AA_ODD>, row_smem)) != cudaSuccess) return e;
        k_sc_rows_fwd<T, AA_ODD><<<n, th_row, row_smem, a.stream>>>(buf, a.g, logn, tw, spec);
    }
    if ((e = columns<R>(s, false)) != cudaSuccess) return e;
    k_sc_shells<R><<<(K + 7) / 8, 256, 0, a.stream>>>(s.partials, n, nblk, s.sigma0 ? s.l0 : nullptr, s.cutoff,
                                                      s.sigma, s.grad, s.r2);
    *launches += 3;
    if (!s.sigma0) return cudaGetLastError();
    if (!s.du && !step) {
        k_sc_cost<<<1, 32, 0, a.stream>>>(s.r2, K, s.cost);
        *launches += 1;
        return cudaGetLastError();
    }
    if ((e = columns<R>(s, true)) != cudaSuccess) return e;
    *launches += 1;
    const R scale = (R)(-s.kappa / ((double)n * n * (double)n * n));
    if (step) {  // inverse rows fused with the step
        const T* src = (const T*)a.src;
        T* dst = (T*)a.dst;
        const R om = (R)a.omega;
        if (a.mode == AB) {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AB>, row_smem)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AB><<<n, th_row, row_smem, a.stream>>>(spec, logn, tw, scale, src, dst, a.g, om,
                                                                         a.status);
        } else if (a.mode == AA_EVEN) {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AA_EVEN>, row_smem)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AA_EVEN><<<n, th_row, row_smem, a.stream>>>(spec, logn, tw, scale, src, dst, a.g,
                                                                              om, a.status);
        } else {
            if ((e = smem_attr(k_sc_rows_inv_step<T, AA_ODD>, row_smem)) != cudaSuccess) return e;
            k_sc_rows_inv_step<T, AA_ODD><<<n, th_row, row_smem, a.stream>>>(spec, logn, tw, scale, src, dst, a.g,
                                                                             om, a.status);
        }
        *launches += 1;
        return cudaGetLastError();
    }
    if ((e = smem_attr(k_sc_rows_inv<R>, row_smem)) != cudaSuccess) return e;
    k_sc_rows_inv<R><<<n, th_row, row_smem, a.stream>>>(spec, n, logn, tw, scale, (R*)s.du, a.g.plane);
    *launches += 1;
    return cudaGetLastError();
}

static cudaError_t shift_or_step(const SpectralArgs& s, int* launches, bool step)
{
    if (s.a.g.nx != s.n || s.a.g.ny != s.n || s.a.g.nz != 1 || s.n < 4 || s.n > kSpecMaxN || (1 << s.logn) != s.n)
        return cudaErrorInvalidValue;
    if (step && !s.sigma0) return cudaErrorInvalidValue;
    if (!s.tw) return cudaErrorInvalidValue;
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

cudaError_t spectral_twiddles(void* tw, int n, int storage, cudaStream_t st)
{
    if (n < 4 || n > kSpecMaxN) return cudaErrorInvalidValue;
    const int blocks = (n / 2 + 127) / 128;
    if (storage == S_F64) k_sc_twiddles<double><<<blocks, 128, 0, st>>>((Cx<double>*)tw, n);
    else k_sc_twiddles<float><<<blocks, 128, 0, st>>>((Cx<float>*)tw, n);
    return cudaGetLastError();
}

}  // namespace lb
