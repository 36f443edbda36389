// Line transforms of the spectral flow control (Sec. 3.2) and the row kernels built on them.
//
// A grid line of N = 2^L complex values is transformed by M = N / P threads that each hold P
// values in registers: the Stockham form of the Cooley-Tukey FFT, in levels. Level 0 gives
// thread t the values t + r M (r < P) and runs one P-point DFT on them (no twiddle factors);
// each later level, of radix R, reads its values back from shared memory at stride N / R,
// multiplies value r of the thread's virtual index j by exp(-+2 pi i m r / (Ns R)) (Ns = the
// product of the earlier radices, m = j mod Ns) and runs R-point DFTs; a level's result k of
// index j goes to (j / Ns) Ns R + m + k Ns. After the last level thread t holds element
// t + M s + k N / R in register s R + k: natural order, strided across the threads, so a
// line's loads and stores are coalesced. P = 2^ceil(L/2) up to L = 2 kMaxB0 (two levels, one
// exchange through shared memory), P = 2^kMaxB0 beyond (three levels). The DFTs in registers are
// radix-2 decimation-in-time networks whose rotations (multiples of 2 pi / 32) are constants.
// Every size is a separate instantiation, so all indexing is resolved at compile time.
#pragma once

#include "lb_collide.cuh"
#include "lb_spectral.cuh"

namespace lb {
namespace sc {

template <class R>
struct Cx {
    R re, im;
};

// Largest radix of a level, as log2: 16 values per thread (a 1024-point line is 64 threads in
// three levels; 32 values per thread took two levels but left too few warps per SM to hide the
// loads).
constexpr int kMaxB0 = 4;

// values per thread of an N = 2^L point line transform
LB_HD constexpr int plan_b0(int L) { return L <= kMaxB0 ? L : (L <= 2 * kMaxB0 ? (L + 1) / 2 : kMaxB0); }
LB_HD constexpr int Plan_P(int L) { return 1 << plan_b0(L); }

// Level structure of an N = 2^L point line transform.
template <int L>
struct Plan {
    static constexpr int N = 1 << L;
    static constexpr int B0 = plan_b0(L);
    static constexpr int REST = L - B0;
    static constexpr int NLEV = REST == 0 ? 1 : (REST <= B0 ? 2 : 3);
    static constexpr int B1 = NLEV == 1 ? 0 : (NLEV == 2 ? REST : (REST + 1) / 2);
    static constexpr int B2 = NLEV == 3 ? REST - B1 : 0;
    static_assert(B1 <= B0 && B2 <= B0 && B0 + B1 + B2 == L, "levels of at most B0 bits");
    static constexpr int P = 1 << B0, M = N / P, R1 = 1 << B1, R2 = 1 << B2;
    // radix and sub-DFTs per thread of the last level
    static constexpr int RL = NLEV == 1 ? P : (NLEV == 2 ? R1 : R2);
    static constexpr int SUBL = P / RL;
    // twiddle table: level 1 [R1 - 1][P], then level 2 [R2 - 1][P R1]
    static constexpr int TW2 = NLEV >= 2 ? (R1 - 1) * P : 0;
    static constexpr int TWN = TW2 + (NLEV == 3 ? (R2 - 1) * P * R1 : 0);
    // shared-memory line: one spare slot after every P values (the level-0 writes of the
    // threads, P apart, then fall in distinct banks), stride = 4 mod 16 elements (lines of
    // adjacent columns start in different banks)
    static constexpr int BASE = N + N / P;
    static constexpr int LS = BASE + (20 - BASE % 16) % 16;
    LB_HD static constexpr int pad(int p) { return p + (p >> B0); }
    // element held in register s RL + k of thread t after the last level
    LB_HD static constexpr int out_index(int t, int s, int k) { return t + M * s + k * (N / RL); }
};

// cos and sin of 2 pi e / 32, e in [0, 16)
LB_HD constexpr double cos32_0to8(int e)
{
    return e == 0 ? 1.0
         : e == 1 ? 0.98078528040323044913
         : e == 2 ? 0.92387953251128675613
         : e == 3 ? 0.83146961230254523708
         : e == 4 ? 0.70710678118654752440
         : e == 5 ? 0.55557023301960222474
         : e == 6 ? 0.38268343236508977173
         : e == 7 ? 0.19509032201612826785
                  : 0.0;
}
LB_HD constexpr double cos32(int e) { return e <= 8 ? cos32_0to8(e) : -cos32_0to8(16 - e); }
LB_HD constexpr double sin32(int e) { return e <= 8 ? cos32_0to8(8 - e) : cos32_0to8(e - 8); }

LB_HD constexpr int brev_bits(int v, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
    return r;
}
LB_HD constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// x exp(-+2 pi i e / 32) (forward -, inverse +); e is a constant after unrolling
template <class R, bool INV>
LB_DEV Cx<R> rot32(Cx<R> x, int e)
{
    if (e == 0) return x;
    if (e == 8) return INV ? Cx<R>{-x.im, x.re} : Cx<R>{x.im, -x.re};
    const R c = R(cos32(e)), s = R(sin32(e));
    if (INV) return {c * x.re - s * x.im, c * x.im + s * x.re};
    return {c * x.re + s * x.im, c * x.im - s * x.re};
}

template <class R, bool INV>
LB_DEV Cx<R> cmul_tw(Cx<R> w, Cx<R> x)  // x w (forward) or x conj(w) (inverse)
{
    if (INV) return {w.re * x.re + w.im * x.im, w.re * x.im - w.im * x.re};
    return {w.re * x.re - w.im * x.im, w.re * x.im + w.im * x.re};
}

// In place, natural order in and out: a[off + k] <- sum_r a[off + r] exp(-+2 pi i r k / RAD),
// RAD <= 32 (a bit-reversal renaming of registers, then the radix-2 stages)
template <class R, int RAD, bool INV, int NA>
LB_DEV void dft(Cx<R> (&a)[NA], int off)
{
    constexpr int LR = ilog2(RAD);
#pragma unroll
    for (int i = 0; i < RAD; ++i) {
        const int j = brev_bits(i, LR);
        if (j > i) {
            const Cx<R> tmp = a[off + i];
            a[off + i] = a[off + j];
            a[off + j] = tmp;
        }
    }
    // stage lh: butterfly b pairs i0 = g + k and i0 + h (h = 2^lh, k = b mod h, g = 2h (b / h))
    // with the twiddle exp(-+2 pi i k / 2h); every loop has a constant trip count, so all of them
    // unroll and the array stays in registers
#pragma unroll
    for (int lh = 0; lh < LR; ++lh)
#pragma unroll
        for (int b = 0; b < RAD / 2; ++b) {
            const int h = 1 << lh, k = b & (h - 1), i0 = ((b >> lh) << (lh + 1)) + k;
            const Cx<R> u = a[off + i0];
            const Cx<R> v = rot32<R, INV>(a[off + i0 + h], k * (16 >> lh));
            a[off + i0] = {u.re + v.re, u.im + v.im};
            a[off + i0 + h] = {u.re - v.re, u.im - v.im};
        }
}

// Level LEV >= 1 of the line transform: read from the shared line z, twiddle, DFTs; the result
// goes back to z unless this is the last level (then it stays in a). Threads with act = false
// do no work but take part in the block's barriers.
template <class R, int L, int LEV, bool INV>
LB_DEV void fft_level(Cx<R> (&a)[Plan<L>::P], Cx<R>* z, const Cx<R>* __restrict__ tw, int t, bool act)
{
    using PL = Plan<L>;
    constexpr int RB = LEV == 1 ? PL::B1 : PL::B2;
    constexpr int RAD = 1 << RB, NS = LEV == 1 ? PL::P : PL::P * PL::R1, SUB = PL::P / RAD;
    constexpr int TWO = LEV == 1 ? 0 : PL::TW2;
    constexpr bool LAST = LEV == PL::NLEV - 1;
    if (act) {
#pragma unroll
        for (int s = 0; s < SUB; ++s) {
            const int j = t + PL::M * s, m = j & (NS - 1);
#pragma unroll
            for (int r = 0; r < RAD; ++r) a[s * RAD + r] = z[PL::pad(j + r * (PL::N / RAD))];
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                const Cx<R> w = tw[TWO + (r - 1) * NS + m];
                a[s * RAD + r] = cmul_tw<R, INV>(w, a[s * RAD + r]);
            }
        }
#pragma unroll
        for (int s = 0; s < SUB; ++s) dft<R, RAD, INV>(a, s * RAD);
    }
    if constexpr (!LAST) {
        __syncthreads();  // every thread has read its values
        if (act) {
#pragma unroll
            for (int s = 0; s < SUB; ++s) {
                const int j = t + PL::M * s, m = j & (NS - 1);
                const int d = (j / NS) * NS * RAD + m;
#pragma unroll
                for (int k = 0; k < RAD; ++k) z[PL::pad(d + k * NS)] = a[s * RAD + k];
            }
        }
        __syncthreads();
    }
}

// The whole line transform: a[r] = element t + r M on entry; on return register s RL + k
// holds element out_index(t, s, k) of the (unnormalised) DFT. z: this line's shared memory
// (unused by a one-level transform); every thread of the block calls this together (barriers), those with
// act = false without work.
template <class R, int L, bool INV>
LB_DEV void line_fft(Cx<R> (&a)[Plan<L>::P], Cx<R>* z, const Cx<R>* __restrict__ tw, int t, bool act = true)
{
    using PL = Plan<L>;
    if (act) dft<R, PL::P, INV>(a, 0);
    if constexpr (PL::NLEV >= 2) {
        if (act) {
#pragma unroll
            for (int k = 0; k < PL::P; ++k) z[PL::pad(t * PL::P + k)] = a[k];
        }
        __syncthreads();
        fft_level<R, L, 1, INV>(a, z, tw, t, act);
    }
    if constexpr (PL::NLEV == 3) fft_level<R, L, 2, INV>(a, z, tw, t, act);
}

// The level twiddles of Plan<L> into shared memory (block-wide; the first barrier of line_fft
// comes before their first use)
template <class R, int L>
LB_DEV void stage_twiddles(Cx<R>* tws, const Cx<R>* __restrict__ tw)
{
    for (int i = threadIdx.x; i < Plan<L>::TWN; i += blockDim.x) tws[i] = tw[i];
}

// Programmatic dependent launch. On small grids the spectral kernels are launched so that each
// may start while its predecessor in the stream drains: a kernel first does the work that reads only
// per-context constants (tables, setup), then waits for its predecessor's results
// (griddepcontrol.wait: the predecessor grid has completed and its memory is visible), and
// only then lets its own dependent launch (launch_dependents). A kernel that runs therefore
// knows that every kernel two or more launches back has completed. Without the launch
// attribute both instructions return at once.
LB_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
LB_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The attribute is set for grid edges up to kPdlMaxN, where every launch of a step fits in one
// wave and the step is bound by launch latency (128^2: 22.0 -> 18.6 us per controlled step);
// at 1024^2, with multi-wave row launches, the early launches measured slower (51.7 -> 57.5 us).
constexpr int kPdlMaxN = 256;

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// R = sum_s r2[s] by one full warp in a fixed order
LB_DEV void sum_cost(const double* r2, int K, double* cost)
{
    double acc = 0.0;
    for (int s = threadIdx.x; s < K; s += 32) acc += r2[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) cost[0] = acc;
}

// ---------------------------------------------------------------------------------------------
// Row kernels. A block takes LPB grid rows: the line transforms run on its first LPB M threads
// (one or more whole warps: LPB = 32 / M lines when M < 32), the per-node work (moments, the
// shifted step) on all THREADS threads, NPT nodes each, through the rows' shared-memory lines.
// Few threads per line transform keep its instruction count low; the node work spread over
// every thread of the block keeps enough population loads in flight, and one or two grid rows
// per block let the blocks of an SM overlap their transforms with other blocks' node work
// (four rows per block, every thread in the transform, measured slower).
// ---------------------------------------------------------------------------------------------
template <int L>
struct RowShape {
    static constexpr int N = Plan<L>::N, M = Plan<L>::M;
    static constexpr int LPB = M >= 32 ? 1 : 32 / M;
    static constexpr int FFT_T = LPB * M;
    static constexpr int THREADS = LPB * N < 32 ? 32 : (LPB * N < 256 ? LPB * N : 256);  // >= one warp
    static constexpr int NPT = (LPB * N + THREADS - 1) / THREADS;  // nodes per thread
    static constexpr int NB = NPT < 4 ? NPT : 4;            // nodes per batch of loads
};

// Slot offsets of the access mode (run-time), per direction: loads of the pre-collision state
// (AB: slot i of x - c_i; AA even: slot i of x; AA odd: slot opp(i) of x - c_i) and stores of
// the post-collision values (AB: slot i of x; AA even: slot opp(i) of x; AA odd: slot i of
// x + c_i). pull / push: whether the loads / stores take the neighbour. 32-bit offsets
// (9 x plane < 2^31 for every grid the spectral calls accept).
struct SlotAccess {
    int ld[9], st[9];
    bool pull, push;
};
LB_DEV SlotAccess slot_access(int mode, int plane)
{
    SlotAccess a;
    a.pull = mode != AA_EVEN;
    a.push = mode == AA_ODD;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        a.ld[i] = ((mode == AA_ODD) ? opp(i) : i) * plane;
        a.st[i] = ((mode == AA_EVEN) ? opp(i) : i) * plane;
    }
    return a;
}
LB_DEV int wrap_dec(int x, int n) { return x == 0 ? n - 1 : x - 1; }
LB_DEV int wrap_inc(int x, int n) { return x == n - 1 ? 0 : x + 1; }

// deviations of node (x, y)'s pre-collision populations
template <class T>
LB_DEV void node_load(const T* buf, const SlotAccess& sa, int x, int y, int n, typename Store<T>::Real* f)
{
    const int xm = sa.pull ? wrap_dec(x, n) : x, xp = sa.pull ? wrap_inc(x, n) : x;
    const int r0 = y * n, rm = sa.pull ? wrap_dec(y, n) * n : r0, rp = sa.pull ? wrap_inc(y, n) * n : r0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c2(i, 0), cy = c2(i, 1);
        const int col = cx > 0 ? xm : (cx < 0 ? xp : x), row = cy > 0 ? rm : (cy < 0 ? rp : r0);
        f[i] = load_pop<D2Q9>(buf + (sa.ld[i] + row + col), i);  // (w of slot opp(i) is w_i)
    }
}

template <class T>
LB_DEV void node_store(T* buf, const SlotAccess& sa, int x, int y, int n, const typename Store<T>::Real* f)
{
    const int xm = sa.push ? wrap_dec(x, n) : x, xp = sa.push ? wrap_inc(x, n) : x;
    const int r0 = y * n, rm = sa.push ? wrap_dec(y, n) * n : r0, rp = sa.push ? wrap_inc(y, n) * n : r0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c2(i, 0), cy = c2(i, 1);
        const int col = cx > 0 ? xp : (cx < 0 ? xm : x), row = cy > 0 ? rp : (cy < 0 ? rm : r0);
        store_pop<D2Q9>(buf + (sa.st[i] + row + col), i, f[i]);
    }
}


template <class R>
constexpr int row_min_blocks() { return sizeof(R) == 4 ? 2 : 1; }

// rows, forward: u of every node of the block's rows (pre-collision moments) into the shared
// lines, then w = u_x + i u_y transformed along x into spec[y][kx]
template <class T, int L>
__global__ void __launch_bounds__(RowShape<L>::THREADS, row_min_blocks<typename Store<T>::Real>())
    k_sc_rows_fwd(const T* buf, int mode, int plane, const Cx<typename Store<T>::Real>* __restrict__ tw,
                  Cx<typename Store<T>::Real>* spec)
{
    using R = typename Store<T>::Real;
    using PL = Plan<L>;
    using RS = RowShape<L>;
    constexpr int n = PL::N;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* zs = reinterpret_cast<Cx<R>*>(sc_smem);
    const int y0 = blockIdx.x * RS::LPB;
    const SlotAccess sa = slot_access(mode, plane);
    const R Fz[3] = {R(0), R(0), R(0)};
    pdl_wait();  // the state comes from the previous launch
    pdl_trigger();
    // a batch's loads are all issued before its first shared-memory store
#pragma unroll
    for (int b = 0; b < RS::NPT; b += RS::NB) {
        R f[RS::NB][9];
#pragma unroll
        for (int u = 0; u < RS::NB; ++u) {
            const int idx = threadIdx.x + (b + u) * RS::THREADS, l = idx / n, x = idx % n;
            if (l < RS::LPB && y0 + l < n) node_load<T>(buf, sa, x, y0 + l, n, f[u]);
        }
#pragma unroll
        for (int u = 0; u < RS::NB; ++u) {
            const int idx = threadIdx.x + (b + u) * RS::THREADS, l = idx / n, x = idx % n;
            if (l < RS::LPB && y0 + l < n) {
                const NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f[u], Fz);
                zs[l * PL::LS + x] = {m.ux, m.uy};
            }
        }
    }
    __syncthreads();
    const int l = threadIdx.x / PL::M, t = threadIdx.x % PL::M;
    const bool act = threadIdx.x < RS::FFT_T && y0 + l < n;
    Cx<R>* z = zs + (act ? l : 0) * PL::LS;
    Cx<R> a[PL::P];
    if (act) {
#pragma unroll
        for (int r = 0; r < PL::P; ++r) a[r] = z[t + r * PL::M];
    }
    __syncthreads();  // the transform overwrites the lines
    line_fft<R, L, false>(a, z, tw, t, act);
    if (act) {
        Cx<R>* row = spec + (y0 + l) * n;
#pragma unroll
        for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
            for (int k = 0; k < PL::RL; ++k) row[PL::out_index(t, s, k)] = a[s * PL::RL + k];
    }
}

// rows, inverse, fused with the step: the inverse DFT of row y of spec gives du of the row's
// nodes (times 1 / scale) in the shared line, and every thread then steps its nodes with the
// equilibrium at u + du (the step reads only the pre-step state, which no kernel of this step
// writes; every node is stepped by one thread). The first warp of block 0 also totals the cost
// R = sum_s r2[s].
template <class T, int L>
__global__ void __launch_bounds__(RowShape<L>::THREADS, row_min_blocks<typename Store<T>::Real>())
    k_sc_rows_inv_step(const Cx<typename Store<T>::Real>* __restrict__ spec,
                       const Cx<typename Store<T>::Real>* __restrict__ tw, typename Store<T>::Real scale,
                       const T* src, T* dst, int mode, int plane, typename Store<T>::Real omega, unsigned* status,
                       const double* r2, double* cost)
{
    using R = typename Store<T>::Real;
    using PL = Plan<L>;
    using RS = RowShape<L>;
    constexpr int n = PL::N;
    extern __shared__ __align__(16) unsigned char sc_smem[];
    Cx<R>* zs = reinterpret_cast<Cx<R>*>(sc_smem);
    const int y0 = blockIdx.x * RS::LPB;
    const SlotAccess sa = slot_access(mode, plane);
    // the first batch of populations is loaded before the transform: its latency overlaps the
    // transform (which only some of the block's warps run), and, the state being the output of
    // the launch five back, it may be loaded before the wait for the previous launch
    R f[RS::NB][9];
#pragma unroll
    for (int u = 0; u < RS::NB; ++u) {
        const int idx = threadIdx.x + u * RS::THREADS, l = idx / n, x = idx % n;
        if (l < RS::LPB && y0 + l < n) node_load<T>(src, sa, x, y0 + l, n, f[u]);
    }
    pdl_wait();  // the filtered spectrum comes from the previous launch
    pdl_trigger();
    if (blockIdx.x == 0 && threadIdx.x < 32) sum_cost(r2, n / 2, cost);
    {
        const int l = threadIdx.x / PL::M, t = threadIdx.x % PL::M;
        const bool act = threadIdx.x < RS::FFT_T && y0 + l < n;
        Cx<R>* z = zs + (act ? l : 0) * PL::LS;
        Cx<R> a[PL::P];
        if (act) {
            const Cx<R>* row = spec + (y0 + l) * n;
#pragma unroll
            for (int r = 0; r < PL::P; ++r) a[r] = row[t + r * PL::M];
        }
        line_fft<R, L, true>(a, z, tw, t, act);
        __syncthreads();  // the last level's reads of the lines are done
        if (act) {
#pragma unroll
            for (int s = 0; s < PL::SUBL; ++s)
#pragma unroll
                for (int k = 0; k < PL::RL; ++k) z[PL::out_index(t, s, k)] = a[s * PL::RL + k];
        }
        __syncthreads();
    }
    const R Fz[3] = {R(0), R(0), R(0)};
    bool bad = false;
#pragma unroll
    for (int b = 0; b < RS::NPT; b += RS::NB) {
        if (b > 0) {
#pragma unroll
            for (int u = 0; u < RS::NB; ++u) {
                const int idx = threadIdx.x + (b + u) * RS::THREADS, l = idx / n, x = idx % n;
                if (l < RS::LPB && y0 + l < n) node_load<T>(src, sa, x, y0 + l, n, f[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < RS::NB; ++u) {
            const int idx = threadIdx.x + (b + u) * RS::THREADS, l = idx / n, x = idx % n;
            if (l < RS::LPB && y0 + l < n) {
                R feq[9];
                NodeMoments<D2Q9, R> m = node_moments<D2Q9, false>(f[u], Fz);
                bad |= !(m.rho > R(0) && m.rho < R(1e30));
                const Cx<R> d = zs[l * PL::LS + x];
                m.ux += scale * d.re;
                m.uy += scale * d.im;
                equilibrium<D2Q9>(m, feq);
#pragma unroll
                for (int i = 0; i < 9; ++i) f[u][i] = f[u][i] - omega * (f[u][i] - feq[i]);
                node_store<T>(dst, sa, x, y0 + l, n, f[u]);
            }
        }
    }
    if (bad) atomicOr(status, 1u);
}

template <class K>
inline cudaError_t sc_smem_attr(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class R, int L>
inline size_t row_smem_bytes()  // the lines, then the twiddles (used by k_sc_rows_inv)
{
    return ((size_t)RowShape<L>::LPB * Plan<L>::LS + Plan<L>::TWN) * sizeof(Cx<R>);
}

// The row kernels of storage type T for the grid edge 2^L: the forward rows (step = false) or
// the inverse rows fused with the step.
template <class T, int L>
cudaError_t rows_sized(const SpectralArgs& s, bool step)
{
    using R = typename Store<T>::Real;
    const OpArgs& a = s.a;
    const int blocks = (Plan<L>::N + RowShape<L>::LPB - 1) / RowShape<L>::LPB;
    const size_t smem = row_smem_bytes<R, L>();
    const int plane = (int)a.g.plane;
    const Cx<R>* tw = (const Cx<R>*)s.tw;
    cudaError_t e;
    if (!step) {
        if ((e = sc_smem_attr(k_sc_rows_fwd<T, L>, smem)) != cudaSuccess) return e;
        return launch_pdl(s.n <= kPdlMaxN, k_sc_rows_fwd<T, L>, blocks, RowShape<L>::THREADS, smem, a.stream, (const T*)a.src, a.mode,
                          plane, tw, (Cx<R>*)s.spec);
    } else {
        const R scale = (R)(-s.kappa / ((double)s.n * s.n * (double)s.n * s.n));
        if ((e = sc_smem_attr(k_sc_rows_inv_step<T, L>, smem)) != cudaSuccess) return e;
        return launch_pdl(s.n <= kPdlMaxN, k_sc_rows_inv_step<T, L>, blocks, RowShape<L>::THREADS, smem, a.stream,
                          (const Cx<R>*)s.spec, tw, scale, (const T*)a.src, (T*)a.dst, a.mode, plane, (R)a.omega,
                          a.status, (const double*)s.r2, s.cost);
    }
}

template <class T>
cudaError_t rows_typed(const SpectralArgs& s, bool step)
{
    switch (s.logn) {
    case 2: return rows_sized<T, 2>(s, step);
    case 3: return rows_sized<T, 3>(s, step);
    case 4: return rows_sized<T, 4>(s, step);
    case 5: return rows_sized<T, 5>(s, step);
    case 6: return rows_sized<T, 6>(s, step);
    case 7: return rows_sized<T, 7>(s, step);
    case 8: return rows_sized<T, 8>(s, step);
    case 9: return rows_sized<T, 9>(s, step);
    case 10: return rows_sized<T, 10>(s, step);
    case 11: return rows_sized<T, 11>(s, step);
    case 12: return rows_sized<T, 12>(s, step);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace sc
}  // namespace lb
