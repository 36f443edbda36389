// The learned collision's inference option (learned_tc): the forward step of Eq. 5
// (Sec. 3.1) with the network in half precision on the tensor cores, for both networks
// (6-24-24-1 with one shared higher-moment rate; 6-53-3 with one rate per higher moment),
// FP32 / FP16 / BF16 population storage, AB and AA layouts. Training and the adjoint keep
// the FP32 kernels (lb_learned_x3.cu); this path only has to be fast.
//
// Warp tiles. A warp handles the 32 consecutive nodes of one grid row (one per lane); blocks
// of four warps walk the grid's tiles with a persistent grid, and each warp loads the
// populations of its next tile into registers before it works on the current one, so the
// loads of one tile are in flight while the network of the previous one runs.
//
// The network: mma.sync m16n8k16 with the warp's 32 nodes as two 16-row tiles.
//   layer 1: inputs [32 x 16] (x_0..x_5, then the constant 1 whose weights are the biases b1)
//            times W1^T, FP16 operands and FP16 accumulation;
//   layer 2: tanh activations (FP16, the accumulator registers of layer 1 are the A operand
//            of layer 2 as they are) times W2^T, again FP16 with FP16 accumulation, b2 as the
//            weights of a constant-1 activation in the padding column 24;
//   output : FP16 operands with FP32 accumulation started from the FP32 output biases.
// tanh is the hardware tanh.approx.f16x2. Half-precision accumulation rounds each
// pre-activation to about 2^-11 relative, the same order as the FP16 activations
// themselves; the network inputs are converted with saturation (no infinities).
//
// The node's own arithmetic (moments, invariants, post-collision populations) is FP32 and
// written per opposite pair: with E_i and O_i the parts of the post-collision bracket that
// are even and odd in c_i, f*_i - w_i = w_i (E_i + O_i) and f*_opp(i) - w_i = w_i (E_i - O_i).
// 1/rho and the rates 1/(e^z + 1/2) use the hardware reciprocal and base-2 exponential
// (relative errors about 2^-22), well inside the network's half-precision error.
//
// Element offsets are 32-bit: the option needs Q x plane < 2^31 (lb_create checks it).
#include <cstring>

#include "lb_learned_node.cuh"

namespace lb {
namespace {

constexpr int kTcWarps = 4;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------- weight tables
// Per lane (g = lane / 4, q = lane % 4) the B-operand words of m16n8k16, each two FP16
// values (lower k in the low half): register 0 holds k = 2q, 2q + 1 of column g,
// register 1 holds k = 2q + 8, 2q + 9.
// 6-24-24-1, w[lane][.]: 0..2 layer 1 (n-tile t; k = 6 carries b1), 3..14 layer 2
// (n-tile t, k-step s, register r at 3 + 4t + 2s + r; k = 24 carries b2), 15..18 the output
// weights (k-step s, register r at 15 + 2s + r; the same in every column).
struct Tc1Tab {
    uint32_t w[32][20];
    float xs[8], xo[8];  // x_k = I_k xs_k + xo_k: standardisation with the invariants' factors folded in
    float b3, pad[3];
};
// 6-53-3, w[lane][.]: 0..6 layer 1 (n-tile t; k = 6 carries b1), 7..14 layer 2 (k-step s,
// register r at 7 + 2s + r; column o < 3 is output o); b2: the lane's output biases
// (columns 2q, 2q + 1).
struct Tc3Tab {
    uint32_t w[32][16];
    float b2[32][4];
    float xs[8], xo[8];
};
static_assert(sizeof(Tc1Tab) % 16 == 0 && sizeof(Tc3Tab) % 16 == 0, "tables copy as 16-byte vectors");

uint16_t f16_bits(double v)
{
    const __half h = __float2half_rn((float)v);
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
}
uint32_t f16_pair(double lo, double hi) { return (uint32_t)f16_bits(lo) | ((uint32_t)f16_bits(hi) << 16); }

// the invariants as tc_inputs forms them lack these factors (I2, I3 carry 3, I4, I5 carry 9)
constexpr double kInvFactor[kNetIn] = {1.0, 3.0, 3.0, 9.0, 9.0, 1.0};

void standardisation(const double* shift, const double* scale, float* xs, float* xo)
{
    for (int k = 0; k < kNetIn; ++k) {
        xs[k] = (float)(scale[k] * kInvFactor[k]);
        xo[k] = (float)(-shift[k] * scale[k]);
    }
}

void pack_tc1(const double* v, Tc1Tab& t)
{
    const double* W1 = v;
    const double* b1 = W1 + kNetHidden * kNetIn;
    const double* W2 = b1 + kNetHidden;
    const double* b2 = W2 + kNetHidden * kNetHidden;
    const double* W3 = b2 + kNetHidden;
    const double* b3 = W3 + kNetHidden;
    const double* shift = b3 + 1;
    const double* scale = shift + kNetIn;
    std::memset(&t, 0, sizeof(t));
    auto w1 = [&](int k, int j) { return k < kNetIn ? W1[j * kNetIn + k] : (k == kNetIn ? b1[j] : 0.0); };
    auto w2 = [&](int k, int j) { return k < kNetHidden ? W2[j * kNetHidden + k] : (k == kNetHidden ? b2[j] : 0.0); };
    auto w3 = [&](int k) { return k < kNetHidden ? W3[k] : 0.0; };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3;
        for (int nt = 0; nt < 3; ++nt) {
            const int j = 8 * nt + g;
            t.w[lane][nt] = f16_pair(w1(2 * q, j), w1(2 * q + 1, j));
            for (int s = 0; s < 2; ++s)
                for (int r = 0; r < 2; ++r) {
                    const int k = 16 * s + 8 * r + 2 * q;
                    t.w[lane][3 + 4 * nt + 2 * s + r] = f16_pair(w2(k, j), w2(k + 1, j));
                }
        }
        for (int s = 0; s < 2; ++s)
            for (int r = 0; r < 2; ++r) {
                const int k = 16 * s + 8 * r + 2 * q;
                t.w[lane][15 + 2 * s + r] = f16_pair(w3(k), w3(k + 1));
            }
    }
    standardisation(shift, scale, t.xs, t.xo);
    t.b3 = (float)b3[0];
}

void pack_tc3(const double* v, Tc3Tab& t)
{
    constexpr int H = kNet3Hidden;
    const double* W1 = v;
    const double* b1 = W1 + H * kNetIn;
    const double* W2 = b1 + H;
    const double* b2 = W2 + 3 * H;
    const double* shift = b2 + 3;
    const double* scale = shift + kNetIn;
    std::memset(&t, 0, sizeof(t));
    auto w1 = [&](int k, int j) { return j >= H ? 0.0 : k < kNetIn ? W1[j * kNetIn + k] : (k == kNetIn ? b1[j] : 0.0); };
    auto w2 = [&](int k, int o) { return (o < 3 && k < H) ? W2[o * H + k] : 0.0; };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3;
        for (int nt = 0; nt < 7; ++nt) t.w[lane][nt] = f16_pair(w1(2 * q, 8 * nt + g), w1(2 * q + 1, 8 * nt + g));
        for (int s = 0; s < 4; ++s)
            for (int r = 0; r < 2; ++r) {
                const int k = 16 * s + 8 * r + 2 * q;
                t.w[lane][7 + 2 * s + r] = f16_pair(w2(k, g), w2(k + 1, g));
            }
        for (int e = 0; e < 2; ++e) t.b2[lane][e] = 2 * q + e < 3 ? (float)b2[2 * q + e] : 0.f;
    }
    standardisation(shift, scale, t.xs, t.xo);
}

// ---------------------------------------------------------------- device helpers
// D = A B + C, FP16 operands and accumulators (two packed registers: rows g and g + 8)
LB_DEV uint32_t mma_hh(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1, uint32_t c0,
                       uint32_t c1, uint32_t& d1)
{
    uint32_t d0;
    asm("mma.sync.aligned.m16n8k16.row.col.f16.f16.f16.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%8,%9};\n"
        : "=r"(d0), "=r"(d1)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "r"(c0), "r"(c1));
    return d0;
}
// D = A B + C, FP16 operands, FP32 accumulators
LB_DEV void mma_hf(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1,
                   const float* c)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}
LB_DEV uint32_t tanh_h2(uint32_t x)
{
    uint32_t y;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
// two FP32 values to packed FP16 (lo in the low half), saturating at the largest finite value
LB_DEV uint32_t pack_h2_sat(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
constexpr uint32_t kOneLow = 0x00003C00u;  // FP16 (1, 0)

// 1 / (e^z + 1/2)
LB_DEV float tc_rate(float z) { return rcp_approx(ex2_approx(z * kLog2e) + 0.5f); }

template <class T> LB_DEV float tc_to_float(T v);
template <> LB_DEV float tc_to_float<float>(float v) { return v; }
template <> LB_DEV float tc_to_float<__half>(__half v) { return __half2float(v); }
template <> LB_DEV float tc_to_float<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Periodic neighbourhood of node (x, y): columns x - 1, x, x + 1 and row offsets
// (y - 1) nx, y nx, (y + 1) nx, wrapped.
struct TcAddr {
    int col[3], row[3];
};
LB_DEV TcAddr tc_addr(int x, int y, int nx, int ny)
{
    TcAddr a;
    a.col[0] = x == 0 ? nx - 1 : x - 1;
    a.col[1] = x;
    a.col[2] = x == nx - 1 ? 0 : x + 1;
    a.row[0] = (y == 0 ? ny - 1 : y - 1) * nx;
    a.row[1] = y * nx;
    a.row[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    return a;
}

// pre-collision deviations f_i - w_i of the node (access modes as in lb_device.cuh)
template <int MODE, class T>
LB_DEV void tc_load(const T* buf, int plane, const TcAddr& a, float* f)
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int s = (MODE == AA_EVEN) ? 0 : -1;
        const T* p = buf + (slot * plane + a.row[1 + s * c2(i, 1)] + a.col[1 + s * c2(i, 0)]);
        f[i] = tc_to_float<T>(MODE == AB ? __ldg(p) : *p);
    }
}
template <int MODE, class T>
LB_DEV void tc_store(T* buf, int plane, const TcAddr& a, const float* f)
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int slot = (MODE == AA_EVEN) ? opp(i) : i;
        const int s = (MODE == AA_ODD) ? 1 : 0;
        Store<T>::store(buf + (slot * plane + a.row[1 + s * c2(i, 1)] + a.col[1 + s * c2(i, 0)]), f[i]);
    }
}

// Moments of one node from the deviations d_i = f_i - w_i, formed from the opposite pairs'
// sums and differences, and the six invariants without their constant factors
// (kInvFactor, folded into the standardisation): rho - 1, |u|^2, tr Pi, Pi:Pi, u.Pi.u and
// sum_g g_g^2 / |H_g|^2_w.
struct TcNode {
    float rho1, rho, ux, uy, pxx, pyy, pxy, g6, g7, g8;
};
LB_DEV TcNode tc_inputs(const float* d, float* I)
{
    TcNode s;
    const float a13 = d[1] + d[2], a24 = d[3] + d[4], e56 = d[5] + d[6], e78 = d[7] + d[8];
    const float ox = d[1] - d[2], oy = d[3] - d[4], o56 = d[5] - d[6], o78 = d[7] - d[8];
    const float diag = e56 + e78;
    s.rho1 = ((d[0] + a13) + a24) + diag;
    const float jx = ox + (o56 + o78), jy = oy + (o56 - o78);
    s.rho = 1.f + s.rho1;
    const float inv = rcp_approx(s.rho);
    s.ux = jx * inv;
    s.uy = jy * inv;
    // Pi = sum c c d - rho u u - (rho - 1)/3 I  (rho u = j)
    const float r3 = s.rho1 * (1.f / 3.f);
    s.pxx = (a13 + diag) - fmaf(jx, s.ux, r3);
    s.pyy = (a24 + diag) - fmaf(jy, s.uy, r3);
    s.pxy = (e56 - e78) - jx * s.uy;
    // g = sum H d for the rows (cx^2 - 1/3) cy, cx (cy^2 - 1/3), (cx^2 - 1/3)(cy^2 - 1/3)
    s.g6 = fmaf(2.f / 3.f, o56 - o78, oy * (-1.f / 3.f));
    s.g7 = fmaf(2.f / 3.f, o56 + o78, ox * (-1.f / 3.f));
    s.g8 = fmaf(4.f / 9.f, diag, fmaf(-2.f / 9.f, a13 + a24, d[0] * (1.f / 9.f)));
    const float uxx = s.ux * s.ux, uyy = s.uy * s.uy, uxy = s.ux * s.uy;
    I[0] = s.rho1;
    I[1] = uxx + uyy;
    I[2] = s.pxx + s.pyy;
    I[3] = fmaf(s.pxx, s.pxx, fmaf(2.f * s.pxy, s.pxy, s.pyy * s.pyy));
    I[4] = fmaf(uxx, s.pxx, fmaf(2.f * uxy, s.pxy, uyy * s.pyy));
    I[5] = fmaf(13.5f, s.g6 * s.g6, fmaf(13.5f, s.g7 * s.g7, 20.25f * s.g8 * s.g8));  // 1/|H|^2_w = 27/2, 27/2, 81/4
    return s;
}

// Post-collision deviations f*_i - w_i = w_i [rho - 1 + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
// + 4.5 (1 - omega) Q_i : Pi + sum_g (1 - omega_g) H_g(c_i) g_g / |H_g|^2_w], with
// kg_g = 1 - omega_g per higher row.
LB_DEV void tc_post(const TcNode& s, float kg6, float kg7, float kg8, float omega, float* f)
{
    const float ks = 4.5f * (1.f - omega);
    const float tr3 = (s.pxx + s.pyy) * (1.f / 3.f);
    const float P0 = fmaf(-s.rho, 1.5f * fmaf(s.ux, s.ux, s.uy * s.uy), s.rho1);
    const float K6 = kg6 * 13.5f * s.g6, K7 = kg7 * 13.5f * s.g7, K8 = kg8 * 20.25f * s.g8;
    // even parts: rest, axis x, axis y, diagonals (1, 1) and (1, -1)
    const float E0 = fmaf(K8, 1.f / 9.f, fmaf(-ks, tr3, P0));
    const float base = fmaf(K8, -2.f / 9.f, P0);
    const float Ea = fmaf(ks, s.pxx - tr3, base), Eb = fmaf(ks, s.pyy - tr3, base);
    const float bd = fmaf(K8, 4.f / 9.f, P0), sd = (s.pxx + s.pyy) - tr3;
    const float Ec = fmaf(ks, fmaf(2.f, s.pxy, sd), bd), Ed = fmaf(ks, fmaf(-2.f, s.pxy, sd), bd);
    // odd parts of the higher rows
    const float Oa = K7 * (-1.f / 3.f), Ob = K6 * (-1.f / 3.f);
    const float Oc = (K6 + K7) * (2.f / 3.f), Od = (K7 - K6) * (2.f / 3.f);
    const float r3 = 3.f * s.rho, r45 = 4.5f * s.rho;
    f[0] = (4.f / 9.f) * E0;
    auto pair = [&](float cu, float E, float O, float w, int i) {
        const float ev = fmaf(r45 * cu, cu, E), od = fmaf(r3, cu, O);
        f[i] = w * (ev + od);
        f[i + 1] = w * (ev - od);
    };
    pair(s.ux, Ea, Oa, 1.f / 9.f, 1);
    pair(s.uy, Eb, Ob, 1.f / 9.f, 3);
    pair(s.ux + s.uy, Ec, Oc, 1.f / 36.f, 5);
    pair(s.ux - s.uy, Ed, Od, 1.f / 36.f, 7);
}

// the warp's standardised inputs, FP16 per node with the constant 1 at k = 6
LB_DEV void tc_stage_inputs(const float* I, const float* xs, const float* xo, uint32_t (*sx)[4], int lane)
{
    float x[kNetIn];
#pragma unroll
    for (int k = 0; k < kNetIn; ++k) x[k] = fmaf(I[k], xs[k], xo[k]);
    uint4 pk;
    pk.x = pack_h2_sat(x[0], x[1]);
    pk.y = pack_h2_sat(x[2], x[3]);
    pk.z = pack_h2_sat(x[4], x[5]);
    pk.w = kOneLow;
    *reinterpret_cast<uint4*>(&sx[lane][0]) = pk;
}

// Tile walk shared by both kernels: tile wt is row wt / ntx, nodes 32 (wt % ntx) + lane.
struct TcWalk {
    int wt, tx, ty, stride, dxt, dyt;
    LB_DEV TcWalk(int first, int stride_, int ntx) : wt(first), stride(stride_)
    {
        ty = first / ntx;
        tx = first - ty * ntx;
        dyt = stride_ / ntx;
        dxt = stride_ - dyt * ntx;
    }
    LB_DEV void next(int ntx)
    {
        wt += stride;
        tx += dxt;
        ty += dyt;
        if (tx >= ntx) {
            tx -= ntx;
            ++ty;
        }
    }
};

template <int MODE, class T>
LB_DEV void tc_fetch(const T* src, int plane, const Geom& g, int tx, int ty, int lane, float* f)
{
    const int x = 32 * tx + lane;
    if (x < g.nx) {
        tc_load<MODE>(src, plane, tc_addr(x, ty, g.nx, g.ny), f);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = 0.f;  // rest state: takes part in the warp's products
    }
}

// ---------------------------------------------------------------- 6-24-24-1
template <class T, int MODE>
__global__ void __launch_bounds__(kTcThreads, 6) k_learned_tc(const T* src, T* dst, Geom g, float omega,
                                                             unsigned* status, const uint32_t* __restrict__ table,
                                                             int ntx, int ntiles)
{
    __shared__ __align__(16) uint32_t stab[sizeof(Tc1Tab) / 4];
    __shared__ __align__(16) uint32_t sx[kTcWarps][32][4];
    __shared__ float sz[kTcWarps][32];
    {
        const uint4* s4 = reinterpret_cast<const uint4*>(table);
        uint4* d4 = reinterpret_cast<uint4*>(stab);
        for (int k = threadIdx.x; k < (int)(sizeof(Tc1Tab) / 16); k += blockDim.x) d4[k] = s4[k];
        __syncthreads();
    }
    const Tc1Tab& tb = *reinterpret_cast<const Tc1Tab*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, q = lane & 3;
    uint32_t w[20];
#pragma unroll
    for (int k = 0; k < 5; ++k) *reinterpret_cast<uint4*>(&w[4 * k]) = *reinterpret_cast<const uint4*>(&tb.w[lane][4 * k]);
    const uint32_t ones = q == 0 ? kOneLow : 0u;  // the constant-1 activation at k = 24
    const float b3[4] = {tb.b3, tb.b3, tb.b3, tb.b3};
    const int plane = (int)g.plane;
    TcWalk tw(blockIdx.x * kTcWarps + warp, gridDim.x * kTcWarps, ntx);
    float fn[9];
    if (tw.wt < ntiles) tc_fetch<MODE>(src, plane, g, tw.tx, tw.ty, lane, fn);
    while (tw.wt < ntiles) {
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fn[i];
        const int x = 32 * tw.tx + lane, y = tw.ty;
        tw.next(ntx);
        if (tw.wt < ntiles) tc_fetch<MODE>(src, plane, g, tw.tx, tw.ty, lane, fn);
        float I[kNetIn];
        const TcNode s = tc_inputs(f, I);
        tc_stage_inputs(I, tb.xs, tb.xo, sx[warp], lane);
        __syncwarp();
        float zc[2][2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const uint32_t a0 = sx[warp][16 * m + gq][q], a1 = sx[warp][16 * m + gq + 8][q];
            uint32_t h1[3][2], h2[3][2];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                uint32_t d1;
                const uint32_t d0 = mma_hh(a0, a1, 0u, 0u, w[t], 0u, 0u, 0u, d1);
                h1[t][0] = tanh_h2(d0);
                h1[t][1] = tanh_h2(d1);
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                uint32_t e1, d1;
                const uint32_t e0 = mma_hh(h1[0][0], h1[0][1], h1[1][0], h1[1][1], w[3 + 4 * t], w[4 + 4 * t], 0u, 0u, e1);
                const uint32_t d0 = mma_hh(h1[2][0], h1[2][1], ones, ones, w[5 + 4 * t], w[6 + 4 * t], e0, e1, d1);
                h2[t][0] = tanh_h2(d0);
                h2[t][1] = tanh_h2(d1);
            }
            float c[4];
            mma_hf(c, h2[0][0], h2[0][1], h2[1][0], h2[1][1], w[15], w[16], b3);
            mma_hf(c, h2[2][0], h2[2][1], 0u, 0u, w[17], w[18], c);
            zc[m][0] = c[0];  // row g of tile m (every column holds z)
            zc[m][1] = c[2];  // row g + 8
        }
        // lane (g, q) hands row 16 (q / 2) + 8 (q % 2) + g to the node's lane
        sz[warp][16 * (q >> 1) + 8 * (q & 1) + gq] = (q >> 1) ? zc[1][q & 1] : zc[0][q & 1];
        __syncwarp();
        const float kg = 1.f - tc_rate(sz[warp][lane]);
        __syncwarp();  // sx and sz are rewritten by the next tile
        if (x < g.nx) {
            tc_post(s, kg, kg, kg, omega, f);
            tc_store<MODE>(dst, plane, tc_addr(x, y, g.nx, g.ny), f);
            if (!(s.rho > 0.f && s.rho < 1e30f)) atomicOr(status, 1u);
        }
    }
}

// ---------------------------------------------------------------- 6-53-3
template <class T, int MODE>
__global__ void __launch_bounds__(kTcThreads, 6) k_learned3_tc(const T* src, T* dst, Geom g, float omega,
                                                              unsigned* status, const uint32_t* __restrict__ table,
                                                              int ntx, int ntiles)
{
    __shared__ __align__(16) uint32_t stab[sizeof(Tc3Tab) / 4];
    __shared__ __align__(16) uint32_t sx[kTcWarps][32][4];
    __shared__ __align__(16) float sz[kTcWarps][32][4];
    {
        const uint4* s4 = reinterpret_cast<const uint4*>(table);
        uint4* d4 = reinterpret_cast<uint4*>(stab);
        for (int k = threadIdx.x; k < (int)(sizeof(Tc3Tab) / 16); k += blockDim.x) d4[k] = s4[k];
        __syncthreads();
    }
    const Tc3Tab& tb = *reinterpret_cast<const Tc3Tab*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, q = lane & 3;
    uint32_t w[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) *reinterpret_cast<uint4*>(&w[4 * k]) = *reinterpret_cast<const uint4*>(&tb.w[lane][4 * k]);
    const float b2[4] = {tb.b2[lane][0], tb.b2[lane][1], tb.b2[lane][0], tb.b2[lane][1]};
    const int plane = (int)g.plane;
    TcWalk tw(blockIdx.x * kTcWarps + warp, gridDim.x * kTcWarps, ntx);
    float fn[9];
    if (tw.wt < ntiles) tc_fetch<MODE>(src, plane, g, tw.tx, tw.ty, lane, fn);
    while (tw.wt < ntiles) {
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fn[i];
        const int x = 32 * tw.tx + lane, y = tw.ty;
        tw.next(ntx);
        if (tw.wt < ntiles) tc_fetch<MODE>(src, plane, g, tw.tx, tw.ty, lane, fn);
        float I[kNetIn];
        const TcNode s = tc_inputs(f, I);
        tc_stage_inputs(I, tb.xs, tb.xo, sx[warp], lane);
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const uint32_t a0 = sx[warp][16 * m + gq][q], a1 = sx[warp][16 * m + gq + 8][q];
            uint32_t h[8][2];
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                uint32_t d1;
                const uint32_t d0 = mma_hh(a0, a1, 0u, 0u, w[t], 0u, 0u, 0u, d1);
                h[t][0] = tanh_h2(d0);
                h[t][1] = tanh_h2(d1);
            }
            h[7][0] = h[7][1] = 0u;
            float c[4] = {b2[0], b2[1], b2[2], b2[3]};
#pragma unroll
            for (int st = 0; st < 4; ++st)
                mma_hf(c, h[2 * st][0], h[2 * st][1], h[2 * st + 1][0], h[2 * st + 1][1], w[7 + 2 * st], w[8 + 2 * st], c);
            // lanes q = 0, 1 hold outputs 2q, 2q + 1 of rows g (c0, c1) and g + 8 (c2, c3)
            if (q < 2) {
                *reinterpret_cast<float2*>(&sz[warp][16 * m + gq][2 * q]) = make_float2(c[0], c[1]);
                *reinterpret_cast<float2*>(&sz[warp][16 * m + gq + 8][2 * q]) = make_float2(c[2], c[3]);
            }
        }
        __syncwarp();
        const float4 z = *reinterpret_cast<const float4*>(&sz[warp][lane][0]);
        __syncwarp();
        // output 0 sets the fourth-order row, 1 the row (cx^2 - 1/3) cy, 2 the row cx (cy^2 - 1/3)
        const float kg8 = 1.f - tc_rate(z.x), kg6 = 1.f - tc_rate(z.y), kg7 = 1.f - tc_rate(z.z);
        if (x < g.nx) {
            tc_post(s, kg6, kg7, kg8, omega, f);
            tc_store<MODE>(dst, plane, tc_addr(x, y, g.nx, g.ny), f);
            if (!(s.rho > 0.f && s.rho < 1e30f)) atomicOr(status, 1u);
        }
    }
}

// persistent grid: the multiprocessors times the blocks that fit one, at most one block per
// four tiles
template <class K>
int tc_grid(K kernel, int sms, int ntiles)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTcThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int want = (ntiles + kTcWarps - 1) / kTcWarps;
    const int cap = (sms > 0 ? sms : 1) * per_sm;
    return want < cap ? want : cap;
}

template <class T>
cudaError_t launch_tc(const OpArgs& a, bool three)
{
    const uint32_t* tab = (const uint32_t*)a.tc_table;
    if (!tab || a.op != OP_UPDATE) return cudaErrorInvalidValue;
    if ((int64_t)9 * a.g.plane > (int64_t)0x7FFFFFFF) return cudaErrorInvalidValue;
    const int ntx = (a.g.nx + 31) / 32;
    const int ntiles = ntx * a.g.ny;
    const T* src = (const T*)a.src;
    T* dst = (T*)a.dst;
    const float omega = (float)a.omega;
#define LB_TC_LAUNCH(KER, MODE)                                                                              \
    do {                                                                                                     \
        const int grid = tc_grid(KER<T, MODE>, a.sms, ntiles);                                               \
        KER<T, MODE><<<grid, kTcThreads, 0, a.stream>>>(src, dst, a.g, omega, a.status, tab, ntx, ntiles);   \
    } while (0)
    if (three) {
        if (a.mode == AB) LB_TC_LAUNCH(k_learned3_tc, AB);
        else if (a.mode == AA_EVEN) LB_TC_LAUNCH(k_learned3_tc, AA_EVEN);
        else LB_TC_LAUNCH(k_learned3_tc, AA_ODD);
    } else {
        if (a.mode == AB) LB_TC_LAUNCH(k_learned_tc, AB);
        else if (a.mode == AA_EVEN) LB_TC_LAUNCH(k_learned_tc, AA_EVEN);
        else LB_TC_LAUNCH(k_learned_tc, AA_ODD);
    }
#undef LB_TC_LAUNCH
    return cudaGetLastError();
}

}  // namespace

size_t learned_tc_table_bytes() { return sizeof(Tc1Tab); }
size_t learned3_tc_table_bytes() { return sizeof(Tc3Tab); }

void learned_tc_pack(const double* net, void* out)
{
    Tc1Tab t;
    pack_tc1(net, t);
    std::memcpy(out, &t, sizeof(t));
}

void learned3_tc_pack(const double* net, void* out)
{
    Tc3Tab t;
    pack_tc3(net, t);
    std::memcpy(out, &t, sizeof(t));
}

cudaError_t run_learned_tc(const OpArgs& a, bool three)
{
    if (a.g.nz != 1) return cudaErrorInvalidValue;
    switch (a.storage) {
    case S_F32: return launch_tc<float>(a, three);
    case S_F16: return launch_tc<__half>(a, three);
    case S_BF16: return launch_tc<__nv_bfloat16>(a, three);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lb
