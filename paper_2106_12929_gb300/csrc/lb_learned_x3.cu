// The learned collision (Eq. 5, Sec. 3.1) in FP32 arithmetic with its networks on the
// tensor cores: the forward step and the discrete adjoint with the network-parameter
// gradient, for both networks (6-24-24-1 with one shared higher-moment rate; 6-53-3 with
// one rate per higher moment) and FP32 / FP16 / BF16 population storage. The FP64
// arithmetic keeps its scalar kernels (lb_learned.cu).
//
// Warp tiles. A warp handles the 32 consecutive nodes of one grid row (one per lane) at a
// time; blocks of four warps loop over the grid's warp tiles with a fixed grid, so every
// warp sums the same nodes on every launch. The per-node parts (moments, network inputs,
// post-collision populations, the adjoint outside the network) run one node per lane. The
// network's products run as warp-level mma.sync m16n8k16 (FP16 operands, FP32
// accumulation) with the warp's 32 nodes as two 16-row tiles: a layer's pre-activations
// are C[node][unit] = sum_k A[node][k] W[unit][k]; the accumulator tiles of one layer,
// packed in pairs, are the A operand of the next, so activations stay in registers.
//
// FP32 operands on FP16 tensor cores: a value v is split into v_hi = fp16(v) and
// v_lo = fp16(v - v_hi) (11 + 11 significant bits), and a product is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation: about 2^-21 relative per
// product, close enough to FP32 that the parameter gradient stays within 1e-4 of the FP64
// reference (a split into BF16 terms, 2^-16 per product, was measured at up to 9e-4).
// FP16 needs its operands in range: the tanh activations are within [-1, 1]; every other
// operand is scaled by a power of two (exact) so that its largest magnitude is in
// [1/2, 1) -- the weight matrices once on the host, the network inputs and the cotangents
// per warp tile over the tile's 32 nodes -- and the products are scaled back in FP32.
// Values far below their operand's largest then keep an absolute error of about 2^-25 of
// it (FP16 subnormals), which is what the matrix products feel.
//
// Parameter gradient. The sums over nodes of outer products (dW = sum_n a_n b_n^T) are
// matrix products whose contraction runs over the nodes. The per-node vectors sit in the
// accumulator layout (rows = nodes); movmatrix.trans turns each packed 8 x 8 block into
// the operand layout with the nodes along k. The products of each 16-node row tile start
// from zero and are added to the warp's FP32 accumulators with round-to-nearest additions
// (the tensor cores' own accumulation may truncate; kept to three products per sum, its
// bias cannot build up over the hundreds of tiles a warp sums). At the end of the launch
// the four warps of a block are added in a fixed order into the block's row of partials,
// which accumulate over the adjoint steps of a run and are reduced deterministically by
// learned_reduce_theta.
//
// Fragment layouts of m16n8k16 (g = lane / 4, q = lane % 4; pairs are two FP16 in one
// register, lower index in the low half): A rows g, g + 8 and columns 2q, 2q + 1 (a0, a1),
// columns 2q + 8, 2q + 9 (a2, a3); B column g, rows 2q, 2q + 1 (b0) and 2q + 8, 2q + 9 (b1);
// C rows g (c0, c1) and g + 8 (c2, c3), columns 2q, 2q + 1.
#include <cmath>
#include <cstring>

#include "lb_learned_node.cuh"

namespace lb {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;

// ---------------------------------------------------------------- fragment helpers
struct Pair {
    uint32_t h, l;  // FP16 leading terms and remainders of two values
};

LB_DEV uint32_t pack2(float lo, float hi)
{
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
LB_DEV float low_half(uint32_t v) { return __low2float(*reinterpret_cast<const __half2*>(&v)); }
LB_DEV float high_half(uint32_t v) { return __high2float(*reinterpret_cast<const __half2*>(&v)); }

LB_DEV Pair split(float a, float b)
{
    Pair p;
    p.h = pack2(a, b);
    p.l = pack2(a - low_half(p.h), b - high_half(p.h));
    return p;
}

// Power of two s with |mx| s in [1/2, 1), and 1/s; s = 1 for zero, subnormal or non-finite mx.
struct Scale {
    float s, inv;
};
LB_DEV Scale pow2_scale(float mx)
{
    const int e = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
    if (e < 1 || e > 252) return {1.f, 1.f};
    return {__uint_as_float((uint32_t)(253 - e) << 23), __uint_as_float((uint32_t)(e + 1) << 23)};
}
// the scale of the largest |v| over the warp
LB_DEV Scale warp_scale(float lane_max)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lane_max = fmaxf(lane_max, __shfl_xor_sync(0xffffffffu, lane_max, o));
    return pow2_scale(lane_max);
}
template <int NT>
LB_DEV float absmax(const float (*t)[4])
{
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < NT; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) m = fmaxf(m, fabsf(t[k][e]));
    return m;
}

// transpose of the 8 x 8 FP16 block held one packed pair per lane (row g, columns 2q, 2q + 1)
LB_DEV uint32_t trans(uint32_t v)
{
    uint32_t r;
    asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(r) : "r"(v));
    return r;
}
LB_DEV Pair trans(Pair p) { return {trans(p.h), trans(p.l)}; }

constexpr Pair kZero = {0u, 0u};

LB_DEV void mma(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct AFrag {
    Pair r[4];
};
struct BFrag {
    Pair r[2];
};

// c += A B in the three-product split
LB_DEV void mma3(float* c, const AFrag& a, const BFrag& b)
{
    mma(c, a.r[0].l, a.r[1].l, a.r[2].l, a.r[3].l, b.r[0].h, b.r[1].h);
    mma(c, a.r[0].h, a.r[1].h, a.r[2].h, a.r[3].h, b.r[0].l, b.r[1].l);
    mma(c, a.r[0].h, a.r[1].h, a.r[2].h, a.r[3].h, b.r[0].h, b.r[1].h);
}

// A operand of k-step s from accumulator tiles 2s and 2s + 1 of one row tile (t[.][4]),
// each value times sc; tiles at or past NT are zero
template <int NT>
LB_DEV AFrag a_from_c(const float (*t)[4], int s, float sc = 1.f)
{
    AFrag a;
    a.r[0] = split(t[2 * s][0] * sc, t[2 * s][1] * sc);
    a.r[1] = split(t[2 * s][2] * sc, t[2 * s][3] * sc);
    if (2 * s + 1 < NT) {
        a.r[2] = split(t[2 * s + 1][0] * sc, t[2 * s + 1][1] * sc);
        a.r[3] = split(t[2 * s + 1][2] * sc, t[2 * s + 1][3] * sc);
    } else {
        a.r[2] = kZero;
        a.r[3] = kZero;
    }
    return a;
}

// B operand stored as [reg][hi/lo][32 lanes] words
LB_DEV BFrag b_load(const uint32_t* p, int lane)
{
    BFrag b;
    b.r[0] = {p[lane], p[32 + lane]};
    b.r[1] = {p[64 + lane], p[96 + lane]};
    return b;
}
// B operand with only its first register (k < 8) nonzero: [hi/lo][32 lanes]
LB_DEV BFrag b_load0(const uint32_t* p, int lane)
{
    BFrag b;
    b.r[0] = {p[lane], p[32 + lane]};
    b.r[1] = kZero;
    return b;
}

// the transposed constant block of a "ones" feature at the first column of an 8-column
// tile: lane (g, q) holds block^T row g = 1 for g == 0
LB_DEV Pair ones_t(int lane) { return {(lane >> 2) == 0 ? 0x3C003C00u : 0u, 0u}; }

// ---------------------------------------------------------------- weight tables
// 6-24-24-1. B operands (weights scaled by powers of two, inverse scales iw1, iw2):
//   w1f: layer 1, B[k][j] = W1[j][k] (k < 6: register 0 only), n-tile t (j = 8t + g)
//   w2f: layer 2, B[k][j] = W2[j][k], n-tile t, k-step s
//   w2b: backward through layer 2, B[k][j] = W2[k][j] (k: layer-2 unit, j: layer-1 unit)
//   w1b: backward through layer 1, B[j][m] = W1[j][m] (m: input, one n-tile), k-step s
// Biases b1t, b2t are the hidden layers' biases times 2 / ln 2 (tanh_of_t takes that
// argument); iw2t = iw2 2 / ln 2.
struct Tab1 {
    uint32_t w1f[3][2][32];
    uint32_t w2f[3][2][2][2][32];
    uint32_t w2b[3][2][2][2][32];
    uint32_t w1b[2][2][2][32];
    float b1t[24], b2t[24], w3[24], shift[6], scale[6];
    float b3, iw1, iw2, iw2t;
};
// 6-53-3 (hidden units padded to 56, outputs to 8):
//   w1f: B[k][j] = W1[j][k] (k < 6), n-tile t < 7
//   w2f: B[j][o] = W2[o][j], k-step s < 4 (j = 16s + ...)
//   w2b: backward through layer 2, B[o][j] = W2[o][j] (o < 3: register 0 only), n-tile t < 7
//   w1b: backward through layer 1, B[j][m] = W1[j][m], k-step s < 4
struct Tab3 {
    uint32_t w1f[7][2][32];
    uint32_t w2f[4][2][2][32];
    uint32_t w2b[7][2][32];
    uint32_t w1b[4][2][2][32];
    float b1t[56], b2[8], shift[6], scale[6];  // b1t = b1 2 / ln 2
    float iw1, iw2, pad[2];
};
static_assert(sizeof(Tab1) % 16 == 0 && sizeof(Tab3) % 16 == 0, "tables copy as 16-byte vectors");

// power of two s with max |W| s in [1/2, 1) over the n FP32-rounded values of W
double host_scale(const double* W, int n)
{
    float mx = 0.f;
    for (int k = 0; k < n; ++k) mx = std::fmax(mx, std::fabs((float)W[k]));
    if (!(mx > 0.f)) return 1.0;
    int e = 0;
    std::frexp(mx, &e);  // mx = f 2^e, f in [1/2, 1)
    return std::ldexp(1.0, -e);
}

// hi / lo words of the pair (a, b) of FP32-rounded weights times the scale s
void split_host(double a, double b, double s, uint32_t& hi, uint32_t& lo)
{
    const float fa = (float)a * (float)s, fb = (float)b * (float)s;
    const __half ha = __float2half_rn(fa), hb = __float2half_rn(fb);
    const __half la = __float2half_rn(fa - __half2float(ha)), lb = __float2half_rn(fb - __half2float(hb));
    uint16_t u[4];
    std::memcpy(&u[0], &ha, 2);
    std::memcpy(&u[1], &hb, 2);
    std::memcpy(&u[2], &la, 2);
    std::memcpy(&u[3], &lb, 2);
    hi = (uint32_t)u[0] | ((uint32_t)u[1] << 16);
    lo = (uint32_t)u[2] | ((uint32_t)u[3] << 16);
}

template <class F>
void put(uint32_t* hl, int lane, F w, int k0, int n, double s)  // words hl[lane], hl[32 + lane]
{
    uint32_t hi, lo;
    split_host(w(k0, n), w(k0 + 1, n), s, hi, lo);
    hl[lane] = hi;
    hl[32 + lane] = lo;
}

void pack1(const double* v, Tab1& t)
{
    const double* W1 = v;
    const double* b1 = W1 + 24 * 6;
    const double* W2 = b1 + 24;
    const double* b2 = W2 + 24 * 24;
    const double* W3 = b2 + 24;
    const double* b3 = W3 + 24;
    const double* shift = b3 + 1;
    const double* scale = shift + 6;
    std::memset(&t, 0, sizeof(t));
    const double s1 = host_scale(W1, 24 * 6), s2 = host_scale(W2, 24 * 24);
    auto w1f = [&](int k, int j) { return k < 6 ? W1[j * 6 + k] : 0.0; };
    auto w2f = [&](int k, int j) { return k < 24 ? W2[j * 24 + k] : 0.0; };
    auto w2b = [&](int k, int j) { return k < 24 ? W2[k * 24 + j] : 0.0; };
    auto w1b = [&](int j, int m) { return (j < 24 && m < 6) ? W1[j * 6 + m] : 0.0; };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3;
        for (int nt = 0; nt < 3; ++nt) {
            put(&t.w1f[nt][0][0], lane, w1f, 2 * q, 8 * nt + g, s1);
            for (int s = 0; s < 2; ++s)
                for (int r = 0; r < 2; ++r) {
                    put(&t.w2f[nt][s][r][0][0], lane, w2f, 16 * s + 8 * r + 2 * q, 8 * nt + g, s2);
                    put(&t.w2b[nt][s][r][0][0], lane, w2b, 16 * s + 8 * r + 2 * q, 8 * nt + g, s2);
                }
        }
        for (int s = 0; s < 2; ++s)
            for (int r = 0; r < 2; ++r) put(&t.w1b[s][r][0][0], lane, w1b, 16 * s + 8 * r + 2 * q, g, s1);
    }
    for (int k = 0; k < 24; ++k) {
        t.b1t[k] = (float)b1[k] * kTwoOverLn2;
        t.b2t[k] = (float)b2[k] * kTwoOverLn2;
        t.w3[k] = (float)W3[k];
    }
    for (int k = 0; k < 6; ++k) {
        t.shift[k] = (float)shift[k];
        t.scale[k] = (float)scale[k];
    }
    t.b3 = (float)b3[0];
    t.iw1 = (float)(1.0 / s1);
    t.iw2 = (float)(1.0 / s2);
    t.iw2t = t.iw2 * kTwoOverLn2;
}

void pack3(const double* v, Tab3& t)
{
    constexpr int H = kNet3Hidden;
    const double* W1 = v;
    const double* b1 = W1 + H * 6;
    const double* W2 = b1 + H;
    const double* b2 = W2 + 3 * H;
    const double* shift = b2 + 3;
    const double* scale = shift + 6;
    std::memset(&t, 0, sizeof(t));
    const double s1 = host_scale(W1, H * 6), s2 = host_scale(W2, 3 * H);
    auto w1f = [&](int k, int j) { return (k < 6 && j < H) ? W1[j * 6 + k] : 0.0; };
    auto w2f = [&](int j, int o) { return (j < H && o < 3) ? W2[o * H + j] : 0.0; };
    auto w2b = [&](int o, int j) { return (o < 3 && j < H) ? W2[o * H + j] : 0.0; };
    auto w1b = [&](int j, int m) { return (j < H && m < 6) ? W1[j * 6 + m] : 0.0; };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3;
        for (int nt = 0; nt < 7; ++nt) {
            put(&t.w1f[nt][0][0], lane, w1f, 2 * q, 8 * nt + g, s1);
            put(&t.w2b[nt][0][0], lane, w2b, 2 * q, 8 * nt + g, s2);
        }
        for (int s = 0; s < 4; ++s)
            for (int r = 0; r < 2; ++r) {
                put(&t.w2f[s][r][0][0], lane, w2f, 16 * s + 8 * r + 2 * q, g, s2);
                put(&t.w1b[s][r][0][0], lane, w1b, 16 * s + 8 * r + 2 * q, g, s1);
            }
    }
    for (int k = 0; k < 56; ++k) t.b1t[k] = k < H ? (float)b1[k] * kTwoOverLn2 : 0.f;
    for (int k = 0; k < 8; ++k) t.b2[k] = k < 3 ? (float)b2[k] : 0.f;
    for (int k = 0; k < 6; ++k) {
        t.shift[k] = (float)shift[k];
        t.scale[k] = (float)scale[k];
    }
    t.iw1 = (float)(1.0 / s1);
    t.iw2 = (float)(1.0 / s2);
}

// ---------------------------------------------------------------- per-warp-tile pieces
template <class Tab>
LB_DEV void stage_table(uint32_t* stab, const uint32_t* __restrict__ table)
{
    constexpr int kVec = (int)(sizeof(Tab) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(table);
    uint4* dst = reinterpret_cast<uint4*>(stab);
    for (int k = threadIdx.x; k < kVec; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// Nodes of warp tile wt: row y, x = x0 + lane; lanes past the row's end (valid = false)
// take part in the warp's matrix products with the rest state and zero cotangents.
struct TileNode {
    int x, y, n;
    bool valid;
    Nbr nb;
};
template <class T>
LB_DEV TileNode tile_node(const Geom& g, unsigned wt, unsigned ntx, int lane)
{
    TileNode t;
    const unsigned y = wt / ntx;
    t.y = (int)y;
    t.x = (int)(wt - y * ntx) * 32 + lane;
    t.valid = t.x < g.nx;
    const int xs = t.valid ? t.x : 0;
    t.nb = make_nbr_2d<sizeof(T)>(g, xs, t.y);
    t.n = xs + g.nx * t.y;
    return t;
}

// Standardised network inputs x_0..5, the constant 1 (column 6: the first-layer bias of the
// parameter gradient; its layer-1 weights are zero) and 0, scaled by the warp's power of two,
// split and stored per node. Returns the scale.
LB_DEV Scale stage_inputs(const float* I, const float* shift, const float* scale, uint32_t (*sx)[32][4], int lane)
{
    float xv[8];
    float mx = 1.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        xv[k] = (I[k] - shift[k]) * scale[k];
        mx = fmaxf(mx, fabsf(xv[k]));
    }
    xv[6] = 1.f;
    xv[7] = 0.f;
    const Scale sc = warp_scale(mx);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const Pair pr = split(xv[2 * p] * sc.s, xv[2 * p + 1] * sc.s);
        sx[0][lane][p] = pr.h;
        sx[1][lane][p] = pr.l;
    }
    return sc;
}

// layer-1 A operand of row tile m from the staged inputs (k < 8; k = 8..15 zero)
LB_DEV AFrag a_inputs(const uint32_t (*sx)[32][4], int m, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    AFrag a;
    a.r[0] = {sx[0][16 * m + g][q], sx[1][16 * m + g][q]};
    a.r[1] = {sx[0][16 * m + g + 8][q], sx[1][16 * m + g + 8][q]};
    a.r[2] = kZero;
    a.r[3] = kZero;
    return a;
}

// value of row r (0..31 = the lane's node) from per-row-group values v[4] (index 2m + half,
// row 16m + 8 half + g, held by lane 4g after the reduction over q)
LB_DEV float to_node(const float* v, int lane)
{
    const int src = 4 * (lane & 7);
    const float v0 = __shfl_sync(0xffffffffu, v[0], src), v1 = __shfl_sync(0xffffffffu, v[1], src);
    const float v2 = __shfl_sync(0xffffffffu, v[2], src), v3 = __shfl_sync(0xffffffffu, v[3], src);
    const int sel = lane >> 3;
    return sel == 0 ? v0 : sel == 1 ? v1 : sel == 2 ? v2 : v3;
}

// ---------------------------------------------------------------- asynchronous copies
// 4-byte global -> shared copies (cp.async) that complete in the background: the adjoint
// fetches a tile's state and cotangent while the network of the tile before it runs.
LB_DEV void cp_async4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
LB_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
LB_DEV void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The pre-collision state of the lane's node (pull: slot i of x - c_i) into pf[i][lane]; FP32
// storage only (the copies move whole 4-byte words)
LB_DEV void fetch_state(const float* state, const TileNode& nd, float (*pf)[32], int lane)
{
    if (!nd.valid) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async4(&pf[i][lane], at(state, nd.nb, i, -c2(i, 0), -c2(i, 1), 0));
}
// the cotangent mu_i of the post-collision value that node x sends to x + c_i
LB_DEV void fetch_mu(const float* lam_in, const Geom& g, const TileNode& nd, float (*pm)[32], int lane)
{
    if (!nd.valid) return;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        cp_async4(&pm[i][lane], lam_in + ((int64_t)i * g.plane + nd.nb.node(g, c2(i, 0), c2(i, 1), 0)));
}

// ---------------------------------------------------------------- 6-24-24-1
// The network of row tile m: h1, h2 (accumulator layout) and the partial output sums of rows
// g and g + 8 over the lane's columns; kxt = 2 / ln 2 / (input scale x W1 scale).
LB_DEV void net1_forward(const Tab1& tb, const AFrag& ax, float kxt, int lane, float (*h1)[4], float (*h2)[4],
                         float& z0, float& z1)
{
    const int q = lane & 3;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma3(c, ax, b_load0(&tb.w1f[t][0][0], lane));
        const float b0 = tb.b1t[8 * t + 2 * q], b1 = tb.b1t[8 * t + 2 * q + 1];
        h1[t][0] = tanh_of_t(fmaf(c[0], kxt, b0));
        h1[t][1] = tanh_of_t(fmaf(c[1], kxt, b1));
        h1[t][2] = tanh_of_t(fmaf(c[2], kxt, b0));
        h1[t][3] = tanh_of_t(fmaf(c[3], kxt, b1));
    }
    const AFrag a0 = a_from_c<3>(h1, 0), a1 = a_from_c<3>(h1, 1);
    z0 = 0.f;
    z1 = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma3(c, a0, b_load(&tb.w2f[t][0][0][0][0], lane));
        mma3(c, a1, b_load(&tb.w2f[t][1][0][0][0], lane));
        const float b0 = tb.b2t[8 * t + 2 * q], b1 = tb.b2t[8 * t + 2 * q + 1];
        h2[t][0] = tanh_of_t(fmaf(c[0], tb.iw2t, b0));
        h2[t][1] = tanh_of_t(fmaf(c[1], tb.iw2t, b1));
        h2[t][2] = tanh_of_t(fmaf(c[2], tb.iw2t, b0));
        h2[t][3] = tanh_of_t(fmaf(c[3], tb.iw2t, b1));
        const float wa = tb.w3[8 * t + 2 * q], wb = tb.w3[8 * t + 2 * q + 1];
        z0 += wa * h2[t][0] + wb * h2[t][1];
        z1 += wa * h2[t][2] + wb * h2[t][3];
    }
}

// per-lane output z of the lane's node from the partial sums zp[2m + half]
LB_DEV float reduce_z(float* zp, int lane)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        zp[k] += __shfl_xor_sync(0xffffffffu, zp[k], 1);
        zp[k] += __shfl_xor_sync(0xffffffffu, zp[k], 2);
    }
    return to_node(zp, lane);
}

template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_learned_fwd_x3(const T* src, T* dst, Geom g, float omega, unsigned* status,
                                                             const uint32_t* __restrict__ table, unsigned ntx, unsigned ntiles)
{
    __shared__ __align__(16) uint32_t stab[sizeof(Tab1) / 4];
    __shared__ uint32_t sx[kWarps][2][32][4];
    stage_table<Tab1>(stab, table);
    const Tab1& tb = *reinterpret_cast<const Tab1*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned wt = blockIdx.x * kWarps + warp; wt < ntiles; wt += gridDim.x * kWarps) {
        const TileNode nd = tile_node<T>(g, wt, ntx, lane);
        float f[9];
        if (nd.valid) load_node<D2Q9, MODE>(src, g, nd.nb, nd.n, f);
        else
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = 0.f;
        LearnedMoments<float> s;
        float I[kNetIn];
        learned_inputs(f, s, I);
        const Scale sx_sc = stage_inputs(I, tb.shift, tb.scale, sx[warp], lane);
        __syncwarp();
        const float kxt = sx_sc.inv * tb.iw1 * kTwoOverLn2;
        float zp[4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            float h1[3][4], h2[3][4];
            net1_forward(tb, a_inputs(sx[warp], m, lane), kxt, lane, h1, h2, zp[2 * m], zp[2 * m + 1]);
        }
        __syncwarp();  // the staged inputs are read before the next tile overwrites them
        const float z = reduce_z(zp, lane) + tb.b3;
        const float omg = recip(expf(z) + 0.5f);
        if (nd.valid) {
            learned_post(s, omg, omega, f);
            store_node<D2Q9, MODE>(dst, g, nd.nb, nd.n, f);
            if (!(s.m.rho > 0.f && s.m.rho < 1e30f)) atomicOr(status, 1u);
        }
    }
}

// Adjoint step with the parameter gradient (6-24-24-1). Partials: one row of kNetTheta
// floats per block, added to. The hidden activations of the tile wait in shared memory
// (accumulator layout, one float4 per lane and tile) while the node-parallel adjoint runs;
// the backward pass then takes one 16-node row tile at a time.
struct Adj1Smem {
    uint32_t stab[sizeof(Tab1) / 4];
    uint32_t sx[kWarps][2][32][4];
    union {
        float sh[kWarps][2][2][3][32][4];  // [warp][h1, h2][row tile][n-tile][lane], during the loop
        float red[kWarps][kNetTheta];      // the warps' sums, after it
    };
    float sg[kWarps][32][9];
    float acc[kWarps][36][32];  // dW2^T (24 values) and dW1^T (12) per lane
    float pf[kWarps][9][32];    // the tile's state (FP32 storage), copied in during the tile before
    float pm[kWarps][9][32];    // the tile's cotangent mu, copied in while its network runs
};

template <class T>
__global__ void __launch_bounds__(kThreads, 3) k_learned_adj_x3(const T* state, const float* lam_in, float* lam_out,
                                                                Geom g, float omega, float* gth_partials,
                                                                const uint32_t* __restrict__ table, unsigned ntx,
                                                                unsigned ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Adj1Smem& sm = *reinterpret_cast<Adj1Smem*>(smem_raw);
    auto& stab = sm.stab;
    auto& sx = sm.sx;
    auto& sh = sm.sh;
    auto& sg = sm.sg;
    auto& red = sm.red;
    auto& acc = sm.acc;
    stage_table<Tab1>(stab, table);
    const Tab1& tb = *reinterpret_cast<const Tab1*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, q = lane & 3;
    // parameter-gradient accumulators: dW2^T (rows k < 24, row 24 = b2; columns j) and
    // dW1^T (rows m < 6, row 6 = b1; columns j) in accumulator layout, one shared-memory slot
    // per lane and value (registers are the occupancy limit); dW3 over the lane's columns and
    // b3 over the lane's nodes in registers
    float* aW2 = &acc[warp][0][lane];   // value 12 mm + 4 t + e at aW2[32 (12 mm + 4 t + e)]
    float* aW1 = &acc[warp][24][lane];  // value 4 t + e at aW1[32 (4 t + e)]
#pragma unroll
    for (int v = 0; v < 36; ++v) acc[warp][v][lane] = 0.f;
    float aW3[3][2], aB3 = 0.f;
#pragma unroll
    for (int t = 0; t < 3; ++t) aW3[t][0] = aW3[t][1] = 0.f;
    // Copies: the state of tile wt arrives during tile wt - stride (FP32 storage), its cotangent
    // during its own network; each lane copies and reads only its own column of pf and pm, and
    // reuses a slot only after the values read from it have been used.
    constexpr bool kAsyncState = sizeof(T) == 4;
    const unsigned stride = gridDim.x * kWarps;
    if (kAsyncState && blockIdx.x * kWarps + warp < ntiles) {
        fetch_state((const float*)state, tile_node<T>(g, blockIdx.x * kWarps + warp, ntx, lane), sm.pf[warp], lane);
        cp_async_commit();
    }
    for (unsigned wt = blockIdx.x * kWarps + warp; wt < ntiles; wt += stride) {
        const TileNode nd = tile_node<T>(g, wt, ntx, lane);
        LearnedMoments<float> s;
        Scale sx_sc;
        float z;
        {
            float f[9];
            cp_async_wait<0>();
            if (nd.valid) {
                if constexpr (kAsyncState) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = sm.pf[warp][i][lane];
                } else {
                    load_node<D2Q9, AB>(state, g, nd.nb, nd.n, f);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = 0.f;
            }
            fetch_mu(lam_in, g, nd, sm.pm[warp], lane);
            cp_async_commit();
            float I[kNetIn];
            learned_inputs(f, s, I);
            if (kAsyncState && wt + stride < ntiles) {
                fetch_state((const float*)state, tile_node<T>(g, wt + stride, ntx, lane), sm.pf[warp], lane);
                cp_async_commit();
            }
            sx_sc = stage_inputs(I, tb.shift, tb.scale, sx[warp], lane);
            __syncwarp();
            const float kxt = sx_sc.inv * tb.iw1 * kTwoOverLn2;
            float zp[4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                float h1[3][4], h2[3][4];
                net1_forward(tb, a_inputs(sx[warp], m, lane), kxt, lane, h1, h2, zp[2 * m], zp[2 * m + 1]);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    *reinterpret_cast<float4*>(&sh[warp][0][m][t][lane][0]) = make_float4(h1[t][0], h1[t][1], h1[t][2], h1[t][3]);
                    *reinterpret_cast<float4*>(&sh[warp][1][m][t][lane][0]) = make_float4(h2[t][0], h2[t][1], h2[t][2], h2[t][3]);
                }
            }
            z = reduce_z(zp, lane) + tb.b3;
        }
        const float ez = expf(z);
        const float omg = recip(ez + 0.5f);
        // the node's adjoint through the equilibrium, the stress rows and the higher rows
        LearnedCot<float> c;
        {
            float mu[9];
            // the cotangent's group; the next tile's state (committed after it) may still be in flight
            if (kAsyncState && wt + stride < ntiles) cp_async_wait<1>();
            else cp_async_wait<0>();
            if (nd.valid)
#pragma unroll
                for (int i = 0; i < 9; ++i) mu[i] = sm.pm[warp][i][lane];
            else
#pragma unroll
                for (int i = 0; i < 9; ++i) mu[i] = 0.f;
            c = learned_adj_head(s, mu, omega);
        }
        const float kg = 1.f - omg;
        c.gg6 = kg * c.q6;
        c.gg7 = kg * c.q7;
        c.gg8 = kg * c.q8;
        const float gomg = -(c.q6 * s.g6 + c.q7 * s.g7 + c.q8 * s.g8);
        const float gz = nd.valid ? gomg * (-ez * omg * omg) : 0.f;  // d w_g / dz = -e^z w_g^2
        aB3 += gz;
        const Pair one = ones_t(lane);
#pragma unroll 1
        for (int m = 0; m < 2; ++m) {
            float h[3][4];
            // back through W3 and the second tanh: ga2 = gz W3 (1 - h2^2); dW3 += gz h2
            float ga[3][4];
            {
                const float gr0 = __shfl_sync(0xffffffffu, gz, 16 * m + gq);
                const float gr1 = __shfl_sync(0xffffffffu, gz, 16 * m + 8 + gq);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const float4 v = *reinterpret_cast<const float4*>(&sh[warp][1][m][t][lane][0]);
                    const float hv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float gr = (e < 2) ? gr0 : gr1;
                        ga[t][e] = gr * tb.w3[8 * t + 2 * q + (e & 1)] * (1.f - hv[e] * hv[e]);
                        aW3[t][e & 1] += gr * hv[e];
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const float4 v = *reinterpret_cast<const float4*>(&sh[warp][0][m][t][lane][0]);
                h[t][0] = v.x;
                h[t][1] = v.y;
                h[t][2] = v.z;
                h[t][3] = v.w;
            }
            // back through W2 and the first tanh: ga1 = (ga2 W2) (1 - h1^2); dW2 (and b2) with
            // the nodes as the contraction, this row tile being its k-step:
            // D[k][j] = sum_n [h1 | 1][n][k] ga2[n][j]
            {
                const Scale s2 = warp_scale(absmax<3>(ga));
                const AFrag g0 = a_from_c<3>(ga, 0, s2.s), g1 = a_from_c<3>(ga, 1, s2.s);
                const float k2 = s2.inv * tb.iw2;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    float cc[4] = {0.f, 0.f, 0.f, 0.f};
                    mma3(cc, g0, b_load(&tb.w2b[t][0][0][0][0], lane));
                    mma3(cc, g1, b_load(&tb.w2b[t][1][0][0][0], lane));
#pragma unroll
                    for (int e = 0; e < 4; ++e) ga[t][e] = cc[e] * k2 * (1.f - h[t][e] * h[t][e]);  // now ga1
                }
                const BFrag bv[3] = {{{trans(g0.r[0]), trans(g0.r[1])}}, {{trans(g0.r[2]), trans(g0.r[3])}},
                                     {{trans(g1.r[0]), trans(g1.r[1])}}};
                Pair u[3][2];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    u[t][0] = trans(split(h[t][0], h[t][1]));
                    u[t][1] = trans(split(h[t][2], h[t][3]));
                }
                const AFrag au[2] = {{{u[0][0], u[1][0], u[0][1], u[1][1]}}, {{u[2][0], one, u[2][1], one}}};
#pragma unroll
                for (int mm = 0; mm < 2; ++mm)
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        float cc[4] = {0.f, 0.f, 0.f, 0.f};
                        mma3(cc, au[mm], bv[t]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            float& a = aW2[32 * (12 * mm + 4 * t + e)];
                            a = fmaf(cc[e], s2.inv, a);
                        }
                    }
            }
            // back through W1: gI = (ga1 W1) scale (into sg); dW1 (and b1):
            // D[m][j] = sum_n [x | 1][n][m] ga1[n][j]
            {
                const Scale s1 = warp_scale(absmax<3>(ga));
                const AFrag g0 = a_from_c<3>(ga, 0, s1.s), g1 = a_from_c<3>(ga, 1, s1.s);
                float cc[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(cc, g0, b_load(&tb.w1b[0][0][0][0], lane));
                mma3(cc, g1, b_load(&tb.w1b[1][0][0][0], lane));
                const float k1 = s1.inv * tb.iw1;
                sg[warp][16 * m + gq][2 * q] = cc[0] * k1;
                sg[warp][16 * m + gq][2 * q + 1] = cc[1] * k1;
                sg[warp][16 * m + gq + 8][2 * q] = cc[2] * k1;
                sg[warp][16 * m + gq + 8][2 * q + 1] = cc[3] * k1;
                const AFrag ax = a_inputs(sx[warp], m, lane);
                const AFrag au = {{trans(ax.r[0]), kZero, trans(ax.r[1]), kZero}};
                const BFrag bv[3] = {{{trans(g0.r[0]), trans(g0.r[1])}}, {{trans(g0.r[2]), trans(g0.r[3])}},
                                     {{trans(g1.r[0]), trans(g1.r[1])}}};
                const float kd1 = s1.inv * sx_sc.inv;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    float cw[4] = {0.f, 0.f, 0.f, 0.f};
                    mma3(cw, au, bv[t]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float& a = aW1[32 * (4 * t + e)];
                        a = fmaf(cw[e], kd1, a);
                    }
                }
            }
        }
        __syncwarp();
        float gI[kNetIn];
#pragma unroll
        for (int k = 0; k < kNetIn; ++k) gI[k] = sg[warp][lane][k] * tb.scale[k];
        if (nd.valid) learned_adj_tail(s, c, gI, lam_out, g.plane, nd.n);
        __syncwarp();  // staged inputs, activations and gI rows are read before the next tile writes them
    }
    // the warp's sums into red[warp][.] in parameter order (red overlays the activations, which
    // every warp of the block has finished with)
    __syncthreads();
    constexpr int oW1 = 0, ob1 = 24 * 6, oW2 = ob1 + 24, ob2 = oW2 + 24 * 24, oW3 = ob2 + 24, ob3 = oW3 + 24;
    float* rw = red[warp];
#pragma unroll
    for (int mm = 0; mm < 2; ++mm)
#pragma unroll
        for (int t = 0; t < 3; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 16 * mm + gq + 8 * (e >> 1), j = 8 * t + 2 * q + (e & 1);
                const float v = aW2[32 * (12 * mm + 4 * t + e)];
                if (k < 24) rw[oW2 + j * 24 + k] = v;
                else if (k == 24) rw[ob2 + j] = v;
            }
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int e = 0; e < 2; ++e) {  // rows 8..15 (e >= 2) hold nothing
            const int mrow = gq, j = 8 * t + 2 * q + e;
            const float v = aW1[32 * (4 * t + e)];
            if (mrow < 6) rw[oW1 + j * 6 + mrow] = v;
            else if (mrow == 6) rw[ob1 + j] = v;
        }
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            float v = aW3[t][e];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (gq == 0) rw[oW3 + 8 * t + 2 * q + e] = v;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) aB3 += __shfl_xor_sync(0xffffffffu, aB3, o);
    if (lane == 0) rw[ob3] = aB3;
    __syncthreads();  // every warp's sums are in red
    float* out = gth_partials + (int64_t)blockIdx.x * kNetTheta;
    for (int o = threadIdx.x; o < kNetTheta; o += kThreads) out[o] += ((red[0][o] + red[1][o]) + red[2][o]) + red[3][o];
}

// ---------------------------------------------------------------- 6-53-3
// layer 1 of row tile m: h (accumulator layout, 7 tiles, units >= 53 are zero); kxt as above
LB_DEV void net3_layer1(const Tab3& tb, const AFrag& ax, float kxt, int lane, float (*h)[4])
{
    const int q = lane & 3;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma3(c, ax, b_load0(&tb.w1f[t][0][0], lane));
        const float b0 = tb.b1t[8 * t + 2 * q], b1 = tb.b1t[8 * t + 2 * q + 1];
        h[t][0] = tanh_of_t(fmaf(c[0], kxt, b0));
        h[t][1] = tanh_of_t(fmaf(c[1], kxt, b1));
        h[t][2] = tanh_of_t(fmaf(c[2], kxt, b0));
        h[t][3] = tanh_of_t(fmaf(c[3], kxt, b1));
    }
}

// layer 2 of row tile m: zc (outputs o = 2q, 2q + 1 of rows g, g + 8)
LB_DEV void net3_layer2(const Tab3& tb, const float (*h)[4], int lane, float* zc)
{
    const int q = lane & 3;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int s = 0; s < 4; ++s) mma3(c, a_from_c<7>(h, s), b_load(&tb.w2f[s][0][0][0], lane));
    zc[0] = fmaf(c[0], tb.iw2, tb.b2[2 * q]);
    zc[1] = fmaf(c[1], tb.iw2, tb.b2[2 * q + 1]);
    zc[2] = fmaf(c[2], tb.iw2, tb.b2[2 * q]);
    zc[3] = fmaf(c[3], tb.iw2, tb.b2[2 * q + 1]);
}

// the three outputs of the lane's node from both row tiles' zc
LB_DEV void net3_outputs(const float (*zc)[4], int lane, float* z)
{
    // node r = lane: row tile r / 16, row r % 16 (g = row % 8, upper half = row / 8); its
    // outputs 0, 1 sit in lane 4g (c0, c1 or c2, c3) and output 2 in lane 4g + 1 (c0 or c2)
    const int row = lane & 15, src0 = 4 * (row & 7), up = row >> 3, mt = lane >> 4;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float v0 = __shfl_sync(0xffffffffu, zc[m][0], src0), v1 = __shfl_sync(0xffffffffu, zc[m][1], src0);
        const float v2 = __shfl_sync(0xffffffffu, zc[m][2], src0), v3 = __shfl_sync(0xffffffffu, zc[m][3], src0);
        const float w0 = __shfl_sync(0xffffffffu, zc[m][0], src0 + 1);
        const float w2 = __shfl_sync(0xffffffffu, zc[m][2], src0 + 1);
        if (m == mt) {
            z[0] = up ? v2 : v0;
            z[1] = up ? v3 : v1;
            z[2] = up ? w2 : w0;
        }
    }
}

template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) k_learned3_fwd_x3(const T* src, T* dst, Geom g, float omega,
                                                              unsigned* status, const uint32_t* __restrict__ table,
                                                              unsigned ntx, unsigned ntiles)
{
    __shared__ __align__(16) uint32_t stab[sizeof(Tab3) / 4];
    __shared__ uint32_t sx[kWarps][2][32][4];
    stage_table<Tab3>(stab, table);
    const Tab3& tb = *reinterpret_cast<const Tab3*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned wt = blockIdx.x * kWarps + warp; wt < ntiles; wt += gridDim.x * kWarps) {
        const TileNode nd = tile_node<T>(g, wt, ntx, lane);
        float f[9];
        if (nd.valid) load_node<D2Q9, MODE>(src, g, nd.nb, nd.n, f);
        else
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = 0.f;
        LearnedMoments<float> s;
        float I[kNetIn];
        learned_inputs(f, s, I);
        const Scale sx_sc = stage_inputs(I, tb.shift, tb.scale, sx[warp], lane);
        __syncwarp();
        const float kxt = sx_sc.inv * tb.iw1 * kTwoOverLn2;
        float zc[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            float h[7][4];
            net3_layer1(tb, a_inputs(sx[warp], m, lane), kxt, lane, h);
            net3_layer2(tb, h, lane, zc[m]);
        }
        __syncwarp();
        float z[3], omg[3];
        net3_outputs(zc, lane, z);
#pragma unroll
        for (int o = 0; o < 3; ++o) omg[net3_row(o)] = recip(expf(z[o]) + 0.5f);
        if (nd.valid) {
            learned3_post(s, omg, omega, f);
            store_node<D2Q9, MODE>(dst, g, nd.nb, nd.n, f);
            if (!(s.m.rho > 0.f && s.m.rho < 1e30f)) atomicOr(status, 1u);
        }
    }
}

// Adjoint step with the parameter gradient (6-53-3). The hidden activations of the tile are
// kept in shared memory (accumulator layout, one float4 per lane and tile).
struct Adj3Smem {
    uint32_t stab[sizeof(Tab3) / 4];
    uint32_t sx[kWarps][2][32][4];
    uint32_t sz[kWarps][2][32][4];  // output cotangents gz_0..2, scaled and split, per node
    union {
        float sh[kWarps][2][7][32][4];  // hidden activations per row tile, during the loop
        float red[kWarps][kNet3Theta];  // the warps' sums, after it
    };
    float sg[kWarps][32][9];
    float acc[kWarps][44][32];  // dW1^T (28 values) and dW2^T (16) per lane
};

template <class T>
__global__ void __launch_bounds__(kThreads, 3) k_learned3_adj_x3(const T* state, const float* lam_in,
                                                                 float* lam_out, Geom g, float omega,
                                                                 float* gth_partials,
                                                                 const uint32_t* __restrict__ table, unsigned ntx,
                                                                 unsigned ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Adj3Smem& sm = *reinterpret_cast<Adj3Smem*>(smem_raw);
    auto& stab = sm.stab;
    auto& sx = sm.sx;
    auto& sz = sm.sz;
    auto& sh = sm.sh;
    auto& sg = sm.sg;
    auto& red = sm.red;
    auto& acc = sm.acc;
    stage_table<Tab3>(stab, table);
    const Tab3& tb = *reinterpret_cast<const Tab3*>(stab);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, q = lane & 3;
    // dW1^T: rows m < 6 (row 6 = b1), columns j < 53; dW2^T: rows j < 53 (row 56 = b2), columns
    // o < 3; in accumulator layout, one shared-memory slot per lane and value
    float* aW1 = &acc[warp][0][lane];   // value 4 t + e at aW1[32 (4 t + e)]
    float* aW2 = &acc[warp][28][lane];  // value 4 mm + e at aW2[32 (4 mm + e)]
#pragma unroll
    for (int v = 0; v < 44; ++v) acc[warp][v][lane] = 0.f;
    for (unsigned wt = blockIdx.x * kWarps + warp; wt < ntiles; wt += gridDim.x * kWarps) {
        const TileNode nd = tile_node<T>(g, wt, ntx, lane);
        float f[9], mu[9];
        if (nd.valid) {
            load_node<D2Q9, AB>(state, g, nd.nb, nd.n, f);
#pragma unroll
            for (int i = 0; i < 9; ++i) mu[i] = lam_in[(int64_t)i * g.plane + nd.nb.node(g, c2(i, 0), c2(i, 1), 0)];
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = mu[i] = 0.f;
        }
        LearnedMoments<float> s;
        float I[kNetIn];
        learned_inputs(f, s, I);
        const Scale sx_sc = stage_inputs(I, tb.shift, tb.scale, sx[warp], lane);
        __syncwarp();
        const float kxt = sx_sc.inv * tb.iw1 * kTwoOverLn2;
        float zc[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            float h[7][4];
            net3_layer1(tb, a_inputs(sx[warp], m, lane), kxt, lane, h);
            net3_layer2(tb, h, lane, zc[m]);
#pragma unroll
            for (int t = 0; t < 7; ++t)
                *reinterpret_cast<float4*>(&sh[warp][m][t][lane][0]) = make_float4(h[t][0], h[t][1], h[t][2], h[t][3]);
        }
        float z[3], ez[3], omg[3];
        net3_outputs(zc, lane, z);
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            const int r = net3_row(o);
            ez[r] = expf(z[o]);
            omg[r] = recip(ez[r] + 0.5f);
        }
        LearnedCot<float> c = learned_adj_head(s, mu, omega);
        c.gg6 = (1.f - omg[0]) * c.q6;
        c.gg7 = (1.f - omg[1]) * c.q7;
        c.gg8 = (1.f - omg[2]) * c.q8;
        const float gomg[3] = {-(c.q6 * s.g6), -(c.q7 * s.g7), -(c.q8 * s.g8)};
        float gz[3];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            const int r = net3_row(o);
            gz[o] = nd.valid ? gomg[r] * (-ez[r] * omg[r] * omg[r]) : 0.f;
        }
        const Scale sgz = warp_scale(fmaxf(fabsf(gz[0]), fmaxf(fabsf(gz[1]), fabsf(gz[2]))));
        {
            const Pair p0 = split(gz[0] * sgz.s, gz[1] * sgz.s), p1 = split(gz[2] * sgz.s, 0.f);
            sz[warp][0][lane][0] = p0.h;
            sz[warp][1][lane][0] = p0.l;
            sz[warp][0][lane][1] = p1.h;
            sz[warp][1][lane][1] = p1.l;
            sz[warp][0][lane][2] = sz[warp][0][lane][3] = 0u;
            sz[warp][1][lane][2] = sz[warp][1][lane][3] = 0u;
        }
        __syncwarp();
        const float kz = sgz.inv * tb.iw2;
#pragma unroll 1
        for (int m = 0; m < 2; ++m) {
            float h[7][4];
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                const float4 v = *reinterpret_cast<const float4*>(&sh[warp][m][t][lane][0]);
                h[t][0] = v.x;
                h[t][1] = v.y;
                h[t][2] = v.z;
                h[t][3] = v.w;
            }
            // back through W2 and tanh: ga = (gz W2) (1 - h^2)
            const AFrag agz = a_inputs(sz[warp], m, lane);
            float ga[7][4];
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                float cc[4] = {0.f, 0.f, 0.f, 0.f};
                mma3(cc, agz, b_load0(&tb.w2b[t][0][0], lane));
#pragma unroll
                for (int e = 0; e < 4; ++e) ga[t][e] = cc[e] * kz * (1.f - h[t][e] * h[t][e]);
            }
            // back through W1: gI of the row tile into sg
            const Scale sga = warp_scale(absmax<7>(ga));
            AFrag ag[4];
#pragma unroll
            for (int st = 0; st < 4; ++st) ag[st] = a_from_c<7>(ga, st, sga.s);
            {
                float cc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int st = 0; st < 4; ++st) mma3(cc, ag[st], b_load(&tb.w1b[st][0][0][0], lane));
                const float k1 = sga.inv * tb.iw1;
                sg[warp][16 * m + gq][2 * q] = cc[0] * k1;
                sg[warp][16 * m + gq][2 * q + 1] = cc[1] * k1;
                sg[warp][16 * m + gq + 8][2 * q] = cc[2] * k1;
                sg[warp][16 * m + gq + 8][2 * q + 1] = cc[3] * k1;
            }
            // dW1: D[m][j] = sum_n [x | 1][n][m] ga[n][j]
            {
                const float kd1 = sga.inv * sx_sc.inv;
                const AFrag ax = a_inputs(sx[warp], m, lane);
                const AFrag au = {{trans(ax.r[0]), kZero, trans(ax.r[1]), kZero}};
#pragma unroll
                for (int t = 0; t < 7; ++t) {
                    const AFrag& a = ag[t >> 1];
                    const BFrag bv = (t & 1) ? BFrag{{trans(a.r[2]), trans(a.r[3])}} : BFrag{{trans(a.r[0]), trans(a.r[1])}};
                    float cw[4] = {0.f, 0.f, 0.f, 0.f};
                    mma3(cw, au, bv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float& a = aW1[32 * (4 * t + e)];
                        a = fmaf(cw[e], kd1, a);
                    }
                }
            }
            // dW2: D[j][o] = sum_n [h | 1][n][j] gz[n][o] (the constant 1 at unit 56)
            {
                const BFrag bz = {{trans(agz.r[0]), trans(agz.r[1])}};
                const Pair one = ones_t(lane);
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) {
                    AFrag au;
                    au.r[0] = trans(split(h[2 * mm][0], h[2 * mm][1]));
                    au.r[2] = trans(split(h[2 * mm][2], h[2 * mm][3]));
                    if (2 * mm + 1 < 7) {
                        au.r[1] = trans(split(h[2 * mm + 1][0], h[2 * mm + 1][1]));
                        au.r[3] = trans(split(h[2 * mm + 1][2], h[2 * mm + 1][3]));
                    } else {
                        au.r[1] = one;
                        au.r[3] = one;
                    }
                    float cw[4] = {0.f, 0.f, 0.f, 0.f};
                    mma3(cw, au, bz);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float& a = aW2[32 * (4 * mm + e)];
                        a = fmaf(cw[e], sgz.inv, a);
                    }
                }
            }
        }
        __syncwarp();
        float gI[kNetIn];
#pragma unroll
        for (int k = 0; k < kNetIn; ++k) gI[k] = sg[warp][lane][k] * tb.scale[k];
        if (nd.valid) learned_adj_tail(s, c, gI, lam_out, g.plane, nd.n);
        __syncwarp();
    }
    __syncthreads();  // red overlays the activations, which every warp has finished with
    constexpr int H = kNet3Hidden;
    constexpr int oW1 = 0, ob1 = H * 6, oW2 = ob1 + H, ob2 = oW2 + 3 * H;
    float* rw = red[warp];
#pragma unroll
    for (int t = 0; t < 7; ++t)
#pragma unroll
        for (int e = 0; e < 2; ++e) {  // rows 8..15 (e >= 2) hold nothing
            const int mrow = gq, j = 8 * t + 2 * q + e;
            if (j < H) {
                const float v = aW1[32 * (4 * t + e)];
                if (mrow < 6) rw[oW1 + j * 6 + mrow] = v;
                else if (mrow == 6) rw[ob1 + j] = v;
            }
        }
#pragma unroll
    for (int mm = 0; mm < 4; ++mm)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 16 * mm + gq + 8 * (e >> 1), o = 2 * q + (e & 1);
            if (o < 3) {
                const float v = aW2[32 * (4 * mm + e)];
                if (j < H) rw[oW2 + o * H + j] = v;
                else if (j == 56) rw[ob2 + o] = v;
            }
        }
    __syncthreads();  // every warp's sums are in red
    float* out = gth_partials + (int64_t)blockIdx.x * kNet3Theta;
    for (int o = threadIdx.x; o < kNet3Theta; o += kThreads)
        out[o] += ((red[0][o] + red[1][o]) + red[2][o]) + red[3][o];
}

// ---------------------------------------------------------------- launch
// Persistent grid: as many blocks as fit on the device at once (from the occupancy of the
// kernel with its dynamic shared memory), at most one per four warp tiles. The same grid for
// every launch on a device keeps the parameter-gradient sums in a fixed order.
template <class K>
int grid_for(K kernel, int sms, int64_t ntiles, size_t smem = 0)
{
    int per_sm = 0;
    if (smem > 0) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t want = (ntiles + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * per_sm;
    return (int)(want < cap ? want : cap);
}

template <class T>
cudaError_t launch_x3(const OpArgs& a, bool three)
{
    const uint32_t* tab = (const uint32_t*)a.x3_table;
    if (!tab) return cudaErrorInvalidValue;
    const int ntx = (a.g.nx + 31) / 32;
    const int64_t ntiles = (int64_t)ntx * a.g.ny;
    const float omega = (float)a.omega;
    if (a.op == OP_UPDATE) {
        const T* src = (const T*)a.src;
        T* dst = (T*)a.dst;
#define LB_X3_FWD(KER, MODE)                                                                                   \
    do {                                                                                                       \
        const int grid = grid_for(KER<T, MODE>, a.sms, ntiles);                                                \
        KER<T, MODE><<<grid, kThreads, 0, a.stream>>>(src, dst, a.g, omega, a.status, tab, ntx, ntiles);       \
    } while (0)
        if (three) {
            if (a.mode == AB) LB_X3_FWD(k_learned3_fwd_x3, AB);
            else if (a.mode == AA_EVEN) LB_X3_FWD(k_learned3_fwd_x3, AA_EVEN);
            else LB_X3_FWD(k_learned3_fwd_x3, AA_ODD);
        } else {
            if (a.mode == AB) LB_X3_FWD(k_learned_fwd_x3, AB);
            else if (a.mode == AA_EVEN) LB_X3_FWD(k_learned_fwd_x3, AA_EVEN);
            else LB_X3_FWD(k_learned_fwd_x3, AA_ODD);
        }
#undef LB_X3_FWD
        return cudaGetLastError();
    }
    if (a.op == OP_ADJ_STEP) {
        const T* st = (const T*)a.src;
        if (three) {
            const int grid = grid_for(k_learned3_adj_x3<T>, a.sms, ntiles, sizeof(Adj3Smem));
            k_learned3_adj_x3<T><<<grid, kThreads, sizeof(Adj3Smem), a.stream>>>(
                st, (const float*)a.lam_in, (float*)a.lam_out, a.g, omega, (float*)a.gth, tab, ntx, ntiles);
        } else {
            const int grid = grid_for(k_learned_adj_x3<T>, a.sms, ntiles, sizeof(Adj1Smem));
            k_learned_adj_x3<T><<<grid, kThreads, sizeof(Adj1Smem), a.stream>>>(
                st, (const float*)a.lam_in, (float*)a.lam_out, a.g, omega, (float*)a.gth, tab, ntx, ntiles);
        }
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

template <class T>
int64_t adj_grid(const Geom& g, int sms, bool three)
{
    const int64_t ntiles = (int64_t)((g.nx + 31) / 32) * g.ny;
    return three ? grid_for(k_learned3_adj_x3<T>, sms, ntiles, sizeof(Adj3Smem))
                 : grid_for(k_learned_adj_x3<T>, sms, ntiles, sizeof(Adj1Smem));
}

}  // namespace

size_t learned_x3_table_bytes(bool three) { return three ? sizeof(Tab3) : sizeof(Tab1); }

void learned_x3_pack(const double* net, bool three, void* out)
{
    if (three) {
        Tab3 t;
        pack3(net, t);
        std::memcpy(out, &t, sizeof(t));
    } else {
        Tab1 t;
        pack1(net, t);
        std::memcpy(out, &t, sizeof(t));
    }
}

cudaError_t run_learned_x3(const OpArgs& a, bool three)
{
    if (a.g.nz != 1) return cudaErrorInvalidValue;
    switch (a.storage) {
    case S_F32: return launch_x3<float>(a, three);
    case S_F16: return launch_x3<__half>(a, three);
    case S_BF16: return launch_x3<__nv_bfloat16>(a, three);
    default: return cudaErrorInvalidValue;
    }
}

int64_t learned_x3_partial_count(const Geom& g, int storage, int sms, bool three)
{
    switch (storage) {
    case S_F32: return adj_grid<float>(g, sms, three);
    case S_F16: return adj_grid<__half>(g, sms, three);
    case S_BF16: return adj_grid<__nv_bfloat16>(g, sms, three);
    default: return 0;
    }
}

}  // namespace lb
