// Device-side building blocks of liblb: velocity sets, storage conversion, and
// the per-node load/store patterns of the two-buffer (AB) and in-place (AA)
// layouts. Everything here is header-only and force-inlined into the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#define LB_DEV __device__ __forceinline__
#define LB_HD __host__ __device__ __forceinline__

namespace lb {

// ----------------------------------------------------------------------------
// Velocity sets (Sec. 2.2, 3.1, 3.3 name D2Q9, D3Q19, D3Q27; the tables are the
// textbook ones). Order: rest, +/- axis pairs, +/- edge pairs (xy, xz, yz), +/-
// corner pairs. D3Q19 is the first 19 entries of the D3Q27 table.
// ----------------------------------------------------------------------------
LB_HD constexpr int c3(int i, int a)
{
    constexpr int t[27][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
        {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
        {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    return t[i][a];
}

LB_HD constexpr int c2(int i, int a)
{
    constexpr int t[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
    return a < 2 ? t[i][a] : 0;
}

struct D2Q9 {
    static constexpr int Q = 9, D = 2, ID = 0;
    LB_HD static constexpr int c(int i, int a) { return c2(i, a); }
    LB_HD static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};
struct D3Q19 {
    static constexpr int Q = 19, D = 3, ID = 1;
    LB_HD static constexpr int c(int i, int a) { return c3(i, a); }
    LB_HD static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};
struct D3Q27 {
    static constexpr int Q = 27, D = 3, ID = 2;
    LB_HD static constexpr int c(int i, int a) { return c3(i, a); }
    LB_HD static constexpr double w(int i)
    {
        return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
};

// opposite direction: pairs are stored next to each other after the rest velocity
LB_HD constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// ----------------------------------------------------------------------------
// Storage types. Real is the arithmetic type (FP64 only for FP64 storage).
// FP32 and the half types hold f_i - w_i ("shifted"): near rest the deviation is 10 to 40
// times smaller than f_i, so its rounding in storage is that much smaller too (for FP32
// this is the difference between about 3e-8 and 1e-9 absolute per population and step,
// which the non-equilibrium parts of f, often 1e-4 of it, feel directly). FP64 holds f_i.
// ----------------------------------------------------------------------------
template <class T> struct Store;
template <> struct Store<double> {
    using Real = double;
    static constexpr bool shifted = false;
    static constexpr bool half = false;
    LB_DEV static double load(const double* p) { return *p; }
    LB_DEV static void store(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
    using Real = float;
    static constexpr bool shifted = true;
    static constexpr bool half = false;
    LB_DEV static float load(const float* p) { return *p; }
    LB_DEV static void store(float* p, float v) { *p = v; }
};
template <> struct Store<__half> {
    using Real = float;
    static constexpr bool shifted = true;
    static constexpr bool half = true;
    LB_DEV static float load(const __half* p) { return __half2float(*p); }
    LB_DEV static void store(__half* p, float v) { *p = __float2half_rn(v); }
    LB_DEV static void store(__half* p, double v) { *p = __double2half(v); }
};
template <> struct Store<__nv_bfloat16> {
    using Real = float;
    static constexpr bool shifted = true;
    static constexpr bool half = true;
    LB_DEV static float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    LB_DEV static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    LB_DEV static void store(__nv_bfloat16* p, double v) { *p = __double2bfloat16(v); }
};

// Collision arithmetic works on deviations from rest, delta_i = f_i - w_i: the
// moment sums then add small numbers (rho - 1 = sum delta, j = sum c delta) and
// FP32 keeps its relative precision. Unshifted (FP64) storage converts on load/store;
// shifted storage holds delta itself.
template <class St, class T>
LB_DEV typename Store<T>::Real load_pop(const T* p, int i)
{
    using R = typename Store<T>::Real;
    R v = Store<T>::load(p);
    if constexpr (!Store<T>::shifted) v -= R(St::w(i));
    return v;
}

template <class St, class T>
LB_DEV void store_pop(T* p, int i, typename Store<T>::Real delta)
{
    using R = typename Store<T>::Real;
    if constexpr (!Store<T>::shifted) delta += R(St::w(i));
    Store<T>::store(p, delta);
}

// the stored value itself, unconverted (streaming without collision moves it as is)
template <class St, class T>
LB_DEV typename Store<T>::Real load_raw(const T* p, int)
{
    return Store<T>::load(p);
}
template <class St, class T>
LB_DEV void store_raw(T* p, int, typename Store<T>::Real v)
{
    Store<T>::store(p, v);
}

// FP64 value of the population f_i (for copies out of the library)
template <class St, class T>
LB_DEV double load_f64(const T* p, int i)
{
    double v = (double)Store<T>::load(p);
    if constexpr (Store<T>::shifted) v += St::w(i);
    return v;
}
// store f_i given in FP64 (the shift, if any, is taken in FP64 before rounding)
template <class St, class T>
LB_DEV void store_f64(T* p, int i, double f)
{
    using R = typename Store<T>::Real;
    if constexpr (Store<T>::shifted) f -= St::w(i);
    if constexpr (Store<T>::shifted || sizeof(R) == 8) Store<T>::store(p, f);
    else Store<T>::store(p, (float)f);
}

// Two x-adjacent values (nodes x0 and x0 + 1, x0 even) as one aligned vector access.
template <class T> struct Pair2;
template <> struct Pair2<double> {
    LB_DEV static void load(const double* p, double& a, double& b) { double2 v = *(const double2*)p; a = v.x; b = v.y; }
    LB_DEV static void store(double* p, double a, double b) { *(double2*)p = make_double2(a, b); }
};
template <> struct Pair2<float> {
    LB_DEV static void load(const float* p, float& a, float& b) { float2 v = *(const float2*)p; a = v.x; b = v.y; }
    LB_DEV static void store(float* p, float a, float b) { *(float2*)p = make_float2(a, b); }
};
template <> struct Pair2<__half> {
    LB_DEV static void load(const __half* p, float& a, float& b)
    {
        const float2 v = __half22float2(*(const __half2*)p);
        a = v.x;
        b = v.y;
    }
    LB_DEV static void store(__half* p, float a, float b) { *(__half2*)p = __floats2half2_rn(a, b); }
};
template <> struct Pair2<__nv_bfloat16> {
    LB_DEV static void load(const __nv_bfloat16* p, float& a, float& b)
    {
        const float2 v = __bfloat1622float2(*(const __nv_bfloat162*)p);
        a = v.x;
        b = v.y;
    }
    LB_DEV static void store(__nv_bfloat16* p, float a, float b) { *(__nv_bfloat162*)p = __floats2bfloat162_rn(a, b); }
};

// Four x-adjacent half-precision values (x0 % 4 == 0) as one aligned 8-byte access.
template <class T> struct Quad4;
template <> struct Quad4<__half> {
    LB_DEV static void load(const __half* p, float* v)
    {
        const uint2 r = *(const uint2*)p;
        const float2 a = __half22float2(*(const __half2*)&r.x), b = __half22float2(*(const __half2*)&r.y);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    LB_DEV static void store(__half* p, const float* v)
    {
        const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 r;
        r.x = *(const unsigned*)&a;
        r.y = *(const unsigned*)&b;
        *(uint2*)p = r;
    }
};
template <> struct Quad4<__nv_bfloat16> {
    LB_DEV static void load(const __nv_bfloat16* p, float* v)
    {
        const uint2 r = *(const uint2*)p;
        const float2 a = __bfloat1622float2(*(const __nv_bfloat162*)&r.x);
        const float2 b = __bfloat1622float2(*(const __nv_bfloat162*)&r.y);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    LB_DEV static void store(__nv_bfloat16* p, const float* v)
    {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 r;
        r.x = *(const unsigned*)&a;
        r.y = *(const unsigned*)&b;
        *(uint2*)p = r;
    }
};

// deviations of two adjacent nodes from one vector load / into one vector store
template <class St, class T>
LB_DEV void load_pop2(const T* p, int i, typename Store<T>::Real& a, typename Store<T>::Real& b)
{
    using R = typename Store<T>::Real;
    Pair2<T>::load(p, a, b);
    if constexpr (!Store<T>::shifted) {
        a -= R(St::w(i));
        b -= R(St::w(i));
    }
}
template <class St, class T>
LB_DEV void store_pop2(T* p, int i, typename Store<T>::Real a, typename Store<T>::Real b)
{
    using R = typename Store<T>::Real;
    if constexpr (!Store<T>::shifted) {
        a += R(St::w(i));
        b += R(St::w(i));
    }
    Pair2<T>::store(p, a, b);
}

// ----------------------------------------------------------------------------
// Grid geometry and periodic neighbours of one node.
// ----------------------------------------------------------------------------
struct Geom {
    int nx, ny, nz;
    int64_t plane;  // element stride between population planes (>= N, padded)
    // solid nodes (halfway bounce-back): links[n] bit i (1 <= i < Q) set when x - c_i is
    // solid, bit 31 when n itself is; nullptr = no walls. wall_u: [D][plane] velocity of
    // each solid node in the arithmetic type, or nullptr (resting walls).
    const unsigned* links = nullptr;
    const void* wall_u = nullptr;
};
constexpr unsigned kSolidBit = 1u << 31;

// the exposed state of a solid node is the rest equilibrium f_i = w_i
LB_DEV bool solid_node(const Geom& g, int n) { return g.links && (g.links[n] & kSolidBit); }

// Node coordinates and the wrapped +/-1 neighbours along each axis, plus the byte
// offsets of the populations around the node for an element size S: per thread the
// three x positions, per block (uniform: y, z come from blockIdx) the nine rows.
// A population access is then base + slot * plane_bytes + row + x: one add per load
// instead of index arithmetic per direction.
struct Nbr {
    int x[3], y[3], z[3];  // index 0: coordinate - 1, 1: coordinate, 2: coordinate + 1 (wrapped)
    int64_t xo[3];         // x[k] * S
    int64_t ro[3][3];      // (y[dy] + ny z[dz]) nx S
    int64_t pb;            // plane * S
    LB_DEV int node(const Geom& g, int dx, int dy, int dz) const
    {
        return x[dx + 1] + g.nx * (y[dy + 1] + g.ny * z[dz + 1]);
    }
    LB_DEV int64_t boff(int slot, int dx, int dy, int dz) const
    {
        return slot * pb + ro[dy + 1][dz + 1] + xo[dx + 1];
    }
};

template <int S = 4>
LB_DEV Nbr make_nbr(const Geom& g, int x, int y, int z)
{
    Nbr n;
    n.x[0] = x == 0 ? g.nx - 1 : x - 1; n.x[1] = x; n.x[2] = x == g.nx - 1 ? 0 : x + 1;
    n.y[0] = y == 0 ? g.ny - 1 : y - 1; n.y[1] = y; n.y[2] = y == g.ny - 1 ? 0 : y + 1;
    n.z[0] = z == 0 ? g.nz - 1 : z - 1; n.z[1] = z; n.z[2] = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) n.xo[k] = (int64_t)n.x[k] * S;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) n.ro[a][b] = ((int64_t)n.y[a] + (int64_t)g.ny * n.z[b]) * g.nx * S;
    n.pb = g.plane * S;
    return n;
}

// the same for a 2D grid (nz == 1): the three rows only
template <int S = 4>
LB_DEV Nbr make_nbr_2d(const Geom& g, int x, int y)
{
    Nbr n;
    n.x[0] = x == 0 ? g.nx - 1 : x - 1; n.x[1] = x; n.x[2] = x == g.nx - 1 ? 0 : x + 1;
    n.y[0] = y == 0 ? g.ny - 1 : y - 1; n.y[1] = y; n.y[2] = y == g.ny - 1 ? 0 : y + 1;
    n.z[0] = n.z[1] = n.z[2] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) n.xo[k] = (int64_t)n.x[k] * S;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t r = (int64_t)n.y[a] * g.nx * S;
        n.ro[a][0] = n.ro[a][1] = n.ro[a][2] = r;
    }
    n.pb = g.plane * S;
    return n;
}

template <class T>
LB_DEV const T* at(const T* buf, const Nbr& nb, int slot, int dx, int dy, int dz)
{
    return (const T*)((const char*)buf + nb.boff(slot, dx, dy, dz));
}
template <class T>
LB_DEV T* at(T* buf, const Nbr& nb, int slot, int dx, int dy, int dz)
{
    return (T*)((char*)buf + nb.boff(slot, dx, dy, dz));
}

// ----------------------------------------------------------------------------
// Access modes. The buffer content per mode, for the pre-collision state f^n:
//   AB      : buf_i(x) = f*_i(x) of the previous step, so f^n_i(x) = buf_i(x - c_i)
//             (pull). The next state is written unshifted: out_i(x) = f*_i(x).
//   AA_EVEN : buf_i(x) = f^n_i(x) (natural). Collide writes f*_i(x) into slot opp(i)
//             of the same node.
//   AA_ODD  : slot opp(i) of x holds f*_i(x) of the previous step, so
//             f^n_i(x) = buf_opp(i)(x - c_i). Collide writes f*_i(x) to slot i of
//             x + c_i, which is the natural layout of the next state.
// ----------------------------------------------------------------------------
enum Mode { AB = 0, AA_EVEN = 1, AA_ODD = 2 };

template <class St, int MODE, bool RAW = false, class T>
LB_DEV void load_node(const T* buf, const Geom& g, const Nbr& nb, int n, typename Store<T>::Real* f)
{
    using R = typename Store<T>::Real;
    if (solid_node(g, n)) {
#pragma unroll
        for (int i = 0; i < St::Q; ++i) f[i] = (RAW && !Store<T>::shifted) ? R(St::w(i)) : R(0);
        return;
    }
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int s = (MODE == AA_EVEN) ? 0 : -1;
        const T* p = at(buf, nb, slot, s * St::c(i, 0), s * St::c(i, 1), s * St::c(i, 2));
        if constexpr (RAW) f[i] = load_raw<St>(p, slot);
        else f[i] = load_pop<St>(p, slot);
    }
}

template <class St, int MODE, bool RAW = false, class T>
LB_DEV void store_node(T* buf, const Geom& g, const Nbr& nb, int n, const typename Store<T>::Real* f)
{
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_EVEN) ? opp(i) : i;
        const int s = (MODE == AA_ODD) ? 1 : 0;
        T* p = at(buf, nb, slot, s * St::c(i, 0), s * St::c(i, 1), s * St::c(i, 2));
        if constexpr (RAW) store_raw<St>(p, slot, f[i]);
        else store_pop<St>(p, slot, f[i]);
    }
}

// FP64 populations of one node's pre-collision state (copies out of the library)
template <class St, int MODE, class T>
LB_DEV void load_node_f64(const T* buf, const Geom& g, const Nbr& nb, int n, double* f)
{
    if (solid_node(g, n)) {
#pragma unroll
        for (int i = 0; i < St::Q; ++i) f[i] = St::w(i);
        return;
    }
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int s = (MODE == AA_EVEN) ? 0 : -1;
        f[i] = load_f64<St>(at(buf, nb, slot, s * St::c(i, 0), s * St::c(i, 1), s * St::c(i, 2)), slot);
    }
}

}  // namespace lb
