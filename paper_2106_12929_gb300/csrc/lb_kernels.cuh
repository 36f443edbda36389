// Node kernels of liblb, templated on the velocity set and instantiated once per
// set in fwd_<stencil>.cu. One thread owns one node; blocks tile x-rows; each
// population plane is contiguous (structure of arrays, x fastest), so every
// load and store of a warp touches 32 consecutive elements of one plane.
#pragma once

#include "lb_adjoint.cuh"
#include "lb_collide.cuh"
#include "lb_ops.cuh"

namespace lb {

template <class O> LB_DEV O to_io(double v) { return (O)v; }

LB_DEV double io_load(const void* p, int f64, int64_t k)
{
    return f64 ? ((const double*)p)[k] : (double)((const float*)p)[k];
}
LB_DEV void io_store(void* p, int f64, int64_t k, double v)
{
    if (f64) ((double*)p)[k] = v;
    else ((float*)p)[k] = (float)v;
}
LB_DEV void io_add(void* p, int f64, int64_t k, double v)
{
    if (f64) ((double*)p)[k] += v;
    else ((float*)p)[k] += (float)v;
}

struct NodeIdx {
    int x, y, z, n;
    bool valid;
};

LB_DEV NodeIdx node_index(const Geom& g)
{
    NodeIdx r;
    r.x = blockIdx.x * blockDim.x + threadIdx.x;
    r.y = blockIdx.y;
    r.z = blockIdx.z;
    r.valid = r.x < g.nx;
    r.n = r.x + g.nx * (r.y + g.ny * r.z);
    return r;
}

template <class St, class R>
LB_DEV void load_force(const R* F, const Geom& g, int n, R* Fl)
{
    Fl[0] = F[n];
    Fl[1] = F[g.plane + n];
    Fl[2] = St::D == 3 ? F[2 * g.plane + n] : R(0);
}

// Halfway bounce-back writes of one fluid node with link word lk (AB layout): for every solid
// neighbour x - c_i the next step pulls f_i(x) from slot i of that solid node, which receives
// f*_opp(i)(x) + 2 w_i (c_i . u_wall) / c_s^2 (moving-wall term; wall density 1). Solid slots
// are written by these reflections only (a solid node stores nothing itself), and each
// (solid node, slot) pair has exactly one fluid source, so the writes never collide.
template <class St, bool RAW, class T>
LB_DEV void bounce_back(T* dst, const Geom& g, const Nbr& nb, unsigned lk, const typename Store<T>::Real* f)
{
    using R = typename Store<T>::Real;
    const R* Wu = (const R*)g.wall_u;
#pragma unroll
    for (int i = 1; i < St::Q; ++i) {
        if (!((lk >> i) & 1u)) continue;
        const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
        R v = f[opp(i)];
        if (Wu) {
            const int m = nb.node(g, -cx, -cy, -cz);
            R cu = R(0);
            if (cx) cu += cx > 0 ? Wu[m] : -Wu[m];
            if (cy) cu += cy > 0 ? Wu[g.plane + m] : -Wu[g.plane + m];
            if (St::D == 3 && cz) cu += cz > 0 ? Wu[2 * g.plane + m] : -Wu[2 * g.plane + m];
            v += R(6.0 * St::w(i)) * cu;
        }
        T* p = at(dst, nb, i, -cx, -cy, -cz);
        if constexpr (RAW) store_raw<St>(p, i, v);
        else store_pop<St>(p, i, v);
    }
}

// ------------------------------------------------------------------ step (K1/K2)
template <class St, class T, int COLL, bool FORCE, int MODE>
__global__ void __launch_bounds__(128) k_update(const T* src, T* dst, const typename Store<T>::Real* F, Geom g,
                                                Relax<typename Store<T>::Real> rx, unsigned* status)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    // halfway bounce-back (AB only): a solid node is skipped; its slots are written by
    // the fluid nodes whose populations reflect off it
    const unsigned lk = g.links ? g.links[id.n] : 0u;
    if (lk & kSolidBit) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    R f[St::Q];
    constexpr bool RAW = COLL == NONE;  // streaming only: move the stored values untouched
    load_node<St, MODE, RAW>(src, g, nb, id.n, f);
    R Fl[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
    bool ok = collide<St, COLL, FORCE>(f, Fl, rx);
    store_node<St, MODE, RAW>(dst, g, nb, id.n, f);
    if (MODE == AB && lk) bounce_back<St, RAW>(dst, g, nb, lk, f);
    if (!ok) atomicOr(status, 1u);
}

// links[n] of every node from a solid mask (uint8, nonzero = solid)
template <class St>
__global__ void k_build_links(const unsigned char* mask, Geom g, unsigned* links)
{
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<1>(g, id.x, id.y, id.z);
    unsigned lk = mask[id.n] ? kSolidBit : 0u;
#pragma unroll
    for (int i = 1; i < St::Q; ++i)
        if (mask[nb.node(g, -St::c(i, 0), -St::c(i, 1), -St::c(i, 2))]) lk |= 1u << i;
    links[id.n] = lk;
}

// Two nodes per thread (x0 = 2 t and x0 + 1; nx even). An access whose x shift is 0
// serves both nodes with one aligned vector load or store; a shift of -1 or +1 takes
// two scalar accesses, the inner one at a fixed byte distance from the vector
// address. Every AB store and every non-x-moving load is a vector access, which
// halves the memory instructions and conversions per node.
template <class St, class T, int COLL, bool FORCE, int MODE, bool WALLS = false>
__global__ void __launch_bounds__(128) k_update_pair(const T* src, T* dst, const typename Store<T>::Real* F, Geom g,
                                                     Relax<typename Store<T>::Real> rx, unsigned* status)
{
    using R = typename Store<T>::Real;
    constexpr int S = sizeof(T);
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    // walls (AB only): link words of both nodes (n0 is even: nx is even for this kernel)
    unsigned lk0 = 0u, lk1 = 0u;
    if constexpr (WALLS) {
        const uint2 l = *(const uint2*)(g.links + (x0 + (int64_t)g.nx * (y + (int64_t)g.ny * z)));
        lk0 = l.x;
        lk1 = l.y;
        if (lk0 & lk1 & kSolidBit) return;
    }
    const bool sol0 = WALLS && (lk0 & kSolidBit), sol1 = WALLS && (lk1 & kSolidBit);
    const int yy[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
    const int zz[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
    const int64_t xo_m = (int64_t)(x0 == 0 ? g.nx - 1 : x0 - 1) * S;       // x0 - 1
    const int64_t xo_0 = (int64_t)x0 * S;                                    // x0 (x0 + 1 = xo_0 + S)
    const int64_t xo_2 = (int64_t)(x0 + 2 == g.nx ? 0 : x0 + 2) * S;        // x0 + 2
    const int64_t pb = g.plane * S;
    auto row = [&](int dy, int dz) -> int64_t {
        return ((int64_t)yy[dy + 1] + (int64_t)g.ny * zz[dz + 1]) * g.nx * S;
    };
    R f0[St::Q], f1[St::Q];
    constexpr int ls = (MODE == AA_EVEN) ? 0 : -1;  // load shift along c_i
    constexpr int ss = (MODE == AA_ODD) ? 1 : 0;    // store shift along c_i
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int sx = ls * St::c(i, 0);
        const char* base = (const char*)src + slot * pb + row(ls * St::c(i, 1), ls * St::c(i, 2));
        if (sx == 0) {
            load_pop2<St>((const T*)(base + xo_0), slot, f0[i], f1[i]);
        } else if (sx < 0) {
            f0[i] = load_pop<St>((const T*)(base + xo_m), slot);
            f1[i] = load_pop<St>((const T*)(base + xo_0), slot);
        } else {
            f0[i] = load_pop<St>((const T*)(base + xo_0 + S), slot);
            f1[i] = load_pop<St>((const T*)(base + xo_2), slot);
        }
    }
    R F0[3] = {R(0), R(0), R(0)}, F1[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) {
        const int n0 = x0 + g.nx * (y + g.ny * z);
        Pair2<R>::load(F + n0, F0[0], F1[0]);
        Pair2<R>::load(F + g.plane + n0, F0[1], F1[1]);
        if (St::D == 3) Pair2<R>::load(F + 2 * g.plane + n0, F0[2], F1[2]);
    }
    const bool ok0 = collide<St, COLL, FORCE>(f0, F0, rx) || sol0;  // a solid node's result is dropped
    const bool ok1 = collide<St, COLL, FORCE>(f1, F1, rx) || sol1;
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_EVEN) ? opp(i) : i;
        const int sx = ss * St::c(i, 0);
        char* base = (char*)dst + slot * pb + row(ss * St::c(i, 1), ss * St::c(i, 2));
        if (sx == 0) {
            if (WALLS && (sol0 || sol1)) {  // a solid node's slots belong to the reflections
                if (!sol0) store_pop<St>((T*)(base + xo_0), slot, f0[i]);
                if (!sol1) store_pop<St>((T*)(base + xo_0 + S), slot, f1[i]);
            } else {
                store_pop2<St>((T*)(base + xo_0), slot, f0[i], f1[i]);
            }
        } else if (sx < 0) {
            store_pop<St>((T*)(base + xo_m), slot, f0[i]);
            store_pop<St>((T*)(base + xo_0), slot, f1[i]);
        } else {
            store_pop<St>((T*)(base + xo_0 + S), slot, f0[i]);
            store_pop<St>((T*)(base + xo_2), slot, f1[i]);
        }
    }
    if constexpr (WALLS) {
        if (lk0 && !sol0) bounce_back<St, false>(dst, g, make_nbr<S>(g, x0, y, z), lk0, f0);
        if (lk1 && !sol1) bounce_back<St, false>(dst, g, make_nbr<S>(g, x0 + 1, y, z), lk1, f1);
    }
    if (!(ok0 && ok1)) atomicOr(status, 1u);
}

// Four nodes per thread for the half-precision (shifted) storage types (x0 = 4 t, nx % 4 == 0).
// Half storage moves half the bytes of FP32 with the same instruction count per node, so it
// runs out of issue slots before HBM bandwidth; four nodes per 8-byte access cut the memory
// instructions and conversions per node again. An access with x shift 0 is one vector for all
// four nodes; a load shifted by -1 or +1 takes the vector at x0 (three of its values) plus
// one scalar; a shifted store is four scalar stores.
template <class St, class T, int COLL, bool FORCE, int MODE, bool WALLS = false>
__global__ void __launch_bounds__(128) k_update_quad(const T* src, T* dst, const float* F, Geom g, Relax<float> rx,
                                                     unsigned* status)
{
    static_assert(Store<T>::half, "four-node kernel is for half-precision storage");
    constexpr int S = sizeof(T);
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    // walls (AB only): link words of the four nodes (n0 % 4 == 0: nx % 4 == 0 here)
    unsigned lk[4] = {0u, 0u, 0u, 0u};
    bool sol[4] = {false, false, false, false};
    if constexpr (WALLS) {
        const uint4 l = *(const uint4*)(g.links + (x0 + (int64_t)g.nx * (y + (int64_t)g.ny * z)));
        lk[0] = l.x; lk[1] = l.y; lk[2] = l.z; lk[3] = l.w;
        if (lk[0] & lk[1] & lk[2] & lk[3] & kSolidBit) return;
#pragma unroll
        for (int k = 0; k < 4; ++k) sol[k] = (lk[k] & kSolidBit) != 0u;
    }
    const bool any_solid = WALLS && (sol[0] || sol[1] || sol[2] || sol[3]);
    const int yy[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
    const int zz[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
    const int64_t xo_m = (int64_t)(x0 == 0 ? g.nx - 1 : x0 - 1) * S;  // x0 - 1
    const int64_t xo_0 = (int64_t)x0 * S;                              // x0 .. x0 + 3
    const int64_t xo_4 = (int64_t)(x0 + 4 == g.nx ? 0 : x0 + 4) * S;  // x0 + 4
    const int64_t pb = g.plane * S;
    auto row = [&](int dy, int dz) -> int64_t {
        return ((int64_t)yy[dy + 1] + (int64_t)g.ny * zz[dz + 1]) * g.nx * S;
    };
    float f[4][St::Q];
    constexpr int ls = (MODE == AA_EVEN) ? 0 : -1;
    constexpr int ss = (MODE == AA_ODD) ? 1 : 0;
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_ODD) ? opp(i) : i;
        const int sx = ls * St::c(i, 0);
        const char* base = (const char*)src + slot * pb + row(ls * St::c(i, 1), ls * St::c(i, 2));
        float v[4];
        Quad4<T>::load((const T*)(base + xo_0), v);
        if (sx == 0) {
            f[0][i] = v[0]; f[1][i] = v[1]; f[2][i] = v[2]; f[3][i] = v[3];
        } else if (sx < 0) {
            f[0][i] = Store<T>::load((const T*)(base + xo_m));
            f[1][i] = v[0]; f[2][i] = v[1]; f[3][i] = v[2];
        } else {
            f[0][i] = v[1]; f[1][i] = v[2]; f[2][i] = v[3];
            f[3][i] = Store<T>::load((const T*)(base + xo_4));
        }
    }
    float Fl[4][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    if constexpr (FORCE) {
        const int64_t n0 = x0 + (int64_t)g.nx * (y + (int64_t)g.ny * z);
#pragma unroll
        for (int a = 0; a < St::D; ++a) {
            const float4 q = *(const float4*)(F + a * g.plane + n0);
            Fl[0][a] = q.x; Fl[1][a] = q.y; Fl[2][a] = q.z; Fl[3][a] = q.w;
        }
    }
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) ok = (collide<St, COLL, FORCE>(f[k], Fl[k], rx) || sol[k]) && ok;
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int slot = (MODE == AA_EVEN) ? opp(i) : i;
        const int sx = ss * St::c(i, 0);
        char* base = (char*)dst + slot * pb + row(ss * St::c(i, 1), ss * St::c(i, 2));
        if (sx == 0) {
            if (any_solid) {  // a solid node's slots belong to the reflections
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (!sol[k]) Store<T>::store((T*)(base + xo_0 + k * S), f[k][i]);
            } else {
                const float v[4] = {f[0][i], f[1][i], f[2][i], f[3][i]};
                Quad4<T>::store((T*)(base + xo_0), v);
            }
        } else if (sx < 0) {
            Store<T>::store((T*)(base + xo_m), f[0][i]);
            Store<T>::store((T*)(base + xo_0), f[1][i]);
            Store<T>::store((T*)(base + xo_0 + S), f[2][i]);
            Store<T>::store((T*)(base + xo_0 + 2 * S), f[3][i]);
        } else {
            Store<T>::store((T*)(base + xo_0 + S), f[0][i]);
            Store<T>::store((T*)(base + xo_0 + 2 * S), f[1][i]);
            Store<T>::store((T*)(base + xo_0 + 3 * S), f[2][i]);
            Store<T>::store((T*)(base + xo_4), f[3][i]);
        }
    }
    if constexpr (WALLS) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (lk[k] && !sol[k]) bounce_back<St, false>(dst, g, make_nbr<S>(g, x0 + k, y, z), lk[k], f[k]);
    }
    if (!ok) atomicOr(status, 1u);
}

// Write a natural-layout state value set into the buffer for the given mode:
// AB keeps f*_i(x) at x (the next pull reads it from x + c_i), so the state
// f_i(x) goes to x - c_i; AA (even parity) stores it in place. Values are
// deviations delta_i (store_state) or FP64 populations f_i (store_state_f64).
template <class St, int MODE>
LB_DEV int state_slot_node(const Geom& g, const Nbr& nb, int n, int i)
{
    if constexpr (MODE == AB) return nb.node(g, -St::c(i, 0), -St::c(i, 1), -St::c(i, 2));
    return n;
}

template <class St, int MODE, class T>
LB_DEV void store_state(T* buf, const Geom& g, const Nbr& nb, int n, const typename Store<T>::Real* d)
{
#pragma unroll
    for (int i = 0; i < St::Q; ++i)
        store_pop<St>(buf + (int64_t)i * g.plane + state_slot_node<St, MODE>(g, nb, n, i), i, d[i]);
}

template <class St, int MODE, class T>
LB_DEV void store_state_f64(T* buf, const Geom& g, const Nbr& nb, int n, const double* f)
{
#pragma unroll
    for (int i = 0; i < St::Q; ++i)
        store_f64<St>(buf + (int64_t)i * g.plane + state_slot_node<St, MODE>(g, nb, n, i), i, f[i]);
}

// ------------------------------------------------------------------ init (K5)
template <class St, class T, int MODE>
__global__ void __launch_bounds__(128) k_init_eq(T* buf, Geom g, const void* rho, const void* u, int f64)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    NodeMoments<St, R> m;
    const double r = io_load(rho, f64, id.n);
    m.rho = (R)r;
    m.rho1 = (R)(r - 1.0);
    m.ux = (R)io_load(u, f64, id.n);
    m.uy = (R)io_load(u, f64, N + id.n);
    m.uz = St::D == 3 ? (R)io_load(u, f64, 2 * N + id.n) : R(0);
    R f[St::Q];
    equilibrium<St>(m, f);
    store_state<St, MODE>(buf, g, nb, id.n, f);
}

// ------------------------------------------------------------------ set / get (K11)
template <class St, class T, int MODE>
__global__ void __launch_bounds__(128) k_set(T* buf, Geom g, const void* fin, int f64)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    double f[St::Q];
#pragma unroll
    for (int i = 0; i < St::Q; ++i) f[i] = io_load(fin, f64, (int64_t)i * N + id.n);
    store_state_f64<St, MODE>(buf, g, nb, id.n, f);
}

template <class St, class T, int MODE>
__global__ void __launch_bounds__(128) k_get(const T* buf, Geom g, void* fout, int f64)
{
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    double f[St::Q];
    load_node_f64<St, MODE>(buf, g, nb, id.n, f);
#pragma unroll
    for (int i = 0; i < St::Q; ++i) io_store(fout, f64, (int64_t)i * N + id.n, f[i]);
}

// ------------------------------------------------------------------ moments (K3)
template <class St, class T, int MODE, bool FORCE>
__global__ void __launch_bounds__(128) k_moments(const T* buf, const typename Store<T>::Real* F, Geom g,
                                                 void* rho, void* u, int f64)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    R f[St::Q];
    load_node<St, MODE>(buf, g, nb, id.n, f);
    R Fl[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
    NodeMoments<St, R> m = node_moments<St, FORCE>(f, Fl);
    if (rho) io_store(rho, f64, id.n, (double)m.rho);
    if (u) {
        io_store(u, f64, id.n, (double)m.ux);
        io_store(u, f64, N + id.n, (double)m.uy);
        if (St::D == 3) io_store(u, f64, 2 * N + id.n, (double)m.uz);
    }
}

// ------------------------------------------------------------------ global sums (K4, pass 1)
// Each block writes the FP64 sums of its nodes in a fixed tree order; pass 2
// (reduce_final) adds the block partials in block order, so results are
// deterministic for a given grid.
template <int W>
LB_DEV void block_sum_store(double (&v)[W], double* out)
{
    __shared__ double sh[W][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < W; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[k][w];
            out[k] = s;
        }
    }
}

template <class St, class T, int MODE, bool FORCE>
__global__ void __launch_bounds__(128) k_reduce_partial(const T* buf, const typename Store<T>::Real* F, Geom g,
                                                        double* partials)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (id.valid) {
        Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
        R f[St::Q];
        load_node<St, MODE>(buf, g, nb, id.n, f);
        R Fl[3] = {R(0), R(0), R(0)};
        if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
        NodeMoments<St, R> m = node_moments<St, FORCE>(f, Fl);
        const double r = m.rho, ux = m.ux, uy = m.uy, uz = m.uz;
        const double uu = ux * ux + uy * uy + uz * uz;
        v[0] = r;
        v[1] = r * ux;
        v[2] = r * uy;
        v[3] = r * uz;
        v[4] = uu;
        v[5] = r * uu;
    }
    const int64_t b = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_sum_store<6>(v, partials + 6 * b);
}

// ------------------------------------------------------------------ adjoint seeds (K7)
template <class St, class T, int MODE, bool FORCE>
__global__ void __launch_bounds__(128) k_adj_seed(const T* buf, const typename Store<T>::Real* F, Geom g,
                                                  const void* grho, const void* gu, void* lam, void* gF, int f64)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    R f[St::Q];
    load_node<St, MODE>(buf, g, nb, id.n, f);
    R Fl[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
    NodeMoments<St, R> m = node_moments<St, FORCE>(f, Fl);
    const R gr = grho ? (R)io_load(grho, f64, id.n) : R(0);
    const R gx = (R)io_load(gu, f64, id.n), gy = (R)io_load(gu, f64, N + id.n);
    const R gz = St::D == 3 ? (R)io_load(gu, f64, 2 * N + id.n) : R(0);
    const R inv = R(1) / m.rho;
    const R gdotu = gx * m.ux + gy * m.uy + gz * m.uz;
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        // dL/df_i = dL/drho + dL/du . (c_i - u) / rho
        R v = gr + (cdotu<St>(i, gx, gy, gz) - gdotu) * inv;
        io_store(lam, f64, (int64_t)i * N + id.n, (double)v);
    }
    if (FORCE && gF) {
        io_add(gF, f64, id.n, (double)(R(0.5) * gx * inv));
        io_add(gF, f64, N + id.n, (double)(R(0.5) * gy * inv));
        if (St::D == 3) io_add(gF, f64, 2 * N + id.n, (double)(R(0.5) * gz * inv));
    }
}

// energy-field loss L = sum (rho |u|^2 / 2 - e*)^2: seed and per-block partial sums of L
template <class St, class T, int MODE, bool FORCE>
__global__ void __launch_bounds__(128) k_loss_energy(const T* buf, const typename Store<T>::Real* F, Geom g,
                                                     const void* etarget, void* lam, void* gF, int f64,
                                                     double* partials)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    double v[1] = {0.0};
    if (id.valid) {
        Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
        const int64_t N = (int64_t)g.nx * g.ny * g.nz;
        R f[St::Q];
        load_node<St, MODE>(buf, g, nb, id.n, f);
        R Fl[3] = {R(0), R(0), R(0)};
        if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
        NodeMoments<St, R> m = node_moments<St, FORCE>(f, Fl);
        const R uu = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
        const R diff = R(0.5) * m.rho * uu - (R)io_load(etarget, f64, id.n);
        v[0] = (double)diff * (double)diff;
        // dL/drho at fixed u = diff |u|^2, dL/du = 2 diff rho u
        const R gr = diff * uu;
        const R gx = R(2) * diff * m.rho * m.ux, gy = R(2) * diff * m.rho * m.uy, gz = R(2) * diff * m.rho * m.uz;
        const R inv = R(1) / m.rho;
        const R gdotu = gx * m.ux + gy * m.uy + gz * m.uz;
        if (lam) {
#pragma unroll
            for (int i = 0; i < St::Q; ++i)
                io_store(lam, f64, (int64_t)i * N + id.n, (double)(gr + (cdotu<St>(i, gx, gy, gz) - gdotu) * inv));
        }
        if (FORCE && gF) {
            io_add(gF, f64, id.n, (double)(R(0.5) * gx * inv));
            io_add(gF, f64, N + id.n, (double)(R(0.5) * gy * inv));
            if (St::D == 3) io_add(gF, f64, 2 * N + id.n, (double)(R(0.5) * gz * inv));
        }
    }
    const int64_t b = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    block_sum_store<1>(v, partials + b);
}

// ------------------------------------------------------------------ adjoint step (K6)
// lambda^n(x) = J_C(f^n(x))^T mu(x), mu_i(x) = lambda^{n+1}_i(x + c_i); the state
// buffer holds the previous step's post-collision values (AB layout), so f^n is
// pulled exactly as the forward step pulls it.
template <class St, class T, int COLL, bool FORCE>
__global__ void __launch_bounds__(128) k_adj_step(const T* state, const typename Store<T>::Real* F,
                                                  const typename Store<T>::Real* lam_in,
                                                  typename Store<T>::Real* lam_out, typename Store<T>::Real* gF,
                                                  Geom g, typename Store<T>::Real omega)
{
    using R = typename Store<T>::Real;
    NodeIdx id = node_index(g);
    if (!id.valid) return;
    Nbr nb = make_nbr<sizeof(T)>(g, id.x, id.y, id.z);
    R f[St::Q], mu[St::Q];
    load_node<St, AB>(state, g, nb, id.n, f);
#pragma unroll
    for (int i = 0; i < St::Q; ++i)
        mu[i] = lam_in[(int64_t)i * g.plane + nb.node(g, St::c(i, 0), St::c(i, 1), St::c(i, 2))];
    R Fl[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) load_force<St>(F, g, id.n, Fl);
    R gFl[3];
    adjoint_node<St, COLL, FORCE>(f, Fl, mu, omega, gFl);
#pragma unroll
    for (int i = 0; i < St::Q; ++i) lam_out[(int64_t)i * g.plane + id.n] = mu[i];
    if constexpr (FORCE) {
        gF[id.n] += gFl[0];
        gF[g.plane + id.n] += gFl[1];
        if (St::D == 3) gF[2 * g.plane + id.n] += gFl[2];
    }
}

// Two nodes per thread (x0 = 2 t, x0 + 1; nx even), the access pattern of k_update_pair:
// the state is pulled from x - c_i, the adjoints from x + c_i; accesses whose x shift is 0
// are one aligned vector load / store for both nodes.
template <class St, class T, int COLL, bool FORCE>
__global__ void __launch_bounds__(128) k_adj_step_pair(const T* state, const typename Store<T>::Real* F,
                                                       const typename Store<T>::Real* lam_in,
                                                       typename Store<T>::Real* lam_out,
                                                       typename Store<T>::Real* gF, Geom g,
                                                       typename Store<T>::Real omega)
{
    using R = typename Store<T>::Real;
    constexpr int S = sizeof(T), SR = sizeof(R);
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= g.nx) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int yy[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
    const int zz[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
    const int xm = x0 == 0 ? g.nx - 1 : x0 - 1, x2 = x0 + 2 == g.nx ? 0 : x0 + 2;
    auto row = [&](int dy, int dz) -> int64_t { return (int64_t)yy[dy + 1] + (int64_t)g.ny * zz[dz + 1]; };
    R f0[St::Q], f1[St::Q], m0[St::Q], m1[St::Q];
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const int cx = St::c(i, 0);
        // state: f_i(x) = buf_i(x - c_i)
        const char* b = (const char*)state + (int64_t)i * g.plane * S + row(-St::c(i, 1), -St::c(i, 2)) * g.nx * S;
        if (cx == 0) {
            load_pop2<St>((const T*)(b + (int64_t)x0 * S), i, f0[i], f1[i]);
        } else if (cx > 0) {
            f0[i] = load_pop<St>((const T*)(b + (int64_t)xm * S), i);
            f1[i] = load_pop<St>((const T*)(b + (int64_t)x0 * S), i);
        } else {
            f0[i] = load_pop<St>((const T*)(b + (int64_t)(x0 + 1) * S), i);
            f1[i] = load_pop<St>((const T*)(b + (int64_t)x2 * S), i);
        }
        // adjoints: mu_i(x) = lambda_i(x + c_i)
        const R* l = lam_in + (int64_t)i * g.plane + row(St::c(i, 1), St::c(i, 2)) * g.nx;
        if (cx == 0) {
            Pair2<R>::load(l + x0, m0[i], m1[i]);
        } else if (cx > 0) {
            m0[i] = l[x0 + 1];
            m1[i] = l[x2];
        } else {
            m0[i] = l[xm];
            m1[i] = l[x0];
        }
    }
    (void)SR;
    const int64_t n0 = x0 + (int64_t)g.nx * (y + (int64_t)g.ny * z);
    R F0[3] = {R(0), R(0), R(0)}, F1[3] = {R(0), R(0), R(0)};
    if constexpr (FORCE) {
        Pair2<R>::load(F + n0, F0[0], F1[0]);
        Pair2<R>::load(F + g.plane + n0, F0[1], F1[1]);
        if (St::D == 3) Pair2<R>::load(F + 2 * g.plane + n0, F0[2], F1[2]);
    }
    R g0[3], g1[3];
    adjoint_node<St, COLL, FORCE>(f0, F0, m0, omega, g0);
    adjoint_node<St, COLL, FORCE>(f1, F1, m1, omega, g1);
#pragma unroll
    for (int i = 0; i < St::Q; ++i) Pair2<R>::store(lam_out + (int64_t)i * g.plane + n0, m0[i], m1[i]);
    if constexpr (FORCE) {
#pragma unroll
        for (int a = 0; a < St::D; ++a) {
            R* p = gF + a * g.plane + n0;
            R a0, a1;
            Pair2<R>::load(p, a0, a1);
            Pair2<R>::store(p, a0 + g0[a], a1 + g1[a]);
        }
    }
}

// ------------------------------------------------------------------ dispatch
template <class R>
inline Relax<R> relax_of(const OpArgs& a)
{
    return {(R)a.omega, {(R)a.rx[0], (R)a.rx[1], (R)a.rx[2]}};
}

// the two-nodes-per-thread grid (up to 256 x positions per block, one block row per (y, z))
// would leave SMs without a block. Measured on 152 SMs: D2Q9 FP64 64^2 6.1 us per step with
// one node per thread in 32-thread blocks against 9.2 us with two; D2Q9 FP32 256^2 (256 rows)
// is 1-2 % faster with two.
inline bool small_grid(const OpArgs& a)
{
    const int64_t blocks = (int64_t)((a.g.nx + 255) / 256) * a.g.ny * a.g.nz;
    return a.sms > 0 && blocks < (int64_t)a.sms;
}

// nodes per thread of the stream-collide launch: the requested shape (a.npt), or from the
// grid when a.npt == 0, lowered to what nx and the storage allow
template <class St, class T, int COLL>
inline int update_shape(const OpArgs& a)
{
    if (COLL == NONE) return 1;  // streaming only: stored values move untouched, one per thread
    int npt = a.npt;
    if (npt == 0) {
        // four per thread for half storage, except D3Q27 KBC, whose 27 entropic weights per
        // node make four nodes too many live registers, and with a body force (the Guo source
        // takes the four-node kernel to 168 registers: D3Q19 FP16 at 256^3 runs 64.0 GLUPS
        // with two nodes per thread, 60.5 with four)
        const bool quad_ok = Store<T>::half && !(St::Q == 27 && COLL == KBC) && !a.force;
        npt = small_grid(a) ? 1 : (quad_ok ? 4 : 2);
    }
    if (npt == 4 && !(Store<T>::half && a.g.nx % 4 == 0)) npt = 2;
    if (npt == 2 && a.g.nx % 2 != 0) npt = 1;
    return npt;
}

template <class St, class T, int COLL, bool FORCE>
cudaError_t launch_update(const OpArgs& a)
{
    using R = typename Store<T>::Real;
    const T* src = (const T*)a.src;
    T* dst = (T*)a.dst;
    const R* F = (const R*)a.F;
    const Relax<R> rx = relax_of<R>(a);
    const int npt = update_shape<St, T, COLL>(a);
    if constexpr (Store<T>::half) {
        if (npt == 4) {
            // four nodes per thread for half storage
            const int quads = a.g.nx / 4;
            const dim3 bl(quads >= 128 ? 128 : ((quads + 31) / 32) * 32, 1, 1);
            const dim3 gr((quads + bl.x - 1) / bl.x, a.g.ny, a.g.nz);
            if (a.g.links) {  // walls: AB only
                if constexpr (COLL != NONE)
                    k_update_quad<St, T, COLL, FORCE, AB, true><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx,
                                                                                         a.status);
            } else if (a.mode == AB)
                k_update_quad<St, T, COLL, FORCE, AB><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
            else if (a.mode == AA_EVEN)
                k_update_quad<St, T, COLL, FORCE, AA_EVEN><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx,
                                                                                     a.status);
            else
                k_update_quad<St, T, COLL, FORCE, AA_ODD><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx,
                                                                                    a.status);
            return cudaGetLastError();
        }
    }
    if (npt == 2) {
        // two nodes per thread; 128 threads cover 256 x positions
        const int pairs = a.g.nx / 2;
        const dim3 bl(pairs >= 128 ? 128 : ((pairs + 31) / 32) * 32, 1, 1);
        const dim3 gr((pairs + bl.x - 1) / bl.x, a.g.ny, a.g.nz);
        if (a.g.links) {  // walls: AB only
            if constexpr (COLL != NONE)
                k_update_pair<St, T, COLL, FORCE, AB, true><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
        } else if (a.mode == AB)
            k_update_pair<St, T, COLL, FORCE, AB><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
        else if (a.mode == AA_EVEN)
            k_update_pair<St, T, COLL, FORCE, AA_EVEN><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
        else
            k_update_pair<St, T, COLL, FORCE, AA_ODD><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
        return cudaGetLastError();
    }
    // one node per thread; on a grid too small to give every SM two rows, 32-thread blocks
    // spread the nodes over more SMs (the FP64 collision is ALU-bound on this part)
    const dim3 bl = small_grid(a) ? dim3(32, 1, 1) : node_block(a.g);
    const dim3 gr((a.g.nx + bl.x - 1) / bl.x, a.g.ny, a.g.nz);
    if (a.mode == AB) k_update<St, T, COLL, FORCE, AB><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
    else if (a.mode == AA_EVEN)
        k_update<St, T, COLL, FORCE, AA_EVEN><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
    else k_update<St, T, COLL, FORCE, AA_ODD><<<gr, bl, 0, a.stream>>>(src, dst, F, a.g, rx, a.status);
    return cudaGetLastError();
}

template <class St, class T, int MODE, bool FORCE>
cudaError_t launch_state_op(const OpArgs& a)
{
    using R = typename Store<T>::Real;
    const dim3 gr = node_grid(a.g), bl = node_block(a.g);
    const R* F = (const R*)a.F;
    switch (a.op) {
    case OP_INIT_EQ:
        if (MODE == AA_ODD) return cudaErrorInvalidValue;
        k_init_eq<St, T, MODE><<<gr, bl, 0, a.stream>>>((T*)a.dst, a.g, a.in0, a.in1, a.io_f64);
        break;
    case OP_SET:
        if (MODE == AA_ODD) return cudaErrorInvalidValue;
        k_set<St, T, MODE><<<gr, bl, 0, a.stream>>>((T*)a.dst, a.g, a.in0, a.io_f64);
        break;
    case OP_GET: k_get<St, T, MODE><<<gr, bl, 0, a.stream>>>((const T*)a.src, a.g, a.out0, a.io_f64); break;
    case OP_MOMENTS:
        k_moments<St, T, MODE, FORCE><<<gr, bl, 0, a.stream>>>((const T*)a.src, F, a.g, a.out0, a.out1, a.io_f64);
        break;
    case OP_REDUCE_PARTIAL:
        k_reduce_partial<St, T, MODE, FORCE><<<gr, bl, 0, a.stream>>>((const T*)a.src, F, a.g, a.partials);
        break;
    case OP_ADJ_SEED:
        k_adj_seed<St, T, MODE, FORCE><<<gr, bl, 0, a.stream>>>((const T*)a.src, F, a.g, a.in0, a.in1, a.out0,
                                                                a.out1, a.io_f64);
        break;
    case OP_LINKS:
        if (MODE != AB) return cudaErrorInvalidValue;
        k_build_links<St><<<gr, bl, 0, a.stream>>>((const unsigned char*)a.in0, a.g, (unsigned*)a.out0);
        break;
    case OP_LOSS_ENERGY:
        k_loss_energy<St, T, MODE, FORCE><<<gr, bl, 0, a.stream>>>((const T*)a.src, F, a.g, a.in0, a.out0, a.out1,
                                                                   a.io_f64, a.partials);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class St, class T, int COLL>
cudaError_t launch_adj(const OpArgs& a)
{
    using R = typename Store<T>::Real;
    if (a.g.nx % 2 == 0) {
        const int pairs = a.g.nx / 2;
        const dim3 bl(pairs >= 128 ? 128 : ((pairs + 31) / 32) * 32, 1, 1);
        const dim3 gr((pairs + bl.x - 1) / bl.x, a.g.ny, a.g.nz);
        if (a.force)
            k_adj_step_pair<St, T, COLL, true><<<gr, bl, 0, a.stream>>>((const T*)a.src, (const R*)a.F,
                                                                        (const R*)a.lam_in, (R*)a.lam_out, (R*)a.gF,
                                                                        a.g, (R)a.omega);
        else
            k_adj_step_pair<St, T, COLL, false><<<gr, bl, 0, a.stream>>>((const T*)a.src, nullptr, (const R*)a.lam_in,
                                                                         (R*)a.lam_out, nullptr, a.g, (R)a.omega);
        return cudaGetLastError();
    }
    const dim3 gr = node_grid(a.g), bl = node_block(a.g);
    if (a.force)
        k_adj_step<St, T, COLL, true><<<gr, bl, 0, a.stream>>>((const T*)a.src, (const R*)a.F, (const R*)a.lam_in,
                                                               (R*)a.lam_out, (R*)a.gF, a.g, (R)a.omega);
    else
        k_adj_step<St, T, COLL, false><<<gr, bl, 0, a.stream>>>((const T*)a.src, nullptr, (const R*)a.lam_in,
                                                                (R*)a.lam_out, nullptr, a.g, (R)a.omega);
    return cudaGetLastError();
}

template <class St, class T>
cudaError_t run_op_typed(const OpArgs& a)
{
    if (a.op == OP_UPDATE) {
        switch (a.coll) {
        case BGK: return a.force ? launch_update<St, T, BGK, true>(a) : launch_update<St, T, BGK, false>(a);
        case REG: return a.force ? launch_update<St, T, REG, true>(a) : launch_update<St, T, REG, false>(a);
        case NONE: return launch_update<St, T, NONE, false>(a);
        case TRT: return a.force ? launch_update<St, T, TRT, true>(a) : launch_update<St, T, TRT, false>(a);
        case KBC:
            if constexpr (coll_supported<St>(KBC)) return a.force ? cudaErrorInvalidValue : launch_update<St, T, KBC, false>(a);
            return cudaErrorInvalidValue;
        case MRT:
            if constexpr (coll_supported<St>(MRT)) return a.force ? cudaErrorInvalidValue : launch_update<St, T, MRT, false>(a);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.op == OP_ADJ_STEP) {
        switch (a.coll) {
        case BGK: return launch_adj<St, T, BGK>(a);
        case REG: return launch_adj<St, T, REG>(a);
        case NONE: return launch_adj<St, T, NONE>(a);
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.mode == AB) return a.force ? launch_state_op<St, T, AB, true>(a) : launch_state_op<St, T, AB, false>(a);
    if (a.mode == AA_EVEN)
        return a.force ? launch_state_op<St, T, AA_EVEN, true>(a) : launch_state_op<St, T, AA_EVEN, false>(a);
    return a.force ? launch_state_op<St, T, AA_ODD, true>(a) : launch_state_op<St, T, AA_ODD, false>(a);
}

}  // namespace lb
