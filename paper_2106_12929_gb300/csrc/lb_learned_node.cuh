// Per-node pieces of the learned moment-space collision on D2Q9 (Eq. 5, Sec. 3.1) shared
// by the FP64 kernels (lb_learned.cu) and the tensor-core kernels of the FP32 arithmetic
// (lb_learned_x3.cu): moments and network inputs, the post-collision populations, and the
// parts of the discrete adjoint outside the network.
//
// Populations are handled as deviations delta_i = f_i - w_i (as in lb_collide.cuh).
// Moment basis (Hermite, orthogonal under the weights w_i): 1, cx, cy,
// cx^2 - 1/3, cx cy, cy^2 - 1/3 (stress rows), (cx^2 - 1/3) cy, cx (cy^2 - 1/3),
// (cx^2 - 1/3)(cy^2 - 1/3) (higher rows; their equilibria vanish for the
// second-order f^eq). With d = f - f^eq, Pi = sum c c d and the higher moments
// g = sum H d, the collision is
//   f*_i = f^eq_i + (1 - w_s) 4.5 w_i (c_i c_i - I/3) : Pi
//                 + (1 - w_g) w_i sum_g H_g(c_i) g_g / |H_g|^2_w,
// w_s = 1/tau (stress rows), w_g = 1/(exp(z) + 1/2) from the per-node network output z of
// the standardised invariants x_k = (I_k - shift_k) scale_k:
//   I1 = rho - 1, I2 = 3|u|^2, I3 = 3 tr Pi, I4 = 9 Pi:Pi, I5 = 9 u.Pi.u,
//   I6 = sum_g g_g^2 / |H_g|^2_w.
#pragma once

#include "lb_collide.cuh"
#include "lb_learned.cuh"

namespace lb {

// Hermite higher-moment polynomials on D2Q9 and their weighted norms
LB_HD constexpr double h6(int i) { return (c2(i, 0) * c2(i, 0) - 1.0 / 3.0) * c2(i, 1); }
LB_HD constexpr double h7(int i) { return c2(i, 0) * (c2(i, 1) * c2(i, 1) - 1.0 / 3.0); }
LB_HD constexpr double h8(int i) { return (c2(i, 0) * c2(i, 0) - 1.0 / 3.0) * (c2(i, 1) * c2(i, 1) - 1.0 / 3.0); }
constexpr double kN6 = 2.0 / 27.0, kN7 = 2.0 / 27.0, kN8 = 4.0 / 81.0;

// Activation tanh. FP64: the accurate library tanh (the gradient checks against the
// oracle). FP32: tanh a = 1 - 2 / (e^{2a} + 1) with e^{2a} from the hardware base-2
// exponential of 2a / ln 2 and the hardware reciprocal (PTX ex2.approx, rcp.approx; relative
// errors about 2^-22 and 2^-23), so the result is within about 1e-7 absolute of tanh a
// and saturates to +-1 exactly for large |a|. The forward step, the adjoint's forward
// recomputation and its derivative 1 - tanh^2 all see this function.
LB_DEV float ex2_approx(float a)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}
LB_DEV float rcp_approx(float a)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}
constexpr float kTwoOverLn2 = 2.8853900817779268f;
// tanh a from t = 2a / ln 2 (callers that form a as a fused multiply-add fold the factor in)
LB_DEV float tanh_of_t(float t) { return 1.0f - 2.0f * rcp_approx(ex2_approx(t) + 1.0f); }
template <class R> LB_DEV R act_tanh(R a);
template <> LB_DEV float act_tanh<float>(float a) { return tanh_of_t(a * kTwoOverLn2); }
template <> LB_DEV double act_tanh<double>(double a) { return tanh(a); }
template <class R> LB_DEV R act_exp(R a);
template <> LB_DEV float act_exp<float>(float a) { return expf(a); }
template <> LB_DEV double act_exp<double>(double a) { return exp(a); }

// The moments of one node that both networks read: density and velocity, non-equilibrium
// stress Pi and higher moments g6, g7, g8.
template <class R>
struct LearnedMoments {
    NodeMoments<D2Q9, R> m;
    R pxx, pxy, pyy, g6, g7, g8;
};

// Everything the forward pass of one node computes (kept for the adjoint).
template <class R>
struct LearnedNode : LearnedMoments<R> {
    R x[kNetIn];
    R h1[kNetHidden], h2[kNetHidden];
    R z, ez, omg;
};

// Moments, stress and higher moments, and the six network inputs of one node, from the
// deviations delta_i = f_i - w_i. The second-order equilibrium's moments are closed forms:
// sum c c (f^eq - w) = rho u u + (rho - 1)/3 I, and its higher Hermite moments vanish, so
// Pi = sum c c delta - rho u u - (rho - 1)/3 I and g = sum H delta.
template <class R>
LB_DEV void learned_inputs(const R* f, LearnedMoments<R>& s, R* I)
{
    R Fz[3] = {R(0), R(0), R(0)};
    s.m = node_moments<D2Q9, false>(f, Fz);
    R sxx = R(0), sxy = R(0), syy = R(0), g6 = R(0), g7 = R(0), g8 = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R d = f[i];
        const int cx = c2(i, 0), cy = c2(i, 1);
        if (cx) sxx += d;
        if (cy) syy += d;
        if (cx && cy) sxy += (cx == cy) ? d : -d;
        g6 += R(h6(i)) * d;
        g7 += R(h7(i)) * d;
        g8 += R(h8(i)) * d;
    }
    const R ux = s.m.ux, uy = s.m.uy, rho = s.m.rho;
    const R r3 = s.m.rho1 * R(1.0 / 3.0);
    const R pxx = sxx - rho * ux * ux - r3, pyy = syy - rho * uy * uy - r3, pxy = sxy - rho * ux * uy;
    s.pxx = pxx; s.pxy = pxy; s.pyy = pyy; s.g6 = g6; s.g7 = g7; s.g8 = g8;
    I[0] = s.m.rho1;
    I[1] = R(3) * (ux * ux + uy * uy);
    I[2] = R(3) * (pxx + pyy);
    I[3] = R(9) * (pxx * pxx + R(2) * pxy * pxy + pyy * pyy);
    I[4] = R(9) * (ux * ux * pxx + R(2) * ux * uy * pxy + uy * uy * pyy);
    I[5] = g6 * g6 * R(1.0 / kN6) + g7 * g7 * R(1.0 / kN7) + g8 * g8 * R(1.0 / kN8);
}

// Post-collision populations of one node with higher-moment rate omg (one shared rate).
template <class R>
LB_DEV void learned_post(const LearnedMoments<R>& s, R omg, R omega, R* f)
{
    const R ks = R(4.5) * (R(1) - omega);
    const R kg = R(1) - omg;
    const R tr3 = (s.pxx + s.pyy) * R(1.0 / 3.0);
    const R q6 = s.g6 * R(1.0 / kN6), q7 = s.g7 * R(1.0 / kN7), q8 = s.g8 * R(1.0 / kN8);
    R feq[9];
    equilibrium<D2Q9>(s.m, feq);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c2(i, 0), cy = c2(i, 1);
        R qp = -tr3;
        if (cx) qp += s.pxx;
        if (cy) qp += s.pyy;
        if (cx && cy) qp += (cx == cy) ? R(2) * s.pxy : R(-2) * s.pxy;
        const R ghost = R(h6(i)) * q6 + R(h7(i)) * q7 + R(h8(i)) * q8;
        f[i] = feq[i] + R(D2Q9::w(i)) * (ks * qp + kg * ghost);
    }
}

// Cotangents of the per-node quantities of the learned collision, built up by the adjoint:
// density, velocity, non-equilibrium stress and higher moments; q_g are the adjoint's
// projections sum_i mu_i w_i H_g(c_i) / |H_g|^2_w onto the higher rows.
template <class R>
struct LearnedCot {
    R grho, gux, guy, gPxx, gPxy, gPyy, gg6, gg7, gg8;
    R q6, q7, q8;
};

// The paths through the equilibrium and the stress rows of f*; the higher rows' terms
// (which depend on the network) are added by the caller.
template <class R>
LB_DEV LearnedCot<R> learned_adj_head(const LearnedMoments<R>& s, const R* mu, R omega)
{
    const R ux = s.m.ux, uy = s.m.uy, rho = s.m.rho;
    // sums of mu w over the basis
    R smw = R(0), smwcx = R(0), smwcy = R(0), smwcucx = R(0), smwcucy = R(0), grho = R(0);
    R sxx = R(0), syy = R(0), sxy = R(0), s6 = R(0), s7 = R(0), s8 = R(0);
    const R base = R(1) - R(1.5) * (ux * ux + uy * uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R mw = mu[i] * R(D2Q9::w(i));
        const int cx = c2(i, 0), cy = c2(i, 1);
        const R cu = cdotu<D2Q9>(i, ux, uy, R(0));
        grho += mw * (base + cu * (R(3) + R(4.5) * cu));
        smw += mw;
        smwcx += cx * mw;
        smwcy += cy * mw;
        smwcucx += cx * mw * cu;
        smwcucy += cy * mw * cu;
        if (cx) sxx += mw;
        if (cy) syy += mw;
        if (cx && cy) sxy += (cx == cy) ? mw : -mw;
        s6 += R(h6(i)) * mw;
        s7 += R(h7(i)) * mw;
        s8 += R(h8(i)) * mw;
    }
    LearnedCot<R> c;
    c.grho = grho;
    // equilibrium path: d f^eq / d rho, d f^eq / d u
    c.gux = rho * (R(3) * smwcx + R(9) * smwcucx - R(3) * ux * smw);
    c.guy = rho * (R(3) * smwcy + R(9) * smwcucy - R(3) * uy * smw);
    // stress path: cotangent of (Pxx, Pxy, Pyy) from 4.5 (1 - w_s) w_i Q_i : Pi
    const R ks = R(4.5) * (R(1) - omega);
    c.gPxx = ks * (sxx - smw * R(1.0 / 3.0));
    c.gPyy = ks * (syy - smw * R(1.0 / 3.0));
    c.gPxy = R(2) * ks * sxy;
    c.q6 = s6 * R(1.0 / kN6);
    c.q7 = s7 * R(1.0 / kN7);
    c.q8 = s8 * R(1.0 / kN8);
    return c;
}

// Back through the six network inputs (cotangent gI of the unstandardised invariants) and
// the moments to lambda_i = d(mu . f*)/d f_i, written to lam_out[i][n].
template <class R>
LB_DEV void learned_adj_tail(const LearnedMoments<R>& s, LearnedCot<R> c, const R* gI, R* lam_out, int64_t plane,
                             int n)
{
    const R ux = s.m.ux, uy = s.m.uy, rho = s.m.rho;
    R grho = c.grho, gux = c.gux, guy = c.guy, gPxx = c.gPxx, gPyy = c.gPyy, gPxy = c.gPxy;
    R gg6 = c.gg6, gg7 = c.gg7, gg8 = c.gg8;
    grho += gI[0];
    gux += R(6) * ux * gI[1];
    guy += R(6) * uy * gI[1];
    gPxx += R(3) * gI[2] + R(18) * s.pxx * gI[3] + R(9) * ux * ux * gI[4];
    gPyy += R(3) * gI[2] + R(18) * s.pyy * gI[3] + R(9) * uy * uy * gI[4];
    gPxy += R(36) * s.pxy * gI[3] + R(18) * ux * uy * gI[4];
    gux += R(18) * (ux * s.pxx + uy * s.pxy) * gI[4];
    guy += R(18) * (ux * s.pxy + uy * s.pyy) * gI[4];
    gg6 += R(2) * s.g6 * R(1.0 / kN6) * gI[5];
    gg7 += R(2) * s.g7 * R(1.0 / kN7) * gI[5];
    gg8 += R(2) * s.g8 * R(1.0 / kN8) * gI[5];
    // Pi = sum c c f - rho u u - rho I/3
    grho -= gPxx * (ux * ux + R(1.0 / 3.0)) + gPxy * ux * uy + gPyy * (uy * uy + R(1.0 / 3.0));
    gux -= rho * (R(2) * ux * gPxx + uy * gPxy);
    guy -= rho * (ux * gPxy + R(2) * uy * gPyy);
    const R inv = recip(rho);
    const R gdotu = gux * ux + guy * uy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c2(i, 0), cy = c2(i, 1);
        // direct paths: Pi (c c) and the higher moments (H_g); the equilibrium
        // term of f* has no direct dependence on f
        R v = R(0);
        if (cx) v += gPxx;
        if (cy) v += gPyy;
        if (cx && cy) v += (cx == cy) ? gPxy : -gPxy;
        v += R(h6(i)) * gg6 + R(h7(i)) * gg7 + R(h8(i)) * gg8;
        v += grho + (cdotu<D2Q9>(i, gux, guy, R(0)) - gdotu) * inv;
        lam_out[(int64_t)i * plane + n] = v;
    }
}

// higher row set by output o (0: row (cx^2 - 1/3) cy, 1: cx (cy^2 - 1/3), 2: the fourth-order row)
LB_HD constexpr int net3_row(int o) { return o == 0 ? 2 : o - 1; }

template <class R>
struct Learned3Node : LearnedMoments<R> {
    R x[kNetIn];
    R h[kNet3Hidden];
    R ez[3], omg[3];  // per higher row, in row order
};

// Post-collision populations of one node with one rate per higher row (omg[0..2] for the
// rows (cx^2 - 1/3) cy, cx (cy^2 - 1/3), (cx^2 - 1/3)(cy^2 - 1/3)).
template <class R>
LB_DEV void learned3_post(const LearnedMoments<R>& s, const R* omg, R omega, R* f)
{
    const R ks = R(4.5) * (R(1) - omega);
    const R tr3 = (s.pxx + s.pyy) * R(1.0 / 3.0);
    const R q6 = (R(1) - omg[0]) * s.g6 * R(1.0 / kN6);
    const R q7 = (R(1) - omg[1]) * s.g7 * R(1.0 / kN7);
    const R q8 = (R(1) - omg[2]) * s.g8 * R(1.0 / kN8);
    R feq[9];
    equilibrium<D2Q9>(s.m, feq);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = c2(i, 0), cy = c2(i, 1);
        R qp = -tr3;
        if (cx) qp += s.pxx;
        if (cy) qp += s.pyy;
        if (cx && cy) qp += (cx == cy) ? R(2) * s.pxy : R(-2) * s.pxy;
        const R ghost = R(h6(i)) * q6 + R(h7(i)) * q7 + R(h8(i)) * q8;
        f[i] = feq[i] + R(D2Q9::w(i)) * (ks * qp + ghost);
    }
}

}  // namespace lb
