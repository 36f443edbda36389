// Per-node collision in registers: moments (Eq. 4), second-order equilibrium
// (Eq. 3), BGK (Eq. 2), regularized (Latt & Chopard) and the Guo body-force source.
// R is the arithmetic type (double or float). All values are deviations from rest,
// delta_i = f_i - w_i (so rho - 1 = sum delta, rho u = sum c delta + F/2); the
// arrays d[Q] are replaced by their post-collision deviations.
#pragma once

#include "lb_device.cuh"

namespace lb {

enum Coll { BGK = 0, REG = 1, LEARNED = 2, NONE = 3 };

// 1/x rounded to nearest (FP32: the hardware reciprocal with IEEE rounding, not a division)
LB_DEV float recip(float x) { return __frcp_rn(x); }
LB_DEV double recip(double x) { return 1.0 / x; }

template <class St, class R>
struct NodeMoments {
    R rho, ux, uy, uz;
    R rho1;  // rho - 1
};

// rho - 1 = sum delta, u = (sum c delta + F/2) / rho (sum w c = 0)
template <class St, bool FORCE, class R>
LB_DEV NodeMoments<St, R> node_moments(const R* d, const R* F)
{
    R rho1 = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        rho1 += d[i];
        if (St::c(i, 0)) jx += St::c(i, 0) > 0 ? d[i] : -d[i];
        if (St::c(i, 1)) jy += St::c(i, 1) > 0 ? d[i] : -d[i];
        if (St::D == 3 && St::c(i, 2)) jz += St::c(i, 2) > 0 ? d[i] : -d[i];
    }
    if constexpr (FORCE) {
        jx += R(0.5) * F[0];
        jy += R(0.5) * F[1];
        if (St::D == 3) jz += R(0.5) * F[2];
    }
    const R rho = R(1) + rho1;
    const R inv = recip(rho);
    return {rho, jx * inv, jy * inv, jz * inv, rho1};
}

template <class St, class R>
LB_DEV R cdotu(int i, R ux, R uy, R uz)
{
    R cu = R(0);
    if (St::c(i, 0)) cu += St::c(i, 0) > 0 ? ux : -ux;
    if (St::c(i, 1)) cu += St::c(i, 1) > 0 ? uy : -uy;
    if (St::D == 3 && St::c(i, 2)) cu += St::c(i, 2) > 0 ? uz : -uz;
    return cu;
}

// f^eq_i - w_i, with f^eq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)   (c_s^2 = 1/3):
// deq_i = w_i [(rho - 1) + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)]. The bracket is summed
// before the single multiplication by w_i; splitting it into separately rounded even
// and odd parts of the opposite pair measurably biased the FP32 energy decay.
template <class St, class R>
LB_DEV void equilibrium(const NodeMoments<St, R>& m, R* deq)
{
    const R uu15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
#pragma unroll
    for (int i = 0; i < St::Q; ++i) {
        const R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
        deq[i] = R(St::w(i)) * (m.rho1 + m.rho * (cu * (R(3) + R(4.5) * cu) - uu15));
    }
}

// Guo source: S_i = (1 - omega/2) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]
template <class St, class R>
LB_DEV R guo_source(int i, const NodeMoments<St, R>& m, const R* F, R pre)
{
    R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
    R cF = cdotu<St>(i, F[0], F[1], St::D == 3 ? F[2] : R(0));
    R uF = m.ux * F[0] + m.uy * F[1] + (St::D == 3 ? m.uz * F[2] : R(0));
    return pre * R(St::w(i)) * (R(3) * (cF - uF) + R(9) * cu * cF);
}

// In-place collision of one node (f holds the deviations delta). Returns false if
// the density is not a positive finite number (the caller raises the status flag).
template <class St, int COLL, bool FORCE, class R>
LB_DEV bool collide(R* f, const R* F, R omega)
{
    if constexpr (COLL == NONE) {
        return true;
    } else {
        NodeMoments<St, R> m = node_moments<St, FORCE>(f, F);
        R feq[St::Q];
        const R pre = R(1) - R(0.5) * omega;
        if constexpr (COLL == BGK) {
            // f* = f - omega (f - f^eq) (+ S), Eq. 2 as written: the non-equilibrium part is
            // formed first. Near omega = 2 the forms (1 - omega) f + omega f^eq and
            // f^eq + (1 - omega)(f - f^eq) lose FP32 accuracy (3-20x the TGV energy error
            // in an FP32 emulation of the three forms against FP64).
            equilibrium<St>(m, feq);
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                R v = f[i] - omega * (f[i] - feq[i]);
                if constexpr (FORCE) v += guo_source<St>(i, m, F, pre);
                f[i] = v;
            }
        } else {
            equilibrium<St>(m, feq);  // REG: keep only the Hermite order <= 2 projection of f - f^eq
            R pxx = R(0), pyy = R(0), pzz = R(0), pxy = R(0), pxz = R(0), pyz = R(0);
            R ax = R(0), ay = R(0), az = R(0);
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                const R d = f[i] - feq[i];
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                if (cx) pxx += d;
                if (cy) pyy += d;
                if (St::D == 3 && cz) pzz += d;
                if (cx && cy) pxy += (cx == cy) ? d : -d;
                if (St::D == 3 && cx && cz) pxz += (cx == cz) ? d : -d;
                if (St::D == 3 && cy && cz) pyz += (cy == cz) ? d : -d;
                if constexpr (FORCE) {
                    if (cx) ax += cx > 0 ? d : -d;
                    if (cy) ay += cy > 0 ? d : -d;
                    if (St::D == 3 && cz) az += cz > 0 ? d : -d;
                }
            }
            const R tr = pxx + pyy + pzz;
            const R relax = R(1) - omega;
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                // (c c - cs2 I) : Pi
                R qp = -tr * R(1.0 / 3.0);
                if (cx) qp += pxx;
                if (cy) qp += pyy;
                if (St::D == 3 && cz) qp += pzz;
                if (cx && cy) qp += (cx == cy) ? R(2) * pxy : R(-2) * pxy;
                if (St::D == 3 && cx && cz) qp += (cx == cz) ? R(2) * pxz : R(-2) * pxz;
                if (St::D == 3 && cy && cz) qp += (cy == cz) ? R(2) * pyz : R(-2) * pyz;
                R neq = R(4.5) * qp;
                if constexpr (FORCE) neq += R(3) * cdotu<St>(i, ax, ay, az);
                R v = feq[i] + relax * R(St::w(i)) * neq;
                if constexpr (FORCE) v += guo_source<St>(i, m, F, pre);
                f[i] = v;
            }
        }
        return m.rho > R(0) && m.rho < R(1e30);
    }
}

}  // namespace lb
