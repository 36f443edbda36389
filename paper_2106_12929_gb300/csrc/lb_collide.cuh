// Per-node collision in registers: moments (Eq. 4), second-order equilibrium
// (Eq. 3), BGK (Eq. 2), regularized (Latt & Chopard), two relaxation times (Ginzburg),
// entropic KBC (Karlin, Boesch & Chikatamarla), fixed-rate moment-space MRT (Eq. 5
// with constant higher-moment times) and the Guo body-force source.
// R is the arithmetic type (double or float). All values are deviations from rest,
// delta_i = f_i - w_i (so rho - 1 = sum delta, rho u = sum c delta + F/2); the
// arrays d[Q] are replaced by their post-collision deviations.
#pragma once

#include "lb_device.cuh"

namespace lb {

enum Coll { BGK = 0, REG = 1, LEARNED = 2, NONE = 3, TRT = 4, KBC = 5, MRT = 6, LEARNED3 = 7 };

// Relaxation rates of one collision. omega = 1/tau sets the shear viscosity for every
// model; p holds the model's other constants: TRT p[0] = 1/tau_minus; KBC p[0] = 2 tau
// (= 1/beta); MRT p[0..2] = the rates of the three higher Hermite moments.
template <class R>
struct Relax {
    R omega;
    R p[3];
};

// collision model available for this velocity set (KBC needs a full tensor-product set)
template <class St>
constexpr bool coll_supported(int coll)
{
    return coll == KBC ? (St::Q == 9 || St::Q == 27) : coll == MRT ? St::Q == 9 : coll != LEARNED && coll != LEARNED3;
}

// 1/x rounded to nearest (FP32: the hardware reciprocal with IEEE rounding, not a division)
LB_DEV float recip(float x) { return __frcp_rn(x); }
LB_DEV double recip(double x) { return 1.0 / x; }
// 1/x where a few ulp suffice (FP32: the fast approximate division intrinsic)
LB_DEV float recip_fast(float x) { return __fdividef(1.0f, x); }
LB_DEV double recip_fast(double x) { return 1.0 / x; }

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
LB_DEV bool collide(R* f, const R* F, const Relax<R>& rx)
{
    if constexpr (COLL == NONE) {
        return true;
    } else {
        const R omega = rx.omega;
        NodeMoments<St, R> m = node_moments<St, FORCE>(f, F);
        R feq[St::Q];
        const R pre = R(1) - R(0.5) * omega;
        if constexpr (COLL == TRT) {
            // symmetric half of f - f^eq relaxed by omega, antisymmetric half by omega_minus;
            // the Guo source split the same way: its even part w [9 (c.u)(c.F) - 3 u.F] gets
            // (1 - omega/2), its odd part 3 w c.F gets (1 - omega_minus/2)
            equilibrium<St>(m, feq);
            const R om_m = rx.p[0];
            f[0] = f[0] - omega * (f[0] - feq[0]);
            if constexpr (FORCE) f[0] += guo_source<St>(0, m, F, pre);
#pragma unroll
            for (int i = 1; i < St::Q; i += 2) {
                const int o = i + 1;  // opp(i)
                const R ni = f[i] - feq[i], no = f[o] - feq[o];
                const R np = R(0.5) * (ni + no), nm = R(0.5) * (ni - no);
                R vi = f[i] - omega * np - om_m * nm;
                R vo = f[o] - omega * np + om_m * nm;
                if constexpr (FORCE) {
                    const R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
                    const R cF = cdotu<St>(i, F[0], F[1], St::D == 3 ? F[2] : R(0));
                    const R uF = m.ux * F[0] + m.uy * F[1] + (St::D == 3 ? m.uz * F[2] : R(0));
                    const R ev = pre * R(St::w(i)) * (R(9) * cu * cF - R(3) * uF);
                    const R od = (R(1) - R(0.5) * om_m) * R(St::w(i)) * (R(3) * cF);
                    vi += ev + od;
                    vo += ev - od;
                }
                f[i] = vi;
                f[o] = vo;
            }
        } else if constexpr (COLL == KBC) {
            // D = f - f^eq = Ds + Dh: Ds carries the trace-free second natural moments of D
            // (axis velocities: Mdev_aa / 2, edge velocities: c_a c_b M_ab / 4, rest and
            // corners: 0), Dh the rest. f* = f - beta (2 Ds + gamma Dh), beta = omega/2,
            // gamma = 1/beta - (2 - 1/beta) <Ds|Dh> / (<Dh|Dh> + 1e-6 <Ds|Ds>) with
            // <X|Y> = sum X_i Y_i / f^eq_i. Opposite velocities i, i + 1 share the even parts
            // (f^eq = w (a +- b), the second moments take pair sums, Ds is even in c), so the
            // work runs once per pair.
            static_assert(St::Q == 9 || St::Q == 27, "KBC needs D2Q9 or D3Q27");
            const R uu15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
            const R a0 = m.rho1 - m.rho * uu15, rho45 = R(4.5) * m.rho, rho3 = R(3) * m.rho;
            R D[St::Q];
            feq[0] = R(St::w(0)) * a0;
            D[0] = f[0] - feq[0];
            R mxx = R(0), myy = R(0), mzz = R(0), mxy = R(0), mxz = R(0), myz = R(0);
#pragma unroll
            for (int i = 1; i < St::Q; i += 2) {  // opp(i) = i + 1
                const R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
                const R a = a0 + rho45 * cu * cu, b = rho3 * cu;
                feq[i] = R(St::w(i)) * (a + b);
                feq[i + 1] = R(St::w(i)) * (a - b);
                D[i] = f[i] - feq[i];
                D[i + 1] = f[i + 1] - feq[i + 1];
                const R sp = D[i] + D[i + 1];
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                if (cx) mxx += sp;
                if (cy) myy += sp;
                if (St::D == 3 && cz) mzz += sp;
                if (cx && cy) mxy += (cx == cy) ? sp : -sp;
                if (St::D == 3 && cx && cz) mxz += (cx == cz) ? sp : -sp;
                if (St::D == 3 && cy && cz) myz += (cy == cz) ? sp : -sp;
            }
            const R third = R(1) / R(St::D);
            const R tr = (mxx + myy + mzz) * third;
            const R dxx = R(0.5) * (mxx - tr), dyy = R(0.5) * (myy - tr), dzz = R(0.5) * (mzz - tr);
            // entropic weights 1/f^eq_i = 1/(w_i rho P_i), P_i = 1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u.
            // An opposite pair has P = A +- B (A = 1 + 4.5 (c.u)^2 - 1.5 u.u, B = 3 c.u), so one
            // reciprocal 1/(A^2 - B^2) serves both: 1/P_i = (A - B)/(A^2 - B^2), 1/P_opp = (A + B)/(...).
            const R irho = recip_fast(m.rho);
            const R ie0 = irho * R(1.0 / St::w(0)) * recip_fast(R(1) - uu15);
            R sh = R(0), hh = ie0 * D[0] * D[0], ss = R(0);
            R Ds[St::Q];
            Ds[0] = R(0);
#pragma unroll
            for (int i = 1; i < St::Q; i += 2) {
                const R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
                const R A = R(1) - uu15 + R(4.5) * cu * cu, B = R(3) * cu;
                const R r = irho * R(1.0 / St::w(i)) * recip_fast(A * A - B * B);  // w_i = w_opp(i)
                const R iei = (A - B) * r, iej = (A + B) * r;
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                const int nz = (cx != 0) + (cy != 0) + (cz != 0);
                if (nz == 1 || nz == 2) {
                    R sv;
                    if (nz == 1) sv = cx ? dxx : (cy ? dyy : dzz);
                    else if (cx && cy) sv = (cx == cy) ? R(0.25) * mxy : R(-0.25) * mxy;
                    else if (cx && cz) sv = (cx == cz) ? R(0.25) * mxz : R(-0.25) * mxz;
                    else sv = (cy == cz) ? R(0.25) * myz : R(-0.25) * myz;
                    Ds[i] = Ds[i + 1] = sv;
                    const R hi = D[i] - sv, hj = D[i + 1] - sv;
                    const R wi = iei * hi, wj = iej * hj;
                    sh += sv * (wi + wj);
                    ss += sv * sv * (iei + iej);
                    hh += wi * hi + wj * hj;
                } else {
                    Ds[i] = Ds[i + 1] = R(0);
                    hh += iei * D[i] * D[i] + iej * D[i + 1] * D[i + 1];
                }
            }
            const R beta = R(0.5) * omega, ib = rx.p[0];  // p[0] = 1/beta = 2 tau
            const R den = hh + R(1e-6) * ss;
            const R gamma = den > R(0) ? ib - (R(2) - ib) * sh * recip(den) : R(2);
            const R bg = beta * gamma, b2 = R(2) * beta;
#pragma unroll
            for (int i = 0; i < St::Q; ++i) f[i] = f[i] - (b2 * Ds[i] + bg * (D[i] - Ds[i]));
        } else if constexpr (COLL == MRT) {
            // D2Q9 Hermite moments of D = f - f^eq: stress (order 2) relaxed by omega, the
            // three higher moments (cx^2 - 1/3) cy, cx (cy^2 - 1/3), (cx^2 - 1/3)(cy^2 - 1/3)
            // by p[0..2]; f* = f - sum_a rate_a w_i H_a(c_i) m_a / |H_a|_w^2
            static_assert(St::Q == 9, "MRT is D2Q9 only");
            equilibrium<St>(m, feq);
            R D[9];
            R pxx = R(0), pyy = R(0), pxy = R(0), g6 = R(0), g7 = R(0), g8 = R(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                D[i] = f[i] - feq[i];
                const int cx = St::c(i, 0), cy = St::c(i, 1);
                const R hx = cx ? R(2.0 / 3.0) : R(-1.0 / 3.0), hy = cy ? R(2.0 / 3.0) : R(-1.0 / 3.0);
                if (cx) pxx += D[i];
                if (cy) pyy += D[i];
                if (cx && cy) pxy += (cx == cy) ? D[i] : -D[i];
                if (cy) g6 += cy > 0 ? hx * D[i] : -hx * D[i];
                if (cx) g7 += cx > 0 ? hy * D[i] : -hy * D[i];
                g8 += hx * hy * D[i];
            }
            // |H|_w^2: (cx^2 - 1/3) cy and cx (cy^2 - 1/3): 2/27; (cx^2 - 1/3)(cy^2 - 1/3): 4/81
            g6 *= rx.p[0] * R(27.0 / 2.0);
            g7 *= rx.p[1] * R(27.0 / 2.0);
            g8 *= rx.p[2] * R(81.0 / 4.0);
            const R tr = pxx + pyy;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int cx = St::c(i, 0), cy = St::c(i, 1);
                const R hx = cx ? R(2.0 / 3.0) : R(-1.0 / 3.0), hy = cy ? R(2.0 / 3.0) : R(-1.0 / 3.0);
                R qp = -tr * R(1.0 / 3.0);
                if (cx) qp += pxx;
                if (cy) qp += pyy;
                if (cx && cy) qp += (cx == cy) ? R(2) * pxy : R(-2) * pxy;
                R ghost = hx * hy * g8;
                if (cy) ghost += cy > 0 ? hx * g6 : -hx * g6;
                if (cx) ghost += cx > 0 ? hy * g7 : -hy * g7;
                f[i] = f[i] - R(St::w(i)) * (omega * R(4.5) * qp + ghost);
            }
        } else if constexpr (COLL == BGK) {
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
            // REG: keep only the Hermite order <= 2 projection of f - f^eq. Opposite velocities
            // i, i + 1 share the even parts, which halves the work per pair: f^eq = w (a +- b)
            // with a = (rho - 1) + rho (4.5 (c.u)^2 - 1.5 u.u) and b = 3 rho c.u; the second
            // moments of f - f^eq take the pair sums; the correction (c c - I/3):Pi is even in c.
            const R uu15 = R(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
            const R a0 = m.rho1 - m.rho * uu15, rho45 = R(4.5) * m.rho, rho3 = R(3) * m.rho;
            feq[0] = R(St::w(0)) * a0;
            R pxx = R(0), pyy = R(0), pzz = R(0), pxy = R(0), pxz = R(0), pyz = R(0);
            R ax = R(0), ay = R(0), az = R(0);
#pragma unroll
            for (int i = 1; i < St::Q; i += 2) {  // opp(i) = i + 1
                const R cu = cdotu<St>(i, m.ux, m.uy, m.uz);
                const R a = a0 + rho45 * cu * cu, b = rho3 * cu;
                feq[i] = R(St::w(i)) * (a + b);
                feq[i + 1] = R(St::w(i)) * (a - b);
                const R di = f[i] - feq[i], dj = f[i + 1] - feq[i + 1];
                const R sp = di + dj;
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                if (cx) pxx += sp;
                if (cy) pyy += sp;
                if (St::D == 3 && cz) pzz += sp;
                if (cx && cy) pxy += (cx == cy) ? sp : -sp;
                if (St::D == 3 && cx && cz) pxz += (cx == cz) ? sp : -sp;
                if (St::D == 3 && cy && cz) pyz += (cy == cz) ? sp : -sp;
                if constexpr (FORCE) {
                    const R sm = di - dj;
                    if (cx) ax += cx > 0 ? sm : -sm;
                    if (cy) ay += cy > 0 ? sm : -sm;
                    if (St::D == 3 && cz) az += cz > 0 ? sm : -sm;
                }
            }
            const R tr = pxx + pyy + pzz;
            const R relax = R(1) - omega;
            {
                R v = feq[0] + relax * R(St::w(0)) * (R(4.5) * (-tr * R(1.0 / 3.0)));
                if constexpr (FORCE) v += guo_source<St>(0, m, F, pre);
                f[0] = v;
            }
#pragma unroll
            for (int i = 1; i < St::Q; i += 2) {
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                // (c c - cs2 I) : Pi
                R qp = -tr * R(1.0 / 3.0);
                if (cx) qp += pxx;
                if (cy) qp += pyy;
                if (St::D == 3 && cz) qp += pzz;
                if (cx && cy) qp += (cx == cy) ? R(2) * pxy : R(-2) * pxy;
                if (St::D == 3 && cx && cz) qp += (cx == cz) ? R(2) * pxz : R(-2) * pxz;
                if (St::D == 3 && cy && cz) qp += (cy == cz) ? R(2) * pyz : R(-2) * pyz;
                const R e = R(4.5) * qp;
                R o = R(0);
                if constexpr (FORCE) o = R(3) * cdotu<St>(i, ax, ay, az);
                const R rw = relax * R(St::w(i));
                R vi = feq[i] + rw * (e + o), vj = feq[i + 1] + rw * (e - o);
                if constexpr (FORCE) {
                    vi += guo_source<St>(i, m, F, pre);
                    vj += guo_source<St>(i + 1, m, F, pre);
                }
                f[i] = vi;
                f[i + 1] = vj;
            }
        }
        return m.rho > R(0) && m.rho < R(1e30);
    }
}

}  // namespace lb
