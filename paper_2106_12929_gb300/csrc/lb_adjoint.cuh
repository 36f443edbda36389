// Transposed per-node collision Jacobian (the discrete adjoint of one collision),
// for BGK, regularized and streaming-only steps with an optional Guo force.
//
// Forward node map (see lb_collide.cuh): rho = sum f, u = (sum c f + F/2)/rho,
//   BGK: f*_i = (1 - w) f_i + w f^eq_i(rho, u) + S_i(u, F)
//   REG: f*_i = f^eq_i + (1 - w) w_i [3 c_i.a1 + 4.5 (c_i c_i - I/3):Pi] + S_i
//        with Pi = sum_k c_k c_k f_k - rho u u - rho I/3 and a1 = -F/2.
// Given mu = dL/df*, this returns lambda = (df*/df)^T mu and the force part
// (df*/dF)^T mu, by the chain rule through (rho, u):
//   d rho / d f_j = 1,  d u / d f_j = (c_j - u)/rho,  d u / dF = 1/(2 rho).
#pragma once

#include "lb_collide.cuh"

namespace lb {

template <class St, int COLL, bool FORCE, class R>
LB_DEV void adjoint_node(const R* f, const R* F, R* mu, R omega, R* gF)
{
    gF[0] = gF[1] = gF[2] = R(0);
    if constexpr (COLL == NONE) {
        return;
    } else {
        NodeMoments<St, R> m = node_moments<St, FORCE>(f, F);
        const R ux = m.ux, uy = m.uy, uz = m.uz, rho = m.rho;
        const R base = R(1) - R(1.5) * (ux * ux + uy * uy + uz * uz);
        // cotangents of rho and u collected from every path except d rho/df, du/df
        R grho = R(0), gux = R(0), guy = R(0), guz = R(0);
        R lam[St::Q];
        // equilibrium part: scale e = omega for BGK, 1 for REG
        const R e = (COLL == BGK) ? omega : R(1);
        R smw = R(0), smwcx = R(0), smwcy = R(0), smwcz = R(0);  // sum mu w, sum mu w c
        R smwcucx = R(0), smwcucy = R(0), smwcucz = R(0);        // sum mu w (c.u) c
#pragma unroll
        for (int i = 0; i < St::Q; ++i) {
            const R mw = mu[i] * R(St::w(i));
            const R cu = cdotu<St>(i, ux, uy, uz);
            grho += mw * (base + cu * (R(3) + R(4.5) * cu));
            smw += mw;
            smwcx += St::c(i, 0) * mw;
            smwcy += St::c(i, 1) * mw;
            if (St::D == 3) smwcz += St::c(i, 2) * mw;
            smwcucx += St::c(i, 0) * mw * cu;
            smwcucy += St::c(i, 1) * mw * cu;
            if (St::D == 3) smwcucz += St::c(i, 2) * mw * cu;
        }
        // d f^eq_i / d u = w_i rho (3 c_i + 9 (c_i.u) c_i - 3 u)
        grho *= e;
        gux = e * rho * (R(3) * smwcx + R(9) * smwcucx - R(3) * ux * smw);
        guy = e * rho * (R(3) * smwcy + R(9) * smwcucy - R(3) * uy * smw);
        guz = e * rho * (R(3) * smwcz + R(9) * smwcucz - R(3) * uz * smw);
        R gFx = R(0), gFy = R(0), gFz = R(0);

        if constexpr (COLL == BGK) {
#pragma unroll
            for (int i = 0; i < St::Q; ++i) lam[i] = (R(1) - omega) * mu[i];
        } else {  // REG
            // G = 4.5 (1 - w) sum_i mu_i w_i (c_i c_i - I/3): cotangent of Pi
            const R k = R(4.5) * (R(1) - omega);
            R sxx = R(0), syy = R(0), szz = R(0), sxy = R(0), sxz = R(0), syz = R(0);
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                const R mw = mu[i] * R(St::w(i));
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                if (cx) sxx += mw;
                if (cy) syy += mw;
                if (St::D == 3 && cz) szz += mw;
                if (cx && cy) sxy += (cx == cy) ? mw : -mw;
                if (St::D == 3 && cx && cz) sxz += (cx == cz) ? mw : -mw;
                if (St::D == 3 && cy && cz) syz += (cy == cz) ? mw : -mw;
            }
            const R third = R(1.0 / 3.0);
            const R Gxx = k * (sxx - third * smw), Gyy = k * (syy - third * smw);
            const R Gzz = St::D == 3 ? k * (szz - third * smw) : R(0);
            const R Gxy = k * sxy, Gxz = k * sxz, Gyz = k * syz;
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                const int cx = St::c(i, 0), cy = St::c(i, 1), cz = St::c(i, 2);
                R cgc = R(0);
                if (cx) cgc += Gxx;
                if (cy) cgc += Gyy;
                if (St::D == 3 && cz) cgc += Gzz;
                if (cx && cy) cgc += (cx == cy) ? R(2) * Gxy : R(-2) * Gxy;
                if (St::D == 3 && cx && cz) cgc += (cx == cz) ? R(2) * Gxz : R(-2) * Gxz;
                if (St::D == 3 && cy && cz) cgc += (cy == cz) ? R(2) * Gyz : R(-2) * Gyz;
                lam[i] = cgc;
            }
            // Pi depends on rho and u through - rho u u - rho I/3
            const R Gux = Gxx * ux + Gxy * uy + Gxz * uz;
            const R Guy = Gxy * ux + Gyy * uy + Gyz * uz;
            const R Guz = Gxz * ux + Gyz * uy + Gzz * uz;
            grho -= ux * Gux + uy * Guy + uz * Guz + third * (Gxx + Gyy + Gzz);
            gux -= R(2) * rho * Gux;
            guy -= R(2) * rho * Guy;
            guz -= R(2) * rho * Guz;
            if constexpr (FORCE) {
                // a1 = -F/2 with cotangent A = 3 (1 - w) sum mu w c
                const R k1 = R(-0.5) * R(3) * (R(1) - omega);
                gFx += k1 * smwcx;
                gFy += k1 * smwcy;
                gFz += k1 * smwcz;
            }
        }
        if constexpr (FORCE) {
            // S_i = p w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)], p = 1 - w/2
            const R p = R(1) - R(0.5) * omega;
            const R Fx = F[0], Fy = F[1], Fz = F[2];
            R smwcF = R(0);                                // sum mu w (c.F)
            R smwcFcx = R(0), smwcFcy = R(0), smwcFcz = R(0);  // sum mu w (c.F) c
#pragma unroll
            for (int i = 0; i < St::Q; ++i) {
                const R mw = mu[i] * R(St::w(i));
                const R cF = cdotu<St>(i, Fx, Fy, Fz);
                smwcF += mw * cF;
                smwcFcx += St::c(i, 0) * mw * cF;
                smwcFcy += St::c(i, 1) * mw * cF;
                if (St::D == 3) smwcFcz += St::c(i, 2) * mw * cF;
            }
            // dS/du = p w (-3 F + 9 (c.F) c);  dS/dF = p w (3 (c - u) + 9 (c.u) c)
            gux += p * (R(-3) * Fx * smw + R(9) * smwcFcx);
            guy += p * (R(-3) * Fy * smw + R(9) * smwcFcy);
            guz += p * (R(-3) * Fz * smw + R(9) * smwcFcz);
            gFx += p * (R(3) * (smwcx - ux * smw) + R(9) * smwcucx);
            gFy += p * (R(3) * (smwcy - uy * smw) + R(9) * smwcucy);
            gFz += p * (R(3) * (smwcz - uz * smw) + R(9) * smwcucz);
            (void)smwcF;
        }
        const R inv = R(1) / rho;
        const R gdotu = gux * ux + guy * uy + guz * uz;
#pragma unroll
        for (int i = 0; i < St::Q; ++i) mu[i] = lam[i] + grho + (cdotu<St>(i, gux, guy, guz) - gdotu) * inv;
        if constexpr (FORCE) {
            gF[0] = gFx + R(0.5) * gux * inv;
            gF[1] = gFy + R(0.5) * guy * inv;
            gF[2] = St::D == 3 ? gFz + R(0.5) * guz * inv : R(0);
        }
    }
}

}  // namespace lb
