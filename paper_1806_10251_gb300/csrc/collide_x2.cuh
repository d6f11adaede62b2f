// The GI-preconditioned cascaded collision for two cells at once (packed FP32).
//
// Same arithmetic as collide_cell in d2q9_collide.cuh (Sec. 5 with the
// extended-equilibrium corrections of Eqs. 45-47 and the strain-rate solve of
// Eqs. 53-55), written with shared subexpressions and explicit fused
// multiply-adds on F2 pairs.  Two identities shorten it:
//   g3 = (omega3/12) (M3 - m3) and g4 = (omega4/4) (M4 - m4),
// where m3, m4 are the second-order non-equilibrium moments the strain solve
// already needs (the equilibrium part of g3, g4 is exactly -m3, -m4).
#pragma once

#include "d2q9_collide.cuh"
#include "f32x2.cuh"

namespace lbm {

__device__ __forceinline__ F2 ld(const float2 &v) { return F2{v.x, v.y}; }

template <int MODE, bool FORCED, bool GUARD = false>
__device__ __forceinline__ void collide_x2(F2 (&g)[9], F2 drx, F2 dry, F2 Fx, F2 Fy, const Consts2 &k,
                                           bool guard, unsigned long long *guard_count)
{
    // conserved and raw moments of gbar (Eq. 3; rho = 1 + sum g)
    const F2 s13 = g[1] + g[3], s24 = g[2] + g[4];
    const F2 s56 = g[5] + g[6], s78 = g[7] + g[8];
    const F2 kxxyy = s56 + s78;
    const F2 kxx = s13 + kxxyy;
    const F2 kyy = s24 + kxxyy;
    const F2 dr = (g[0] + s13) + (s24 + kxxyy);
    const F2 rho = ld(k.one) + dr;
    const F2 irho = recip2(rho, ld(k.one));
    const F2 jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
    const F2 jy = ((g[2] - g[4]) + s56) - s78;
    F2 ux, uy;
    if (FORCED) {
        // rho u = sum fbar e + F/(2 gamma)
        ux = fma2(Fx, ld(k.half_ig), jx) * irho;
        uy = fma2(Fy, ld(k.half_ig), jy) * irho;
    } else {
        ux = jx * irho;
        uy = jy * irho;
    }
    const F2 kxy = (g[5] + g[7]) - (g[6] + g[8]);
    const F2 kxxy = s56 - s78;
    const F2 kxyy = (g[5] + g[8]) - (g[6] + g[7]);
    const F2 ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const F2 nux = neg2(ux), nuy = neg2(uy);
    const F2 m2ux = nux + nux, m2uy = nuy + nuy;  // -2 ux, -2 uy

    // preconditioned source raw moments (list after Eq. 15)
    F2 sxx = f2(0.f), syy = f2(0.f), sxy = f2(0.f), sxxy = f2(0.f), sxyy = f2(0.f), sxxyy = f2(0.f);
    F2 sx = f2(0.f), sy = f2(0.f);
    if (FORCED) {
        const F2 ig = ld(k.ig), ig2 = ld(k.ig2);
        sx = Fx * ig;
        sy = Fy * ig;
        const F2 Fxux = Fx * ux, Fyuy = Fy * uy;
        sxx = (Fxux + Fxux) * ig2;
        syy = (Fyuy + Fyuy) * ig2;
        sxy = fma2(Fx, uy, Fy * ux) * ig2;
        const F2 Fxuxy = Fx * uxy, Fyuxy = Fy * uxy;
        sxxy = fma2(Fy, ux2, Fxuxy + Fxuxy);
        sxyy = fma2(Fx, uy2, Fyuxy + Fyuxy);
        const F2 t = fma2(Fx, ux * uy2, Fy * (uy * ux2));
        sxxyy = t + t;
    }

    // second-order non-equilibrium moments of f = fbar + S/2:
    //   m3 = kxx + kyy - (2/3 dr + rho (ux^2 + uy^2)/gamma), m4 = kxx - kyy - rho (ux^2 - uy^2)/gamma
    const F2 rig = rho * ld(k.ig);
    F2 m3 = (kxx + kyy) - fma2(rig, ux2 + uy2, ld(k.two_thirds) * dr);
    F2 m4 = fnma2(rig, ux2 - uy2, kxx - kyy);
    if (FORCED) {
        m3 = fma2(ld(k.half), sxx + syy, m3);
        m4 = fma2(ld(k.half), sxx - syy, m4);
    }

    // extended-equilibrium corrections (Eq. 33 with Eqs. 45-47)
    F2 M3 = f2(0.f), M4 = f2(0.f), M5 = f2(0.f);
    if (MODE == LBM_GI_FULL) {
        const F2 hA = ld(k.hA), hB = ld(k.hB);
        const F2 t1 = hA * ux2, t2 = hB * uy2, t3 = hA * uy2, t4 = hB * ux2;
        const F2 P = t1 + t2, Pt = t1 - t2, Q = t3 + t4, Qt = t3 - t4;
        // Eq. 53
        F2 c1 = (ld(k.a3) + P) * rho, c2 = (ld(k.a3) + Q) * rho;
        F2 c1t = (ld(k.a4) + Pt) * rho, c2t = (ld(k.a4) + Qt) * rho;
        F2 D = neg2(fma2(c1, c2t, c1t * c2));
        if (GUARD && guard) {
            // per cell: drop the velocity-dependent parts where |D| < 0.1 |D0|
            const F2 a3r = ld(k.a3) * rho, a4r = ld(k.a4) * rho;
            const F2 D0 = ld(k.m_two) * (a3r * a4r);
            const bool gx = fabsf(D.x) < 0.1f * fabsf(D0.x), gy = fabsf(D.y) < 0.1f * fabsf(D0.y);
            if (gx || gy) {
                if (gx) {
                    c1.x = c2.x = a3r.x;
                    c1t.x = c2t.x = a4r.x;
                    if (guard_count) atomicAdd(guard_count, 1ull);
                }
                if (gy) {
                    c1.y = c2.y = a3r.y;
                    c1t.y = c2t.y = a4r.y;
                    if (guard_count) atomicAdd(guard_count, 1ull);
                }
                D = neg2(fma2(c1, c2t, c1t * c2));
            }
        }
        // Eq. 54
        const F2 C3 = ld(k.C3);
        const F2 uxdrx = ux * drx;
        const F2 er = C3 * fma2(uy, dry, uxdrx);
        const F2 ert = C3 * fnma2(uy, dry, uxdrx);
        const F2 R3 = m3 - er, R4 = m4 - ert;
        const F2 iD = recip2(D, ld(k.one));
        // Eq. 55a, and 55b with the c~1 term's sign as the solve of Eqs. 51-52 gives it
        const F2 dux = fma2(c2t, R3, c2 * R4) * iD;
        const F2 duy = fnma2(c1, R4, c1t * R3) * iD;
        // Eqs. 45-47
        M3 = ld(k.k3x2) * (rho * fma2(P, dux, Q * duy) - er);
        M4 = ld(k.k4x2) * (rho * fnma2(Qt, duy, Pt * dux) - ert);
        M5 = ld(k.mk5) * fma2(rho * ld(k.B) * uxy, dux + duy, C3 * fma2(uy, drx, ux * dry));
    }

    // cascaded collision (Sec. 5; Eq. 4 bars and source terms kept)
    const F2 g3 = ld(k.w3_12) * (M3 - m3);
    const F2 g4 = ld(k.w4_4) * (M4 - m4);
    F2 e5 = fma2(rig, uxy, M5 - kxy);  // rho uxy / gamma - kxy + M5
    if (FORCED) e5 = fnma2(ld(k.half), sxy, e5);
    const F2 g5 = ld(k.w5_4) * e5;
    const F2 g3x3 = ld(k.three) * g3;
    const F2 t34p = g3x3 + g4, t34m = g3x3 - g4;
    const F2 c6rho = ld(k.c6) * rho;
    const F2 third = ld(k.third);
    const F2 tkxx = third + kxx, tkyy = third + kyy;
    // g6: third-order xxy
    F2 e6 = fma2(m2ux, kxy, fma2(c6rho * ux2, uy, kxxy));
    e6 = fma2(nuy, tkxx, e6);
    if (FORCED) e6 = fnma2(ld(k.half), sxxy, e6);
    const F2 mhuy = ld(k.half) * nuy, mhux = ld(k.half) * nux;  // -uy/2, -ux/2
    const F2 g6 = fma2(ld(k.w6_4), e6, fma2(mhuy, t34p, m2ux * g5));
    // g7: third-order xyy
    F2 e7 = fma2(m2uy, kxy, fma2(c6rho * uy2, ux, kxyy));
    e7 = fma2(nux, tkyy, e7);
    if (FORCED) e7 = fnma2(ld(k.half), sxyy, e7);
    const F2 g7 = fma2(ld(k.w7_4), e7, fma2(mhux, t34m, m2uy * g5));
    // g8: fourth order
    //   e8 = dr/9 + 3 rho ux^2 uy^2 - (kxxyy - 2 ux kxyy - 2 uy kxxy + ux^2 (1/3 + kyy)
    //        + uy^2 (1/3 + kxx) + 4 uxy kxy) - sxxyy/2
    const F2 inner = fma2(ux2, tkyy, fma2(uy2, tkxx, fma2(m2ux, kxyy, fma2(m2uy, kxxy, kxxyy))));
    const F2 uxy4 = ld(k.four) * uxy;
    F2 e8 = fma2(ld(k.ninth), dr, ld(k.three) * (rho * (ux2 * uy2))) - fma2(uxy4, kxy, inner);
    if (FORCED) e8 = fnma2(ld(k.half), sxxyy, e8);
    F2 g8 = fma2(ld(k.w8_4), e8, ld(k.m_two) * g3);
    g8 = fma2(mhuy * uy, t34p, g8);
    g8 = fma2(mhux * ux, t34m, g8);
    g8 = fnma2(uxy4, g5, g8);
    g8 = fma2(m2uy, g6, g8);
    g8 = fma2(m2ux, g7, g8);

    // f~ = fbar + K g^ (columns: K3 = 3|e^2| - 4, K4 = |ex^2 - ey^2|, K5 = |ex ey|,
    // K6 = -3|ex^2 ey| + 2|ey|, K7 = -3|ex ey^2| + 2|ex|, K8 = 9|ex^2 ey^2| - 6|e^2| + 4)
    const F2 A = fma2(ld(k.two), g8, g3);  // directions 1..4 take -(g3 + 2 g8)
    const F2 b13 = g4 - A, b24 = neg2(g4 + A);
    g[0] = fma2(ld(k.four), g8 - g3, g[0]);
    const F2 g7x2 = g7 + g7, g6x2 = g6 + g6;
    g[1] = g[1] + (b13 + g7x2);
    g[3] = g[3] + (b13 - g7x2);
    g[2] = g[2] + (b24 + g6x2);
    g[4] = g[4] + (b24 - g6x2);
    const F2 h = fma2(ld(k.two), g3, g8);  // directions 5..8
    const F2 hp = h + g5, hm = h - g5, s67 = g6 + g7, d67 = g6 - g7;
    g[5] = g[5] + (hp - s67);
    g[7] = g[7] + (hp + s67);
    g[6] = g[6] + (hm - d67);
    g[8] = g[8] + (hm + d67);

    if (FORCED) {
        // S = T^-1 sigma' (inverse of the Eq. 5 map), sigma'_0 = 0
        const F2 half = ld(k.half), quarter = ld(k.half) * ld(k.half);
        g[0] = g[0] + (sxxyy - (sxx + syy));
        const F2 a13 = sxx - sxxyy, a24 = syy - sxxyy;
        g[1] = fma2(half, (a13 + sx) - sxyy, g[1]);
        g[3] = fma2(half, (a13 - sx) + sxyy, g[3]);
        g[2] = fma2(half, (a24 + sy) - sxxy, g[2]);
        g[4] = fma2(half, (a24 - sy) + sxxy, g[4]);
        const F2 p1 = sxxy + sxyy, p2 = sxxy - sxyy;
        const F2 q1 = sxxyy + sxy, q2 = sxxyy - sxy;
        g[5] = fma2(quarter, q1 + p1, g[5]);
        g[6] = fma2(quarter, q2 + p2, g[6]);
        g[7] = fma2(quarter, q1 - p1, g[7]);
        g[8] = fma2(quarter, q2 - p2, g[8]);
    }
}

}  // namespace lbm
