// D2Q9 lattice, storage conversion and the cascaded central-moment collision of
// the GI preconditioned scheme (Hajabdollahi & Premnath, arXiv 1806.10251),
// written for register-resident evaluation in FP32 (FP64 for the FP64 format).
//
// Populations are handled as deviations g = f - w rho0 (rho0 = 1) from the rest
// state: raw moments of f are then the rest-state moments plus those of g, and
// every O(1) constant cancels analytically before any rounding happens.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace lbm {

// Velocity ordering: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
//                    5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
__host__ __device__ constexpr int cx(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
// opposite directions
__host__ __device__ constexpr int opposite(int a)
{
    return a == 0 ? 0 : a == 1 ? 3 : a == 2 ? 4 : a == 3 ? 1 : a == 4 ? 2 : a == 5 ? 7 : a == 6 ? 8 : a == 7 ? 5 : 6;
}
// lattice weights: 4/9, 1/9 (axis), 1/36 (diagonal)
__host__ __device__ constexpr double weight(int a) { return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// ---- storage conversion ------------------------------------------------------
template <typename ST> struct StorageTraits;
//
// 16-bit types also have store_sr: stochastic rounding of an FP32 value with
// 32 random bits r.  The top (23 - kept mantissa bits) bits of r are added to
// the magnitude's dropped bits and the sum is truncated, so the value rounds
// up with probability equal to its distance from the lower neighbour: the
// rounding error has zero mean whatever the state.  (Round-to-nearest errors
// are a fixed function of the state; in a near-steady flow they act as a
// constant forcing that the slowest viscous modes amplify by about
// 1/(nu k^2).)  Values so small that the 16-bit result is subnormal would
// drop more bits than r covers; FP16 storage is scaled so that only
// |g| < 2^-28 gets there.  (The packed kernels store pairs through the
// hardware's stochastic conversion instead, PairIO in stream_collide_x2.cuh.)
template <> struct StorageTraits<float> {
    using R = float;
    static constexpr bool kReduced = false;
    __device__ static __forceinline__ float load(const float *p) { return __ldg(p); }
    __device__ static __forceinline__ float cvt(float v) { return v; }
    __device__ static __forceinline__ void store(float *p, float v) { *p = v; }
    __device__ static __forceinline__ void store_sr(float *p, float v, uint32_t) { *p = v; }
};
template <> struct StorageTraits<double> {
    using R = double;
    static constexpr bool kReduced = false;
    __device__ static __forceinline__ double load(const double *p) { return __ldg(p); }
    __device__ static __forceinline__ double cvt(double v) { return v; }
    __device__ static __forceinline__ void store(double *p, double v) { *p = v; }
    __device__ static __forceinline__ void store_sr(double *p, double v, uint32_t) { *p = v; }
};
// FP16 value h of F16_SCALE * g -> g in FP32 by one mixed-precision FMA,
// h * 2^-14 + (-0): exact (2^-14 is an FP16 normal and the product of two FP16
// values is exact in FP32), the same value as converting and then scaling.
__device__ __forceinline__ float f16_unscaled(__half h)
{
    static_assert(F16_INV_SCALE == 1.0f / 16384.0f, "the FMA constant below is 2^-14");
    float d;
    asm("{.reg .f16 s; mov.b16 s, 0x0400; fma.rn.f32.f16 %0, %1, s, %2;}"
        : "=f"(d)
        : "h"(__half_as_ushort(h)), "f"(-0.0f));
    return d;
}

template <> struct StorageTraits<__half> {  // holds F16_SCALE * g
    using R = float;
    static constexpr bool kReduced = true;
    __device__ static __forceinline__ float load(const __half *p) { return f16_unscaled(__ldg(p)); }
    __device__ static __forceinline__ float cvt(__half v) { return f16_unscaled(v); }
    __device__ static __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v * F16_SCALE); }
    __device__ static __forceinline__ void store_sr(__half *p, float v, uint32_t r)
    {
        // 13 dropped bits for a normal FP16 result
        *p = __float2half_rz(__uint_as_float(__float_as_uint(v * F16_SCALE) + (r >> 19)));
    }
};
template <> struct StorageTraits<__nv_bfloat16> {
    using R = float;
    static constexpr bool kReduced = true;
    __device__ static __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static __forceinline__ void store_sr(__nv_bfloat16 *p, float v, uint32_t r)
    {
        *p = __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (r >> 16)));  // 16 dropped bits
    }
};

// 32-bit integer hash for the rounding bits: Wellons' "lowbias32"
// xorshift-multiply finaliser (hash-prospector), a bijection on 32 bits.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Per-direction odd multipliers: direction a of a cell takes the top bits of
// h * kSrMul[a], where h = mix32(mix32(step) ^ cell).
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, int a)
{
    constexpr uint32_t m[9] = {0x9e3779b1u, 0x85ebca77u, 0xc2b2ae3du, 0x27d4eb2fu, 0x165667b1u,
                               0xd3a2646du, 0xfd7046c5u, 0xb55a4f09u, 0x1b873593u};
    return h * m[a];
}

// Reciprocal: correctly rounded in FP32 (no IEEE division sequence), exact
// division in FP64.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// One cell: g holds the post-streaming deviations gbar on entry and the
// post-collision deviations on exit (Eq. 2a: f~ = fbar + K g^ + S).
// drx, dry: density gradient (used by the full kernel only).  FORCED selects
// the variant with the preconditioned source terms.
template <typename R, int MODE, bool FORCED>
__device__ __forceinline__ void collide_cell(R (&g)[9], R drx, R dry, R Fx, R Fy, const Consts<R> &c,
                                             bool guard, unsigned long long *guard_count)
{
    constexpr bool forced = FORCED;
    const R third = R(1.0 / 3.0);
    // conserved moments (Eq. 3 on gbar; rho = 1 + sum g)
    const R kxxyy = (g[5] + g[6]) + (g[7] + g[8]);
    const R kxx = (g[1] + g[3]) + kxxyy;
    const R kyy = (g[2] + g[4]) + kxxyy;
    const R dr = g[0] + (g[1] + g[3]) + (g[2] + g[4]) + kxxyy;
    const R rho = R(1) + dr;
    const R irho = recip(rho);
    const R jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const R jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    // velocity with the forcing shift: rho u = sum fbar e + F/(2 gamma)
    const R ux = (jx + Fx * c.half_ig) * irho;
    const R uy = (jy + Fy * c.half_ig) * irho;
    // remaining raw moments of gbar (xy, xxy, xyy)
    const R kxy = (g[5] + g[7]) - (g[6] + g[8]);
    const R kxxy = (g[5] + g[6]) - (g[7] + g[8]);
    const R kxyy = (g[5] + g[8]) - (g[6] + g[7]);

    const R ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;

    // preconditioned source raw moments (list after Eq. 15)
    R sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0, sxxy = 0, sxyy = 0, sxxyy = 0;
    if (forced) {
        sx = Fx * c.ig;
        sy = Fy * c.ig;
        sxx = R(2) * Fx * ux * c.ig2;
        syy = R(2) * Fy * uy * c.ig2;
        sxy = (Fx * uy + Fy * ux) * c.ig2;
        sxxy = Fy * ux2 + R(2) * Fx * uxy;
        sxyy = Fx * uy2 + R(2) * Fy * uxy;
        sxxyy = R(2) * (Fx * ux * uy2 + Fy * uy * ux2);
    }

    // extended-equilibrium corrections (Eq. 33 with Eqs. 45-47)
    R M3 = 0, M4 = 0, M5 = 0;
    if (MODE == LBM_GI_FULL) {
        // second-order non-equilibrium moments of f = fbar + S/2
        const R m3 = (kxx + kyy + R(0.5) * (sxx + syy)) - (R(2.0 / 3.0) * dr + rho * (ux2 + uy2) * c.ig);
        const R m4 = (kxx - kyy + R(0.5) * (sxx - syy)) - rho * (ux2 - uy2) * c.ig;
        const R Aux2 = c.A * ux2, Auy2 = c.A * uy2, Bux2 = c.B * ux2, Buy2 = c.B * uy2;
        const R P = R(-0.5) * (Aux2 + Buy2), Q = R(-0.5) * (Auy2 + Bux2);
        const R Pt = R(-0.5) * (Aux2 - Buy2), Qt = R(-0.5) * (Auy2 - Bux2);
        // Eq. 53
        R c1 = (c.a3 + P) * rho, c2 = (c.a3 + Q) * rho;
        R c1t = (c.a4 + Pt) * rho, c2t = (c.a4 + Qt) * rho;
        R D = -c1 * c2t - c1t * c2;
        if (guard) {
            const R D0 = R(-2) * (c.a3 * rho) * (c.a4 * rho);
            if (fabs(D) < R(0.1) * fabs(D0)) {
                c1 = c2 = c.a3 * rho;
                c1t = c2t = c.a4 * rho;
                D = -c1 * c2t - c1t * c2;
                if (guard_count) atomicAdd(guard_count, 1ull);
            }
        }
        // Eq. 54
        const R er = c.C3 * (ux * drx + uy * dry);
        const R ert = c.C3 * (ux * drx - uy * dry);
        const R R3 = m3 - er, R4 = m4 - ert;
        const R iD = recip(D);
        // Eq. 55a, and 55b with the c~1 term's sign as the solve of Eqs. 51-52 gives it
        const R dux = (c2t * R3 + c2 * R4) * iD;
        const R duy = (c1t * R3 - c1 * R4) * iD;
        // Eq. 45: th3x = 2 k3 rho P, th3y = 2 k3 rho Q, (la3x, la3y) = -(2/3) k3 C (ux, uy)
        M3 = R(2) * c.k3 * (rho * (P * dux + Q * duy) - er);
        // Eq. 46: th4x = 2 k4 rho P~, th4y = 2 k4 rho Q~, (la4x, la4y) = -(2/3) k4 C (ux, uy)
        M4 = R(2) * c.k4 * (rho * (Pt * dux - Qt * duy) - ert);
        // Eq. 47: th5x = th5y = -k5 rho B ux uy, (la5x, la5y) = -(1/3) k5 C (uy, ux)
        M5 = -c.k5 * (rho * c.B * uxy * (dux + duy) + c.C3 * (uy * drx + ux * dry));
    }

    // cascaded collision (Sec. 5; Eq. 4 bars and source terms kept)
    const R g3 = c.w3_12 * (R(2.0 / 3.0) * dr + rho * (ux2 + uy2) * c.ig - (kxx + kyy)
                            - R(0.5) * (sxx + syy) + M3);
    const R g4 = c.w4_4 * (rho * (ux2 - uy2) * c.ig - (kxx - kyy) - R(0.5) * (sxx - syy) + M4);
    const R g5 = c.w5_4 * (rho * uxy * c.ig - kxy - R(0.5) * sxy + M5);
    const R t34p = R(3) * g3 + g4, t34m = R(3) * g3 - g4;
    const R g6 = c.w6_4 * (c.c6 * rho * ux2 * uy + kxxy - R(2) * ux * kxy - uy * (third + kxx) - R(0.5) * sxxy)
               - R(0.5) * uy * t34p - R(2) * ux * g5;
    const R g7 = c.w7_4 * (c.c6 * rho * ux * uy2 + kxyy - R(2) * uy * kxy - ux * (third + kyy) - R(0.5) * sxyy)
               - R(0.5) * ux * t34m - R(2) * uy * g5;
    const R g8 = c.w8_4 * (dr * R(1.0 / 9.0) + R(3) * rho * ux2 * uy2
                           - (kxxyy - R(2) * ux * kxyy - R(2) * uy * kxxy + ux2 * (third + kyy)
                              + uy2 * (third + kxx) + R(4) * uxy * kxy)
                           - R(0.5) * sxxyy)
               - R(2) * g3 - R(0.5) * uy2 * t34p - R(0.5) * ux2 * t34m - R(4) * uxy * g5
               - R(2) * uy * g6 - R(2) * ux * g7;

    // f~ = fbar + K g^ (columns: K3 = 3|e^2| - 4, K4 = |ex^2 - ey^2|, K5 = |ex ey|,
    // K6 = -3|ex^2 ey| + 2|ey|, K7 = -3|ex ey^2| + 2|ex|, K8 = 9|ex^2 ey^2| - 6|e^2| + 4)
    const R a14 = -(g3 + R(2) * g8);  // common to directions 1..4
    const R b13 = a14 + g4, b24 = a14 - g4;
    g[0] += R(4) * (g8 - g3);
    g[1] += b13 + R(2) * g7;
    g[3] += b13 - R(2) * g7;
    g[2] += b24 + R(2) * g6;
    g[4] += b24 - R(2) * g6;
    const R h = R(2) * g3 + g8;       // common to directions 5..8
    const R hp = h + g5, hm = h - g5, s67 = g6 + g7, d67 = g6 - g7;
    g[5] += hp - s67;
    g[7] += hp + s67;
    g[6] += hm - d67;
    g[8] += hm + d67;

    if (forced) {
        // S = T^-1 sigma' (inverse of the Eq. 5 map), sigma'_0 = 0
        g[0] += -sxx - syy + sxxyy;
        g[1] += R(0.5) * (sx + sxx - sxyy - sxxyy);
        g[3] += R(0.5) * (-sx + sxx + sxyy - sxxyy);
        g[2] += R(0.5) * (sy + syy - sxxy - sxxyy);
        g[4] += R(0.5) * (-sy + syy + sxxy - sxxyy);
        g[5] += R(0.25) * (sxy + sxxy + sxyy + sxxyy);
        g[6] += R(0.25) * (-sxy + sxxy - sxyy + sxxyy);
        g[7] += R(0.25) * (sxy - sxxy - sxyy + sxxyy);
        g[8] += R(0.25) * (-sxy - sxxy + sxyy + sxxyy);
    }
}

}  // namespace lbm
