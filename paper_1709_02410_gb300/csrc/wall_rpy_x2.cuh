// Two wall-RPY pair blocks at once in packed two-wide FP32 arithmetic.
//
// The same five block scalars as pair_factors in wall_rpy.cuh (free-space
// c1, c2 and the wall part in the reduced variables s^2, e_z^2,
// zi zj/|R|^2), for two pairs held in the .x and .y lanes of float2 values,
// so every add / multiply / FMA is one packed instruction for both pairs.
// Used by the symmetric kernel, which gives each thread two home blobs
// against the same visitor; lengths in units of a.  Only the open cell with
// the wall is covered (the default path); overlapping pairs (r < 2a) and
// self pairs take a scalar branch per lane, as in the one-pair form.
#pragma once

#include <cuda_runtime.h>

#include "wall_rpy.cuh"

namespace rpbd {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Constants of the packed form, each duplicated into both lanes.  Lengths
// are in units of the blob radius (a = 1): the block is homogeneous of degree
// -1 in length, so the caller scales positions by 1/a and the result by 1/a.
struct PairConstX2 {
    float2 a23, m2a2, one, third, m1;
    float four_a2, k_self, k_ovl, inv8a2;
    __device__ static PairConstX2 make_unit()
    {
        PairConstX2 p;
        p.a23 = bc2(2.0f / 3.0f);
        p.m2a2 = bc2(-2.0f);
        p.one = bc2(1.0f);
        p.third = bc2(1.0f / 3.0f);
        p.m1 = bc2(-1.0f);
        p.four_a2 = 4.0f;
        p.k_self = 4.0f / 3.0f;
        p.k_ovl = 3.0f / 8.0f;
        p.inv8a2 = 1.0f / 8.0f;
        return p;
    }
};

// free-space coefficients of one lane in the rare overlapping / self case
__device__ __forceinline__ void overlap_fix(float r2, float rinv, const PairConstX2& c, float& c1, float& c2)
{
    if (r2 < c.four_a2) {
        if (r2 > 0.0f) {
            c1 = c.k_self - c.k_ovl * (r2 * rinv);
            c2 = rinv * c.inv8a2;
        } else {
            c1 = c.k_self;
            c2 = 0.0f;
        }
    }
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha, beta, gx, gz, Mzz of two pairs (see pair_factors for the formulas).
// With a = 1 the wall scalars are polynomials in w = 1/|R|^2, y = e_z^2 and
// u = zi zj, regrouped in Horner form around shared factors:
//   B + 1 = w h1,               h1 = (6u + 2 - 10y) + w (70/3 y - 10/3)
//   A     = -1 + w (2y - 2u - 2/3 + w (2/3 - 10/3 y))
//   -P    = (B + 1) - 20/3 w^2
//   Z     = w (y (20w - 4 - h1) - 8/3 w)
// so Rinv A and Rinv Z become v (...) with v = Rinv w, and no term is formed
// twice.  zi6 = 6 zi and m2zi = -2 zi depend on the target only.
//
// FAR = true: the direct and image terms are combined without cancellation.
// Far from the target (|d| >> z) the free-space coefficients c1 ~ 1/r and
// c2 ~ 1/r^3 and their image counterparts 1/|R|, 1/|R|^3 agree in their
// leading digits while the block itself is only O(zi zj / |R|^3), so the
// default form loses FP32 digits in proportion to |R|^2 / (zi zj) (a block at
// 700 a carries a relative error of ~1e-3; the matvec's rows barely notice,
// since such blocks are tiny).  With |R|^2 - r^2 = 4 zi zj exactly,
//   1/r - 1/R     = 4 zi zj / (r R (r + R)),
//   1/r^3 - 1/R^3 = (1/r - 1/R) (1/r^2 + 1/(r R) + 1/R^2),
// so c1 - 1/R and c2 - 1/R^3 are formed from these differences and every
// block keeps FP32 relative accuracy at any distance, for ~8 more packed
// operations and one reciprocal per pair.
template <bool FAR = false>
__device__ __forceinline__ void pair_factors_x2(float2 dx, float2 dy, float2 dz, float2 zi, float2 zj,
                                                const PairConstX2& c, float2& alpha, float2& beta, float2& gx,
                                                float2& gz, float2& Mzz)
{
    const float2 rho2 = fma2(dy, dy, mul2(dx, dx));
    const float2 r2 = fma2(dz, dz, rho2);
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 rinv2 = mul2(rinv, rinv);
    const float2 rinv3 = mul2(rinv, rinv2);
    const float2 zi6 = mul2(bc2(6.0f), zi);
    const float2 m2zi = mul2(bc2(-2.0f), zi);
    // wall part
    const float2 Rz = add2(zi, zj);
    const float2 q = mul2(Rz, Rz);
    const float2 R2 = add2(rho2, q);
    const float2 Rinv = make_float2(rsqrtf(R2.x), rsqrtf(R2.y));
    const float2 w = mul2(Rinv, Rinv);
    const float2 v = mul2(Rinv, w);
    float2 X1, c2v;  // c1 - 1/R and c2 - 1/R^3
    if constexpr (FAR) {
        const float2 rR = mul2(rinv, Rinv);
        const float2 sR = fma2(r2, rinv, mul2(R2, Rinv));  // r + R
        const float2 isR = make_float2(rcp_approx(sR.x), rcp_approx(sR.y));
        const float2 D1 = mul2(mul2(mul2(mul2(bc2(4.0f), zi), zj), rR), isR);
        const float2 D3 = mul2(D1, add2(add2(rinv2, w), rR));
        X1 = fma2(c.a23, rinv3, D1);
        c2v = fma2(c.m2a2, mul2(rinv3, rinv2), D3);
        if (r2.x < c.four_a2 || r2.y < c.four_a2) {
            // overlapping or self pairs: the plain coefficients (no cancellation here)
            if (r2.x < c.four_a2) {
                float c1x = 0.0f, c2x = 0.0f;
                overlap_fix(r2.x, rinv.x, c, c1x, c2x);
                X1.x = c1x - Rinv.x;
                c2v.x = c2x - v.x;
            }
            if (r2.y < c.four_a2) {
                float c1y = 0.0f, c2y = 0.0f;
                overlap_fix(r2.y, rinv.y, c, c1y, c2y);
                X1.y = c1y - Rinv.y;
                c2v.y = c2y - v.y;
            }
        }
    } else {
        float2 c1 = fma2(c.a23, rinv3, rinv);
        float2 c2 = mul2(rinv3, fma2(c.m2a2, rinv2, c.one));
        if (r2.x < c.four_a2 || r2.y < c.four_a2) {
            overlap_fix(r2.x, rinv.x, c, c1.x, c2.x);
            overlap_fix(r2.y, rinv.y, c, c1.y, c2.y);
        }
        X1 = fma2(c.m1, Rinv, c1);
        c2v = fma2(c.m1, v, c2);
    }
    const float2 y = mul2(q, w);  // e_z^2
    const float2 a1 = fma2(bc2(-10.0f), y, fma2(zi6, zj, bc2(2.0f)));
    const float2 b1 = fma2(bc2(70.0f / 3.0f), y, bc2(-10.0f / 3.0f));
    const float2 eA = fma2(m2zi, zj, fma2(bc2(2.0f), y, bc2(-2.0f / 3.0f)));
    const float2 b2 = fma2(bc2(-10.0f / 3.0f), y, c.a23);
    const float2 h1 = fma2(w, b1, a1);
    const float2 iA = fma2(w, b2, eA);
    const float2 Bp = mul2(w, h1);  // B + 1
    const float2 w2 = mul2(w, bc2(-20.0f / 3.0f));
    const float2 tz = fma2(bc2(20.0f), w, fma2(c.m1, h1, bc2(-4.0f)));
    beta = fma2(v, Bp, c2v);
    alpha = fma2(v, iA, X1);
    const float2 vR = mul2(v, Rz);
    const float2 Pn = fma2(w2, w, Bp);  // -P
    const float2 base = mul2(dz, c2v);
    const float2 vRPn = mul2(vR, Pn);
    const float2 iZ = fma2(y, tz, mul2(bc2(-8.0f / 3.0f), w));
    gx = fma2(c.m1, vRPn, base);
    gz = add2(base, vRPn);
    Mzz = fma2(v, iZ, fma2(dz, base, alpha));
}

}  // namespace rpbd
