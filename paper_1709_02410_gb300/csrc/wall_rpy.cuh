// Device pair block of the wall-corrected RPY blob mobility.
//
// For a target blob at (xi, yi, zi) and a source blob at (xj, yj, zj), with
// heights already clamped to z >= a (the wall-overlap reading), returns
// 8 pi eta times the 3x3 block M_ij = M_RPY(d) + M_wall:
//
//   free-space RPY (Sec. 2.1):  d = r_i - r_j, r = |d|
//     r >= 2a:  (1/r) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) d d^T / r^2]
//     0<r<2a:   (4/(3a)) [(1 - 9r/(32a)) I + 3 d d^T / (32 a r)]
//     r = 0:    (4/(3a)) I                      (self block, Stokes drag)
//
//   wall (Rotne-Prager-Blake, used in Sec. 4): image vector
//   R = (dx, dy, zi + zj), e = R/|R|, t = zj/|R|, s = a/|R|:
//     M_wall = (1/|R|) [A I + B e e^T + C e z^T + D z e^T + E z z^T]
//     A = -1 - 2 e_z t + 2 t^2 + s^2 (2 e_z^2 - 2/3) + s^4 (2/3 - 10/3 e_z^2)
//     B = -1 + 6 e_z t - 6 t^2 + s^2 (2 - 10 e_z^2) + s^4 (70/3 e_z^2 - 10/3)
//     C = t (2 - 12 e_z^2) + 12 e_z t^2 + e_z s^2 (20 e_z^2 - 4)
//         + e_z s^4 (40/3 - 140/3 e_z^2)
//     D = 2 t - 20/3 e_z s^4
//     E = -4 t^2 - 4 e_z^2 s^2 + s^4 (20 e_z^2 - 8/3)
//   This is Blake's image system for a point force with the RPY (Faxen)
//   regularisation (1 + a^2/6 Lap) applied at both blobs, reduced by hand to
//   the five scalar coefficients above.
//
// Because R and d share their x, y components, the block assembles as
//   Mxx = alpha + beta dx^2, Mxy = Myx = beta dx dy, Myy = alpha + beta dy^2,
//   Mxz = dx gx, Myz = dy gx, Mzx = dx gz, Mzy = dy gz,
//   Mzz = alpha + c2 dz^2 + b3 Rz^2 + (C + D) Rz/|R|^2 + E/|R|,
// with alpha = c1 + A/|R|, b3 = B/|R|^3, beta = c2 + b3,
//   gx = c2 dz + b3 Rz + C/|R|^2, gz = c2 dz + b3 Rz + D/|R|^2
// (c1, c2: the free-space coefficients of I and d d^T).
//
// Evaluated form.  With w = 1/|R|^2, s^2 = a^2 w, e_z^2 = Rz^2 w and
//   x1 = zi zj w + s^2/3,  x2 = s^2 (e_z^2 + s^2/3),  x3 = s^4 e_z^2,
// expanding A..E in powers of w gives (dz = zi - zj, Rz = zi + zj)
//   A = -1 - 2 x1 + 2 x2 - 10/3 x3,   B = -1 + 6 x1 - 10 x2 + 70/3 x3,
//   B Rz + C |R| = -dz + Rz P,  B Rz + D |R| = -dz - Rz P,
//     P = 20/3 s^4 - (B + 1),
//   B Rz^2 + (C + D) Rz |R| + E |R|^2 = -dz^2 + |R|^2 Z,
//     Z = 20 x3 - 4 x2 - 4/3 s^4 - e_z^2 (B + 1),
// so with v = 1/|R|^3:
//   alpha = c1 + A/|R|,  beta = c2 + v B,  gx, gz = dz (c2 - v) +- v Rz P,
//   Mzz = alpha + dz^2 (c2 - v) + Z/|R|.
// Every intermediate is O(1) (s^2 <= 1/4, e_z^2 <= 1 once heights are >= a),
// so the regrouping costs no accuracy in FP32.
#pragma once

#include <cuda_runtime.h>

namespace rpbd {

// Geometry constants of one launch (blob radius a).
template <class R>
struct PairConst {
    R a2;        // a^2
    R a23;       // 2 a^2 / 3
    R two_a2;    // 2 a^2
    R four_a2;   // 4 a^2
    R k_self;    // 4 / (3 a)
    R k_ovl;     // 3 / (8 a^2)
    R inv8a2;    // 1 / (8 a^2)
    R Lx, Ly;    // pseudo-periodic cell (used by pair_block_images only)
    R iLx, iLy;  // 1 / Lx, 1 / Ly
    __host__ __device__ static PairConst make(double a, double Lx = 0.0, double Ly = 0.0)
    {
        PairConst c;
        c.Lx = R(Lx);
        c.Ly = R(Ly);
        c.iLx = R(Lx > 0.0 ? 1.0 / Lx : 0.0);
        c.iLy = R(Ly > 0.0 ? 1.0 / Ly : 0.0);
        c.a2 = R(a * a);
        c.a23 = R(2.0 * a * a / 3.0);
        c.two_a2 = R(2.0 * a * a);
        c.four_a2 = R(4.0 * a * a);
        c.k_self = R(4.0 / (3.0 * a));
        c.k_ovl = R(3.0 / (8.0 * a * a));
        c.inv8a2 = R(1.0 / (8.0 * a * a));
        return c;
    }
};

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float val_(float x) { return x; }
__device__ __forceinline__ double val_(double x) { return x; }

// The five scalars that determine the block (8 pi eta times M_ij):
//   M = [[alpha + beta dx^2, beta dx dy, dx gx], [beta dx dy, alpha + beta dy^2, dy gx],
//        [dx gz, dy gz, Mzz]].
// T is float, double or a dual number; K is the plain scalar type of the
// constants.
template <class T, class K, bool WALL>
__device__ __forceinline__ void pair_factors(T dx, T dy, T dz, T zi, T zj, const PairConst<K>& c, T& alpha, T& beta,
                                             T& gx, T& gz, T& Mzz)
{
    T rho2 = dx * dx + dy * dy;
    T r2 = rho2 + dz * dz;
    T rinv = rsqrt_(r2);
    T rinv2 = rinv * rinv;
    // far branch
    T c1 = rinv * (K(1) + c.a23 * rinv2);
    T c2 = rinv * rinv2 * (K(1) - c.two_a2 * rinv2);
    // overlapping pair (r < 2a) or self block (r = 0): rare, so a branch
    // rather than selects on every pair
    if (val_(r2) < val_(c.four_a2)) {
        if (val_(r2) > K(0)) {
            T rr = r2 * rinv;
            c1 = c.k_self - c.k_ovl * rr;
            c2 = rinv * c.inv8a2;
        } else {
            c1 = T(c.k_self);
            c2 = T(K(0));
        }
    }
    if (!WALL) {
        alpha = c1;
        beta = c2;
        gx = c2 * dz;
        gz = gx;
        Mzz = c1 + c2 * dz * dz;
        return;
    }
    // wall part in the reduced variables (see the header comment)
    T Rz = zi + zj;
    T q = Rz * Rz;
    T Rinv = rsqrt_(rho2 + q);
    T w = Rinv * Rinv;
    T v = Rinv * w;
    T sg = c.a2 * w;  // s^2
    T sg2 = sg * sg;  // s^4
    T y = q * w;      // e_z^2
    T x1 = zi * zj * w + K(1.0 / 3.0) * sg;
    T x2 = sg * (y + K(1.0 / 3.0) * sg);
    T x3 = sg2 * y;
    T Ap = K(2) * (x2 - x1) - K(10.0 / 3.0) * x3;       // A + 1
    T Bp = K(6) * x1 - K(10) * x2 + K(70.0 / 3.0) * x3;  // B + 1
    T P = K(20.0 / 3.0) * sg2 - Bp;
    T Zd = K(20) * x3 - K(4) * x2 - K(4.0 / 3.0) * sg2 - y * Bp;
    alpha = c1 + Rinv * (Ap - K(1));
    T c2v = c2 - v;
    beta = c2v + v * Bp;
    T base = dz * c2v;
    T vRP = v * Rz * P;
    gx = base + vRP;
    gz = base - vRP;
    Mzz = alpha + dz * base + Rinv * Zd;
}

// Block entries, 8 pi eta times M_ij (Mxy = Myx).
template <class T, class K, bool WALL>
__device__ __forceinline__ void pair_block(T dx, T dy, T dz, T zi, T zj, const PairConst<K>& c,
                                           T& Mxx, T& Mxy, T& Mxz, T& Myy, T& Myz, T& Mzx,
                                           T& Mzy, T& Mzz)
{
    T alpha, beta, gx, gz;
    pair_factors<T, K, WALL>(dx, dy, dz, zi, zj, c, alpha, beta, gx, gz, Mzz);
    Mxx = alpha + beta * dx * dx;
    Mxy = beta * dx * dy;
    Myy = alpha + beta * dy * dy;
    Mxz = dx * gx;
    Myz = dy * gx;
    Mzx = dx * gz;
    Mzy = dy * gz;
}

__device__ __forceinline__ float rint_(float x) { return rintf(x); }
__device__ __forceinline__ double rint_(double x) { return rint(x); }

// Pseudo-periodic pair block (Sec. 4.2): the separation is reduced to the
// minimum image in x and y, and that image plus its 8 nearest periodic
// images are summed.  PER = false is the plain block.  The self block arises
// from the unshifted image of i = j (zero separation).
template <class T, class K, bool WALL, bool PER>
__device__ __forceinline__ void pair_block_images(T dx, T dy, T dz, T zi, T zj, const PairConst<K>& c, T& Mxx, T& Mxy,
                                                  T& Mxz, T& Myy, T& Myz, T& Mzx, T& Mzy, T& Mzz)
{
    if (!PER) {
        pair_block<T, K, WALL>(dx, dy, dz, zi, zj, c, Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz);
        return;
    }
    dx = dx - c.Lx * K(rint_(val_(dx) * c.iLx));
    dy = dy - c.Ly * K(rint_(val_(dy) * c.iLy));
    Mxx = Mxy = Mxz = Myy = Myz = Mzx = Mzy = Mzz = T(K(0));
#pragma unroll
    for (int a = -1; a <= 1; ++a) {
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
            T xx, xy, xz, yy, yz, zx, zy, zz;
            pair_block<T, K, WALL>(dx + K(a) * c.Lx, dy + K(b) * c.Ly, dz, zi, zj, c, xx, xy, xz, yy, yz, zx, zy, zz);
            Mxx = Mxx + xx; Mxy = Mxy + xy; Mxz = Mxz + xz; Myy = Myy + yy;
            Myz = Myz + yz; Mzx = Mzx + zx; Mzy = Mzy + zy; Mzz = Mzz + zz;
        }
    }
}

// Forward-mode dual number with NP partials (device), scalar S (float or double).
template <int NP, class S = double>
struct Dual {
    S v;
    S g[NP];
    __device__ Dual() {}
    __device__ Dual(S x) : v(x)
    {
#pragma unroll
        for (int q = 0; q < NP; ++q) g[q] = S(0);
    }
};
template <int NP, class S>
__device__ __forceinline__ S val_(const Dual<NP, S>& x) { return x.v; }
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator+(const Dual<NP, S>& a, const Dual<NP, S>& b)
{
    Dual<NP, S> r; r.v = a.v + b.v;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = a.g[q] + b.g[q];
    return r;
}
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator-(const Dual<NP, S>& a, const Dual<NP, S>& b)
{
    Dual<NP, S> r; r.v = a.v - b.v;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = a.g[q] - b.g[q];
    return r;
}
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator*(const Dual<NP, S>& a, const Dual<NP, S>& b)
{
    Dual<NP, S> r; r.v = a.v * b.v;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = fma(a.g[q], b.v, a.v * b.g[q]);
    return r;
}
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator+(const Dual<NP, S>& a, S b) { Dual<NP, S> r = a; r.v += b; return r; }
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator+(S b, const Dual<NP, S>& a) { Dual<NP, S> r = a; r.v += b; return r; }
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator-(const Dual<NP, S>& a, S b) { Dual<NP, S> r = a; r.v -= b; return r; }
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator-(S b, const Dual<NP, S>& a)
{
    Dual<NP, S> r; r.v = b - a.v;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = -a.g[q];
    return r;
}
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator*(const Dual<NP, S>& a, S b)
{
    Dual<NP, S> r; r.v = a.v * b;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = a.g[q] * b;
    return r;
}
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> operator*(S b, const Dual<NP, S>& a) { return a * b; }
template <int NP, class S>
__device__ __forceinline__ Dual<NP, S> rsqrt_(const Dual<NP, S>& a)
{
    Dual<NP, S> r; r.v = rsqrt_(a.v);
    const S d = S(-0.5) * r.v * r.v * r.v;
#pragma unroll
    for (int q = 0; q < NP; ++q) r.g[q] = d * a.g[q];
    return r;
}

}  // namespace rpbd
