/*
 * CPU FP64 oracle for the wall-corrected RPY blob mobility.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * What it computes (FP64, plain loops, OpenMP over target blobs):
 *
 *   M_ij = s_i s_j [ M_RPY(r~_i - r~_j) + M_wall(r~_i, r~_j) ]          (Sec. 2.1)
 *
 *   - M_RPY: the free-space Rotne-Prager-Yamakawa block for two blobs of
 *     hydrodynamic radius a (cited in Sec. 2.1; textbook form, written by
 *     hand below).  The self block i = j is the Stokes drag 1/(6 pi eta a) I.
 *   - M_wall: Faxen-regularised Blake image system for a no-slip wall at
 *     z = 0 (the Rotne-Prager-Blake tensor used in Sec. 4), generated
 *     symbolically by derive_rpb.py into rpb_generated.h.
 *   - Wall-overlap regularisation (Sec. 4 keeps M SPD when blobs overlap the
 *     wall but prints no rule).  Reading used here:
 *       r~_i = (x_i, y_i, max(z_i, a)),  s_i = clamp(z_i / a, s_min, 1),
 *     so M = S M(r~) S is SPD whenever M(r~) is.
 *   - wall = 0 switches the image part and the regularisation off
 *     (unbounded RPY); used by the free-space pins.
 *   - Lx, Ly > 0: pseudo-periodic suspension (Sec. 4.2): every pair sums the
 *     source's minimum image in x, y and its 8 nearest periodic images.
 *
 * Derivatives (adjoint, divergence) are exact: the same block code is
 * instantiated on a forward-mode dual number carrying d/d(x_i, x_j).
 *
 * Layouts: positions SoA r[0..n) = x, r[n..2n) = y, r[2n..3n) = z;
 * vectors [k][3][n].
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

/* forward-mode dual number with 6 partials: d/d(target x,y,z, source x,y,z) */
struct Dual {
    double v;
    double g[6];
    Dual() : v(0.0) { for (double& q : g) q = 0.0; }
    Dual(double x) : v(x) { for (double& q : g) q = 0.0; }
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int q = 0; q < 6; ++q) r.g[q] = a.g[q] + b.g[q]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int q = 0; q < 6; ++q) r.g[q] = a.g[q] - b.g[q]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int q = 0; q < 6; ++q) r.g[q] = -a.g[q]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int q = 0; q < 6; ++q) r.g[q] = a.g[q] * b.v + a.v * b.g[q]; return r; }
inline Dual operator/(const Dual& a, const Dual& b)
{
    Dual r(a.v / b.v);
    for (int q = 0; q < 6; ++q) r.g[q] = (a.g[q] * b.v - a.v * b.g[q]) / (b.v * b.v);
    return r;
}
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int q = 0; q < 6; ++q) r.g[q] = a.g[q] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual pow(const Dual& a, double p)
{
    Dual r(std::pow(a.v, p));
    double d = p * std::pow(a.v, p - 1.0);
    for (int q = 0; q < 6; ++q) r.g[q] = d * a.g[q];
    return r;
}
inline Dual pow(const Dual& a, int p) { return pow(a, (double)p); }
inline Dual sqrt(const Dual& a)
{
    Dual r(std::sqrt(a.v));
    for (int q = 0; q < 6; ++q) r.g[q] = a.g[q] / (2.0 * r.v);
    return r;
}
using std::pow;
using std::sqrt;
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

}  // namespace

#include "rpb_generated.h"

namespace {

const double ORC_PI = 3.14159265358979323846;

struct Params {
    double eta, a;
    int wall;
    double s_min;
    double Lx, Ly;  // pseudo-periodic cell in x, y (0: open)
};

/* regularised height and scale of one blob, with their z-derivatives */
void reg(const Params& p, double z, double* zt, double* s, double* dzt, double* ds)
{
    if (!p.wall) { *zt = z; *s = 1.0; *dzt = 1.0; *ds = 0.0; return; }
    if (z >= p.a) { *zt = z; *dzt = 1.0; } else { *zt = p.a; *dzt = 0.0; }
    double t = z / p.a;
    if (t >= 1.0) { *s = 1.0; *ds = 0.0; }
    else if (t <= p.s_min) { *s = p.s_min; *ds = 0.0; }
    else { *s = t; *ds = 1.0 / p.a; }
}

/* 8 pi eta times the free-space RPY block for separation d (textbook form).
 * same: self block (i == j). */
template <class T>
void rpy(const T* d, double a, bool same, T* B)
{
    if (same) {
        for (int q = 0; q < 9; ++q) B[q] = T(0.0);
        B[0] = B[4] = B[8] = T(4.0 / (3.0 * a));
        return;
    }
    T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    T r = sqrt(r2);
    T c1, c2;
    if (val(r) >= 2.0 * a) {
        c1 = (1.0 + 2.0 * a * a / (3.0 * r2)) / r;
        c2 = (1.0 - 2.0 * a * a / r2) / (r * r2);
    } else {
        c1 = 4.0 / (3.0 * a) * (1.0 - 9.0 * r / (32.0 * a));
        c2 = 4.0 / (3.0 * a) * 3.0 / (32.0 * a * r);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            B[i * 3 + j] = (i == j ? c1 : T(0.0)) + c2 * d[i] * d[j];
}


/* 8 pi eta times Mtilde(xi, xj) = M_RPY + M_wall at regularised positions */
template <class T>
void block_t(const Params& p, const T* xi, const T* xj, bool same, T* B)
{
    T d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    bool coincide = same || (val(d[0]) == 0.0 && val(d[1]) == 0.0 && val(d[2]) == 0.0);
    rpy(d, p.a, coincide, B);
    if (p.wall) {
        T W[9];
        rpb_wall_block(xi, xj, T(p.a), W);
        for (int q = 0; q < 9; ++q) B[q] = B[q] + W[q];
    }
}

/* M_ij in physical units, one image */
void block_one(const Params& p, const double* ri, const double* rj, bool same, double* M)
{
    double zti, si, dzi, dsi, ztj, sj, dzj, dsj;
    reg(p, ri[2], &zti, &si, &dzi, &dsi);
    reg(p, rj[2], &ztj, &sj, &dzj, &dsj);
    double xi[3] = {ri[0], ri[1], zti}, xj[3] = {rj[0], rj[1], ztj};
    double B[9];
    block_t<double>(p, xi, xj, same, B);
    double c = si * sj / (8.0 * ORC_PI * p.eta);
    for (int q = 0; q < 9; ++q) M[q] = c * B[q];
}

/* Derivatives of M_ij(r_i, r_j): Dx[(c*3+d)*3+e] = d(M_ij)_cd / d r_i,e and
 * Dy likewise for r_j, with the overlap regularisation chained in.  For
 * i == j the caller adds Dx + Dy (both arguments are the same blob).  The
 * free-space part of a coincident pair is constant and contributes nothing. */
void dblock_one(const Params& p, const double* ri, const double* rj, bool same, double* Dx, double* Dy)
{
    double zti, si, dzi, dsi, ztj, sj, dzj, dsj;
    reg(p, ri[2], &zti, &si, &dzi, &dsi);
    reg(p, rj[2], &ztj, &sj, &dzj, &dsj);
    double xv[6] = {ri[0], ri[1], zti, rj[0], rj[1], ztj};
    Dual x[6];
    for (int q = 0; q < 6; ++q) { x[q] = Dual(xv[q]); x[q].g[q] = 1.0; }
    Dual B[9];
    block_t<Dual>(p, x, x + 3, same, B);
    double c0 = 1.0 / (8.0 * ORC_PI * p.eta);
    for (int q = 0; q < 9; ++q) {
        for (int e = 0; e < 3; ++e) {
            double gx = B[q].g[e], gy = B[q].g[3 + e];
            if (e == 2) { gx *= dzi; gy *= dzj; }
            double vx = si * sj * gx, vy = si * sj * gy;
            if (e == 2) { vx += dsi * sj * B[q].v; vy += si * dsj * B[q].v; }
            Dx[q * 3 + e] = c0 * vx;
            Dy[q * 3 + e] = c0 * vy;
        }
    }
}

/* Pseudo-periodic sum (Sec. 4.2): the source is moved to its minimum image
 * in x and y, then that image and its 8 nearest periodic images all act on
 * the target.  For i == j the unshifted term is the self block. */
template <class F>
void for_images(const Params& p, const double* ri, const double* rj, bool same, F f)
{
    if (!(p.Lx > 0.0 && p.Ly > 0.0)) {
        f(rj, same);
        return;
    }
    const double mx = std::nearbyint((ri[0] - rj[0]) / p.Lx), my = std::nearbyint((ri[1] - rj[1]) / p.Ly);
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            const double img[3] = {rj[0] + (mx + a) * p.Lx, rj[1] + (my + b) * p.Ly, rj[2]};
            f(img, same && a == 0 && b == 0);
        }
}

void block(const Params& p, const double* ri, const double* rj, bool same, double* M)
{
    for (int q = 0; q < 9; ++q) M[q] = 0.0;
    for_images(p, ri, rj, same, [&](const double* y, bool sm) {
        double B[9];
        block_one(p, ri, y, sm, B);
        for (int q = 0; q < 9; ++q) M[q] += B[q];
    });
}

void dblock(const Params& p, const double* ri, const double* rj, bool same, double* Dx, double* Dy)
{
    for (int q = 0; q < 27; ++q) Dx[q] = Dy[q] = 0.0;
    for_images(p, ri, rj, same, [&](const double* y, bool sm) {
        double X[27], Y[27];
        dblock_one(p, ri, y, sm, X, Y);
        for (int q = 0; q < 27; ++q) {
            Dx[q] += X[q];
            Dy[q] += Y[q];
        }
    });
}

/* Neumaier compensated accumulator */
struct Acc {
    double s = 0.0, c = 0.0;
    void add(double v)
    {
        double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v; else c += (v - t) + s;
        s = t;
    }
    double get() const { return s + c; }
};

inline void load3(const double* r, int64_t n, int64_t i, double* out)
{
    out[0] = r[i]; out[1] = r[n + i]; out[2] = r[2 * n + i];
}

}  // namespace

extern "C" {

/* U = M F for k right-hand sides on the rows listed in `rows` (all rows when
 * rows == NULL, nrows == n).  Output layout [k][3][nrows]. */
void orc_mobility_apply_rows(int64_t n, const double* r, const double* F, double* U, int k,
                             double eta, double a, int wall, double s_min, double Lx, double Ly,
                             const int64_t* rows, int64_t nrows)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows ? rows[q] : q;
        double ri[3], rj[3], M[9];
        load3(r, n, i, ri);
        std::vector<Acc> acc(3 * (size_t)k);
        for (int64_t j = 0; j < n; ++j) {
            load3(r, n, j, rj);
            block(p, ri, rj, i == j, M);
            for (int m = 0; m < k; ++m) {
                const double* Fm = F + (int64_t)m * 3 * n;
                double f0 = Fm[j], f1 = Fm[n + j], f2 = Fm[2 * n + j];
                for (int c = 0; c < 3; ++c)
                    acc[m * 3 + c].add(M[c * 3 + 0] * f0 + M[c * 3 + 1] * f1 + M[c * 3 + 2] * f2);
            }
        }
        for (int m = 0; m < k; ++m)
            for (int c = 0; c < 3; ++c)
                U[(int64_t)m * 3 * nrows + c * nrows + q] = acc[m * 3 + c].get();
    }
}

void orc_mobility_apply(int64_t n, const double* r, const double* F, double* U, int k,
                        double eta, double a, int wall, double s_min, double Lx, double Ly)
{
    orc_mobility_apply_rows(n, r, F, U, k, eta, a, wall, s_min, Lx, Ly, nullptr, n);
}

/* dense 3n x 3n matrix, row-major: entry (3i+c, 3j+d) = (M_ij)_cd */
void orc_mobility_dense(int64_t n, const double* r, double* Md, double eta, double a, int wall, double s_min,
                        double Lx, double Ly)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double ri[3], rj[3], M[9];
        load3(r, n, i, ri);
        for (int64_t j = 0; j < n; ++j) {
            load3(r, n, j, rj);
            block(p, ri, rj, i == j, M);
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d)
                    Md[(3 * i + c) * (3 * n) + 3 * j + d] = M[c * 3 + d];
        }
    }
}

/* g_k = d(u^T M F)/d r_k for the blobs listed in `rows` (all when NULL),
 * output [3][nrows].  Straight from the definition: every ordered pair (i, j)
 * depends on r_i as target and on r_j as source. */
void orc_mobility_grad_rows(int64_t n, const double* r, const double* u, const double* F, double* g,
                            double eta, double a, int wall, double s_min, double Lx, double Ly,
                            const int64_t* rows, int64_t nrows)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t k = rows ? rows[q] : q;
        double rk[3], rj[3], Dx[27], Dy[27];
        load3(r, n, k, rk);
        Acc acc[3];
        double uk[3] = {u[k], u[n + k], u[2 * n + k]};
        double Fk[3] = {F[k], F[n + k], F[2 * n + k]};
        for (int64_t j = 0; j < n; ++j) {
            load3(r, n, j, rj);
            double uj[3] = {u[j], u[n + j], u[2 * n + j]};
            double Fj[3] = {F[j], F[n + j], F[2 * n + j]};
            /* pair (k, j): k is the target */
            dblock(p, rk, rj, k == j, Dx, Dy);
            for (int e = 0; e < 3; ++e) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) s += uk[c] * Dx[(c * 3 + d) * 3 + e] * Fj[d];
                acc[e].add(s);
            }
            /* pair (j, k): k is the source */
            dblock(p, rj, rk, k == j, Dx, Dy);
            for (int e = 0; e < 3; ++e) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) s += uj[c] * Dy[(c * 3 + d) * 3 + e] * Fk[d];
                acc[e].add(s);
            }
        }
        for (int e = 0; e < 3; ++e) g[e * nrows + q] = acc[e].get();
    }
}

/* (div M)_i,c = sum_j sum_d d(M_ij)_cd / d r_j,d for the listed rows
 * (the divergence the RFD identity of Sec. 3 estimates, with B = M).
 * For j = i both arguments move together. Output [3][nrows]. */
void orc_mobility_div_rows(int64_t n, const double* r, double* div, double eta, double a, int wall,
                           double s_min, double Lx, double Ly, const int64_t* rows, int64_t nrows)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t i = rows ? rows[q] : q;
        double ri[3], rj[3], Dx[27], Dy[27];
        load3(r, n, i, ri);
        Acc acc[3];
        for (int64_t j = 0; j < n; ++j) {
            load3(r, n, j, rj);
            dblock(p, ri, rj, i == j, Dx, Dy);
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    s += Dy[(c * 3 + d) * 3 + d];
                    if (i == j) s += Dx[(c * 3 + d) * 3 + d];
                }
                acc[c].add(s);
            }
        }
        for (int c = 0; c < 3; ++c) div[c * nrows + q] = acc[c].get();
    }
}

/* one block M_ij (physical units), for pins */
void orc_pair_block(const double* ri, const double* rj, int same, double eta, double a, int wall,
                    double s_min, double Lx, double Ly, double* M)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
    block(p, ri, rj, same != 0, M);
}

/* one block's derivatives, for pins */
void orc_pair_dblock(const double* ri, const double* rj, int same, double eta, double a, int wall,
                     double s_min, double Lx, double Ly, double* Dx, double* Dy)
{
    Params p{eta, a, wall, s_min, Lx, Ly};
    dblock(p, ri, rj, same != 0, Dx, Dy);
}

/* Blake's point-force solution alone (a = 0, no regularisation), times
 * 8 pi eta: G = S(x - y) + image part.  For the no-slip and reciprocity pins. */
void orc_blake_point(const double* x, const double* y, double* G)
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = std::sqrt(r2);
    double W[9];
    rpb_wall_block<double>(x, y, 0.0, W);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            G[i * 3 + j] = (i == j ? 1.0 / r : 0.0) + d[i] * d[j] / (r * r2) + W[i * 3 + j];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the OpenMP loops from now on (for timing at a fixed core count) */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

}  /* extern "C" */
