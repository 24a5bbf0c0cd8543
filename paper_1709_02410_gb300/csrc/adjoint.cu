// Derivatives of the wall-RPY mobility (FP64; the adjoint also in FP32):
//
//  adjoint:    g_k = d(u^T M(r) F)/d r_k  (derivative of the matvec of
//              Sec. 2.1 with respect to blob positions)
//  divergence: (div M)_i = sum_j d_{r_j} . M_ij  (the drift the RFD of
//              Sec. 3 estimates with B = M)
//
// Both evaluate the pair block on a forward-mode dual number carrying the
// three partials with respect to the TARGET blob's (regularised) position,
// and use the reciprocal symmetry M_ij(r_i, r_j) = M_ji(r_j, r_i)^T to turn
// every source-side derivative into a target-side one.  So each thread owns
// one blob and no atomics are needed:
//
//  With M_ij = s_i s_j Mt(rt_i, rt_j) (rt = (x, y, max(z, a)),
//  s = clamp(z/a, s_min, 1)) and psi_k = sum_j [u_k^T Mt_kj (s_j F_j) +
//  F_k^T Mt_kj (s_j u_j)]:   g_k = s_k d psi_k / d rt_k (z part times
//  d zt/dz) + z^ (d s_k/dz) psi_k.
#include <cuda_runtime.h>

#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"

namespace rpbd {


struct RegBlob {
    double x, y, zt, s, dzt, ds;
};

__device__ __forceinline__ RegBlob reg_blob(const double* r, int64_t n, int64_t i, double a, int wall, double s_min)
{
    RegBlob b;
    b.x = r[i];
    b.y = r[n + i];
    const double z = r[2 * n + i];
    if (wall) {
        if (z >= a) { b.zt = z; b.dzt = 1.0; } else { b.zt = a; b.dzt = 0.0; }
        const double t = z / a;
        if (t >= 1.0) { b.s = 1.0; b.ds = 0.0; }
        else if (t <= s_min) { b.s = s_min; b.ds = 0.0; }
        else { b.s = t; b.ds = 1.0 / a; }
    } else {
        b.zt = z; b.dzt = 1.0; b.s = 1.0; b.ds = 0.0;
    }
    return b;
}

// block of target t (dual: partials w.r.t. t's regularised coordinates) and
// source s; out[9] row-major.  Differences are taken in FP64, then the block
// is evaluated in S (double, or float for the FP32 variant).
template <bool WALL, bool PER, class S>
__device__ __forceinline__ void dual_block(const RegBlob& t, const RegBlob& s, const PairConst<S>& pc,
                                           Dual<3, S> M[9])
{
    using D3 = Dual<3, S>;
    D3 dx(S(t.x - s.x)), dy(S(t.y - s.y)), dz(S(t.zt - s.zt)), zi(S(t.zt)), zj(S(s.zt));
    dx.g[0] = S(1);
    dy.g[1] = S(1);
    dz.g[2] = S(1);
    zi.g[2] = S(1);
    D3 Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz;
    pair_block_images<D3, S, WALL, PER>(dx, dy, dz, zi, zj, pc, Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz);
    M[0] = Mxx; M[1] = Mxy; M[2] = Mxz;
    M[3] = Mxy; M[4] = Myy; M[5] = Myz;
    M[6] = Mzx; M[7] = Mzy; M[8] = Mzz;
}

// nr right-hand-side pairs (u_m, F_m), [nr][3][n] each: the weights
// w_cd = sum_m (u_mk)_c (s_j F_mj)_d + (F_mk)_c (s_j u_mj)_d of one pair are
// summed over m before they meet the block, which is formed once.
template <bool WALL, bool PER, class S>
__global__ void adjoint_kernel(int64_t n, int nr, const double* __restrict__ r, const double* __restrict__ u,
                               const double* __restrict__ F, double a, double s_min, double Lx, double Ly,
                               double inv8pieta, double* __restrict__ g)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const PairConst<S> pc = PairConst<S>::make(a, Lx, Ly);
    const RegBlob bk = reg_blob(r, n, k, a, WALL, s_min);
    double psi = 0.0, gr[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        const RegBlob bj = reg_blob(r, n, j, a, WALL, s_min);
        double w[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int m = 0; m < nr; ++m) {
            const double* um = u + (int64_t)m * 3 * n;
            const double* Fm = F + (int64_t)m * 3 * n;
            const double uk[3] = {um[k], um[n + k], um[2 * n + k]};
            const double Fk[3] = {Fm[k], Fm[n + k], Fm[2 * n + k]};
            const double Fj[3] = {bj.s * Fm[j], bj.s * Fm[n + j], bj.s * Fm[2 * n + j]};
            const double uj[3] = {bj.s * um[j], bj.s * um[n + j], bj.s * um[2 * n + j]};
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) w[c * 3 + d] += uk[c] * Fj[d] + Fk[c] * uj[d];
        }
        Dual<3, S> M[9];
        dual_block<WALL, PER, S>(bk, bj, pc, M);
#pragma unroll
        for (int cd = 0; cd < 9; ++cd) {
            psi += w[cd] * (double)M[cd].v;
#pragma unroll
            for (int e = 0; e < 3; ++e) gr[e] += w[cd] * (double)M[cd].g[e];
        }
    }
    g[k] = inv8pieta * bk.s * gr[0];
    g[n + k] = inv8pieta * bk.s * gr[1];
    g[2 * n + k] = inv8pieta * (bk.s * gr[2] * bk.dzt + bk.ds * psi);
}

// ---------------------------------------------------------------------------
// FP32 adjoint: the same psi_k and target-slot derivative as adjoint_kernel,
// computed with FP32 pair arithmetic, for k right-hand-side pairs in passes
// of up to four (their target vectors stay in registers).  Sources are packed
// per pass into records [x_hi, y_hi, x_lo, y_lo | zt | s F_m, s u_m ...]
// (hi/lo split of x, y so separations keep FP64-level accuracy), staged
// through shared memory in tiles of 128 and split into chunks of 2048 sources
// (FP32 sums per chunk, FP64 across chunks and passes in a fixed order).
// Instead of assembling the nine dual-number entries, psi is contracted
// directly against the five block scalars of pair_factors: with d = (dx, dy),
//   a^T M c = alpha (a_x c_x + a_y c_y) + beta (a.d)(d.c) + gx (a.d) c_z
//             + gz a_z (d.c) + Mzz a_z c_z,
// and the explicit d-dependence of (a.d), (d.c) is differentiated by hand.
namespace adjf32 {

constexpr int BT = 128;    // targets per CTA = sources per shared tile
constexpr int CH = 2048;   // sources per chunk
constexpr int KCMAX = 4;   // right-hand-side pairs per pass (target vectors held in registers)

// Source record of one pass over kc <= KCT right-hand-side pairs:
// [x_hi, y_hi, x_lo, y_lo | zt, 0, 0, 0 | c_0, e_0, c_1, e_1, ...] with
// c_m = s_j F_mj and e_m = s_j u_mj (3 floats each), padded to whole float4s.
template <int KCT>
struct ARec {
    static constexpr int LEN = 8 + (6 * KCT + 3) / 4 * 4;
};

// u, F point at the pass's first right-hand side; stride 3n between pairs
template <int KCT>
__global__ void pack_kernel(int64_t n, int kc, const double* __restrict__ r, const double* __restrict__ u,
                            const double* __restrict__ F, double a, int wall, double s_min, float* __restrict__ rec)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int LEN = ARec<KCT>::LEN;
    const RegBlob b = reg_blob(r, n, i, a, wall, s_min);
    float v[LEN];
#pragma unroll
    for (int q = 0; q < LEN; ++q) v[q] = 0.0f;
    const float xh = (float)b.x, yh = (float)b.y;
    v[0] = xh;
    v[1] = yh;
    v[2] = (float)(b.x - (double)xh);
    v[3] = (float)(b.y - (double)yh);
    v[4] = (float)b.zt;
#pragma unroll
    for (int m = 0; m < KCT; ++m)
        if (m < kc)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[8 + 6 * m + c] = (float)(b.s * F[((int64_t)m * 3 + c) * n + i]);
                v[8 + 6 * m + 3 + c] = (float)(b.s * u[((int64_t)m * 3 + c) * n + i]);
            }
    float4* o = reinterpret_cast<float4*>(rec + i * LEN);
#pragma unroll
    for (int q = 0; q < LEN / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// psi and the target-slot gradient of one pair summed over the pass's
// right-hand-side pairs: the dual-number block scalars are formed once, and
// each pair m (target a = u_m, b = F_m; source c = s_j F_m, e = s_j u_m)
// adds to the scalars they are contracted with.
template <bool WALL, int KCT>
__device__ __forceinline__ void contract(float dxv, float dyv, float dzv, float zi, float zj, const PairConst<float>& pc,
                                         const float* A, const float* B, const float* src, float& psi, float g[3])
{
    using D3 = Dual<3, float>;
    D3 dx(dxv), dy(dyv), dz(dzv), Zi(zi), Zj(zj);
    dx.g[0] = 1.0f;
    dy.g[1] = 1.0f;
    dz.g[2] = 1.0f;
    Zi.g[2] = 1.0f;
    D3 al, be, gx, gz, mzz;
    pair_factors<D3, float, WALL>(dx, dy, dz, Zi, Zj, pc, al, be, gx, gz, mzz);
    // S1 = a_xy.c_xy + b_xy.e_xy, S3 = a_z c_z + b_z e_z, Q = (a.d)(d.c) + (b.d)(d.e),
    // Rr = c_z (a.d) + e_z (b.d), Zz = a_z (d.c) + b_z (d.e), and the explicit
    // d/d(dx), d/d(dy) of Q, Rr, Zz
    float S1 = 0.0f, S3 = 0.0f, Q = 0.0f, Rr = 0.0f, Zz = 0.0f, dQx = 0.0f, dQy = 0.0f;
    float Gx0 = 0.0f, Gx1 = 0.0f, Gz0 = 0.0f, Gz1 = 0.0f;
#pragma unroll
    for (int m = 0; m < KCT; ++m) {
        const float ax = A[3 * m], ay = A[3 * m + 1], az = A[3 * m + 2];
        const float bx = B[3 * m], by = B[3 * m + 1], bz = B[3 * m + 2];
        const float* cs = src + 8 + 6 * m;
        const float cx = cs[0], cy = cs[1], cz = cs[2], ex = cs[3], ey = cs[4], ez = cs[5];
        S1 += fmaf(ay, cy, ax * cx) + fmaf(by, ey, bx * ex);
        S3 += fmaf(bz, ez, az * cz);
        const float P1 = fmaf(ay, dyv, ax * dxv), D1 = fmaf(cy, dyv, cx * dxv);
        const float P2 = fmaf(by, dyv, bx * dxv), D2 = fmaf(ey, dyv, ex * dxv);
        Q += fmaf(P2, D2, P1 * D1);
        Rr += fmaf(ez, P2, cz * P1);
        Zz += fmaf(bz, D2, az * D1);
        dQx += ax * D1 + cx * P1 + bx * D2 + ex * P2;
        dQy += ay * D1 + cy * P1 + by * D2 + ey * P2;
        Gx0 += cz * ax + ez * bx;
        Gx1 += cz * ay + ez * by;
        Gz0 += az * cx + bz * ex;
        Gz1 += az * cy + bz * ey;
    }
    psi += al.v * S1 + be.v * Q + gx.v * Rr + gz.v * Zz + mzz.v * S3;
#pragma unroll
    for (int q = 0; q < 3; ++q) g[q] += al.g[q] * S1 + be.g[q] * Q + gx.g[q] * Rr + gz.g[q] * Zz + mzz.g[q] * S3;
    g[0] += be.v * dQx + gx.v * Gx0 + gz.v * Gz0;
    g[1] += be.v * dQy + gx.v * Gx1 + gz.v * Gz1;
}

// one pass: kc <= KCT right-hand-side pairs, partials of chunk blockIdx.y
// written to part[(blockIdx.y * 4 + q) * n + k], q = (psi, g_x, g_y, g_z)
template <bool WALL, bool PER, int KCT>
__global__ void __launch_bounds__(BT) adjoint_f32_kernel(int64_t n, int kc, const float* __restrict__ rec,
                                                         const double* __restrict__ u, const double* __restrict__ F,
                                                         PairConst<float> pc, float* __restrict__ part)
{
    constexpr int LEN = ARec<KCT>::LEN;
    __shared__ __align__(16) float tile[BT * LEN];
    const int tid = threadIdx.x;
    const int64_t k = blockIdx.x * (int64_t)BT + tid;
    const int64_t kk = k < n ? k : n - 1;
    const float4 t0 = *reinterpret_cast<const float4*>(rec + kk * LEN);
    const float zi = rec[kk * LEN + 4];
    float A[3 * KCT], B[3 * KCT];
#pragma unroll
    for (int m = 0; m < KCT; ++m)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A[3 * m + c] = m < kc ? (float)u[((int64_t)m * 3 + c) * n + kk] : 0.0f;
            B[3 * m + c] = m < kc ? (float)F[((int64_t)m * 3 + c) * n + kk] : 0.0f;
        }
    const int64_t j0 = (int64_t)blockIdx.y * CH;
    const int64_t j1 = (j0 + CH) < n ? (j0 + CH) : n;
    float psi = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
    for (int64_t base = j0; base < j1; base += BT) {
        const int cnt = (int)((j1 - base) < BT ? (j1 - base) : BT);
        const float4* srcv = reinterpret_cast<const float4*>(rec + base * LEN);
        for (int e = tid; e < cnt * (LEN / 4); e += BT) reinterpret_cast<float4*>(tile)[e] = srcv[e];
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            const float* sj = tile + jj * LEN;
            const float dxv = (t0.x - sj[0]) + (t0.z - sj[2]), dyv = (t0.y - sj[1]) + (t0.w - sj[3]);
            const float zj = sj[4];
            if (!PER) {
                contract<WALL, KCT>(dxv, dyv, zi - zj, zi, zj, pc, A, B, sj, psi, g);
            } else {
                const float dxm = dxv - pc.Lx * rintf(dxv * pc.iLx), dym = dyv - pc.Ly * rintf(dyv * pc.iLy);
#pragma unroll
                for (int ia = -1; ia <= 1; ++ia)
#pragma unroll
                    for (int ib = -1; ib <= 1; ++ib)
                        contract<WALL, KCT>(dxm + (float)ia * pc.Lx, dym + (float)ib * pc.Ly, zi - zj, zi, zj, pc, A, B,
                                            sj, psi, g);
            }
        }
        __syncthreads();
    }
    if (k < n) {
        float* o = part + (int64_t)blockIdx.y * 4 * n;
        o[k] = psi;
        o[n + k] = g[0];
        o[2 * n + k] = g[1];
        o[3 * n + k] = g[2];
    }
}

// g_k from the partials of every (pass, chunk), FP64, in a fixed order
__global__ void reduce_kernel(int64_t n, int nparts, const float* __restrict__ part, const double* __restrict__ r,
                              double a, int wall, double s_min, double inv8pieta, double* __restrict__ grad)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < nparts; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += (double)part[((int64_t)c * 4 + q) * n + k];
    const RegBlob b = reg_blob(r, n, k, a, wall, s_min);
    grad[k] = inv8pieta * b.s * acc[1];
    grad[n + k] = inv8pieta * b.s * acc[2];
    grad[2 * n + k] = inv8pieta * (b.s * acc[3] * b.dzt + b.ds * acc[0]);
}

template <int KCT>
static void launch_pass(int64_t n, int kc, const double* r, const double* u, const double* F, const rpbd_params& p,
                        float* rec, float* part, cudaStream_t st)
{
    const unsigned grid = (unsigned)((n + BT - 1) / BT);
    const int nch = (int)((n + CH - 1) / CH);
    const int wall = p.wall ? 1 : 0;
    pack_kernel<KCT><<<grid, BT, 0, st>>>(n, kc, r, u, F, p.a, wall, p.s_min, rec);
    count_launch();
    const PairConst<float> pc = PairConst<float>::make(p.a, p.Lx, p.Ly);
    const dim3 g2(grid, (unsigned)nch);
    if (p.Lx > 0.0) adjoint_f32_kernel<true, true, KCT><<<g2, BT, 0, st>>>(n, kc, rec, u, F, pc, part);
    else if (wall) adjoint_f32_kernel<true, false, KCT><<<g2, BT, 0, st>>>(n, kc, rec, u, F, pc, part);
    else adjoint_f32_kernel<false, false, KCT><<<g2, BT, 0, st>>>(n, kc, rec, u, F, pc, part);
    count_launch();
}

}  // namespace adjf32

template <bool WALL, bool PER>
__global__ void divergence_kernel(int64_t n, const double* __restrict__ r, double a, double s_min, double Lx,
                                  double Ly, double inv8pieta, double* __restrict__ div)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const PairConst<double> pc = PairConst<double>::make(a, Lx, Ly);
    const RegBlob bi = reg_blob(r, n, i, a, WALL, s_min);  // divergence: FP64 only
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        Dual<3, double> T[9];
        if (j == i) {
            dual_block<WALL, PER, double>(bi, bi, pc, T);
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                double v = 2.0 * bi.s * bi.ds * T[aa * 3 + 2].v;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const double dzt = b == 2 ? bi.dzt : 1.0;
                    v += bi.s * bi.s * (T[aa * 3 + b].g[b] + T[b * 3 + aa].g[b]) * dzt;
                }
                acc[aa] += v;
            }
        } else {
            const RegBlob bj = reg_blob(r, n, j, a, WALL, s_min);
            dual_block<WALL, PER, double>(bj, bi, pc, T);  // target j, source i
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                double v = bi.s * bj.ds * T[2 * 3 + aa].v;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const double dzt = b == 2 ? bj.dzt : 1.0;
                    v += bi.s * bj.s * T[b * 3 + aa].g[b] * dzt;
                }
                acc[aa] += v;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) div[c * n + i] = inv8pieta * acc[c];
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

static int adjoint_entry(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F, int nr,
                         double* grad, void* stream, bool f32)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || nr < 1 || nr > 16 || (n > 0 && (!r || !u || !F || !grad)))
        return set_error(h, RPBD_BAD_ARG, "adjoint: bad arguments (need n >= 0, 1 <= k <= 16, non-null pointers)");
    if (n == 0) return RPBD_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const unsigned grid = (unsigned)((n + 127) / 128);
    const double a = h->p.a, sm = h->p.s_min, Lx = h->p.Lx, Ly = h->p.Ly;
    const bool per = Lx > 0.0;
    if (f32) {
        using namespace adjf32;
        const int nch = (int)((n + CH - 1) / CH);
        const int npass = (nr + KCMAX - 1) / KCMAX;
        float* rec;
        float* part;
        RPBD_TRY(ensure_t(h, BUF_PACK, (size_t)n * ARec<KCMAX>::LEN, &rec));
        RPBD_TRY(ensure_t(h, BUF_PARTIAL, (size_t)npass * nch * 4 * n, &part));
        for (int ps = 0; ps < npass; ++ps) {
            const int m0 = ps * KCMAX, kc = nr - m0 < KCMAX ? nr - m0 : KCMAX;
            const double* up = u + (int64_t)m0 * 3 * n;
            const double* Fp = F + (int64_t)m0 * 3 * n;
            float* pp = part + (size_t)ps * nch * 4 * n;
            if (kc == 1) launch_pass<1>(n, kc, r, up, Fp, h->p, rec, pp, st);
            else if (kc == 2) launch_pass<2>(n, kc, r, up, Fp, h->p, rec, pp, st);
            else launch_pass<4>(n, kc, r, up, Fp, h->p, rec, pp, st);
        }
        reduce_kernel<<<grid, 128, 0, st>>>(n, npass * nch, part, r, a, h->p.wall ? 1 : 0, sm, inv8pieta, grad);
    } else {
        if (per) adjoint_kernel<true, true, double><<<grid, 128, 0, st>>>(n, nr, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else if (h->p.wall) adjoint_kernel<true, false, double><<<grid, 128, 0, st>>>(n, nr, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else adjoint_kernel<false, false, double><<<grid, 128, 0, st>>>(n, nr, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
    }
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_mobility_adjoint(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F, double* grad,
                          void* stream)
{
    return adjoint_entry(h, n, r, u, F, 1, grad, stream, false);
}

int rpbd_mobility_adjoint_f32(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F,
                              double* grad, void* stream)
{
    return adjoint_entry(h, n, r, u, F, 1, grad, stream, true);
}

int rpbd_mobility_adjoint_multi(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F, int k,
                                double* grad, int dtype, void* stream)
{
    if (h && dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "adjoint: bad dtype");
    return adjoint_entry(h, n, r, u, F, k, grad, stream, dtype == RPBD_F32);
}

int rpbd_mobility_divergence(rpbd_handle* h, int64_t n, const double* r, double* div, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || (n > 0 && (!r || !div))) return set_error(h, RPBD_BAD_ARG, "divergence: bad arguments");
    if (n == 0) return RPBD_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const unsigned grid = (unsigned)((n + 127) / 128);
    const double Lx = h->p.Lx, Ly = h->p.Ly;
    if (Lx > 0.0) divergence_kernel<true, true><<<grid, 128, 0, st>>>(n, r, h->p.a, h->p.s_min, Lx, Ly, inv8pieta, div);
    else if (h->p.wall) divergence_kernel<true, false><<<grid, 128, 0, st>>>(n, r, h->p.a, h->p.s_min, Lx, Ly, inv8pieta, div);
    else divergence_kernel<false, false><<<grid, 128, 0, st>>>(n, r, h->p.a, h->p.s_min, Lx, Ly, inv8pieta, div);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

}  // extern "C"
