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

template <bool WALL, bool PER, class S>
__global__ void adjoint_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ u,
                               const double* __restrict__ F, double a, double s_min, double Lx, double Ly,
                               double inv8pieta, double* __restrict__ g)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const PairConst<S> pc = PairConst<S>::make(a, Lx, Ly);
    const RegBlob bk = reg_blob(r, n, k, a, WALL, s_min);
    const double uk[3] = {u[k], u[n + k], u[2 * n + k]};
    const double Fk[3] = {F[k], F[n + k], F[2 * n + k]};
    double psi = 0.0, gr[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        const RegBlob bj = reg_blob(r, n, j, a, WALL, s_min);
        const double Fj[3] = {bj.s * F[j], bj.s * F[n + j], bj.s * F[2 * n + j]};
        const double uj[3] = {bj.s * u[j], bj.s * u[n + j], bj.s * u[2 * n + j]};
        Dual<3, S> M[9];
        dual_block<WALL, PER, S>(bk, bj, pc, M);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double w = uk[c] * Fj[d] + Fk[c] * uj[d];
                psi += w * (double)M[c * 3 + d].v;
#pragma unroll
                for (int e = 0; e < 3; ++e) gr[e] += w * (double)M[c * 3 + d].g[e];
            }
    }
    g[k] = inv8pieta * bk.s * gr[0];
    g[n + k] = inv8pieta * bk.s * gr[1];
    g[2 * n + k] = inv8pieta * (bk.s * gr[2] * bk.dzt + bk.ds * psi);
}

// ---------------------------------------------------------------------------
// FP32 adjoint: the same psi_k and target-slot derivative as adjoint_kernel,
// computed with FP32 pair arithmetic.  Sources are packed once into 48-byte
// records [x_hi, y_hi, x_lo, y_lo | zt, s F | s u, 0] (hi/lo split of x, y
// so separations keep FP64-level accuracy), staged through shared memory in
// tiles of 128 and split into chunks of 2048 sources (FP32 sums per chunk,
// FP64 across chunks in a fixed order).  Instead of assembling the nine
// dual-number entries, psi is contracted directly against the five block
// scalars of pair_factors: with d = (dx, dy),
//   a^T M c = alpha (a_x c_x + a_y c_y) + beta (a.d)(d.c) + gx (a.d) c_z
//             + gz a_z (d.c) + Mzz a_z c_z,
// and the explicit d-dependence of (a.d), (d.c) is differentiated by hand.
namespace adjf32 {

constexpr int BT = 128;    // targets per CTA = sources per shared tile
constexpr int CH = 2048;   // sources per chunk

__global__ void pack_kernel(int64_t n, const double* __restrict__ r, const double* __restrict__ u,
                            const double* __restrict__ F, double a, int wall, double s_min, float4* __restrict__ rec)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RegBlob b = reg_blob(r, n, i, a, wall, s_min);
    const float xh = (float)b.x, yh = (float)b.y;
    rec[3 * i] = make_float4(xh, yh, (float)(b.x - (double)xh), (float)(b.y - (double)yh));
    rec[3 * i + 1] = make_float4((float)b.zt, (float)(b.s * F[i]), (float)(b.s * F[n + i]), (float)(b.s * F[2 * n + i]));
    rec[3 * i + 2] = make_float4((float)(b.s * u[i]), (float)(b.s * u[n + i]), (float)(b.s * u[2 * n + i]), 0.0f);
}

struct Vecs {
    float ax, ay, az, bx, by, bz;  // target: a = u_k, b = F_k
    float cx, cy, cz, ex, ey, ez;  // source: c = s_j F_j, e = s_j u_j
    float S1, S3;                  // a_xy.c_xy + b_xy.e_xy, a_z c_z + b_z e_z
};

template <bool WALL>
__device__ __forceinline__ void contract(float dxv, float dyv, float dzv, float zi, float zj, const PairConst<float>& pc,
                                         const Vecs& w, float& psi, float g[3])
{
    using D3 = Dual<3, float>;
    D3 dx(dxv), dy(dyv), dz(dzv), Zi(zi), Zj(zj);
    dx.g[0] = 1.0f;
    dy.g[1] = 1.0f;
    dz.g[2] = 1.0f;
    Zi.g[2] = 1.0f;
    D3 al, be, gx, gz, mzz;
    pair_factors<D3, float, WALL>(dx, dy, dz, Zi, Zj, pc, al, be, gx, gz, mzz);
    const float P1 = fmaf(w.ay, dyv, w.ax * dxv), D1 = fmaf(w.cy, dyv, w.cx * dxv);
    const float P2 = fmaf(w.by, dyv, w.bx * dxv), D2 = fmaf(w.ey, dyv, w.ex * dxv);
    const float Q = fmaf(P2, D2, P1 * D1);
    const float Rr = fmaf(w.ez, P2, w.cz * P1);
    const float Zz = fmaf(w.bz, D2, w.az * D1);
    psi += al.v * w.S1 + be.v * Q + gx.v * Rr + gz.v * Zz + mzz.v * w.S3;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        g[q] += al.g[q] * w.S1 + be.g[q] * Q + gx.g[q] * Rr + gz.g[q] * Zz + mzz.g[q] * w.S3;
    // d/d(dx), d/d(dy) of Q, Rr, Zz
    const float dQx = w.ax * D1 + w.cx * P1 + w.bx * D2 + w.ex * P2;
    const float dQy = w.ay * D1 + w.cy * P1 + w.by * D2 + w.ey * P2;
    g[0] += be.v * dQx + gx.v * (w.cz * w.ax + w.ez * w.bx) + gz.v * (w.az * w.cx + w.bz * w.ex);
    g[1] += be.v * dQy + gx.v * (w.cz * w.ay + w.ez * w.by) + gz.v * (w.az * w.cy + w.bz * w.ey);
}

template <bool WALL, bool PER>
__global__ void __launch_bounds__(BT) adjoint_f32_kernel(int64_t n, const float4* __restrict__ rec,
                                                         const double* __restrict__ u, const double* __restrict__ F,
                                                         PairConst<float> pc, float* __restrict__ part)
{
    __shared__ float4 tile[3 * BT];
    const int tid = threadIdx.x;
    const int64_t k = blockIdx.x * (int64_t)BT + tid;
    const int64_t kk = k < n ? k : n - 1;
    const float4 t0 = rec[3 * kk], t1 = rec[3 * kk + 1];
    Vecs w;
    w.ax = (float)u[kk]; w.ay = (float)u[n + kk]; w.az = (float)u[2 * n + kk];
    w.bx = (float)F[kk]; w.by = (float)F[n + kk]; w.bz = (float)F[2 * n + kk];
    const int64_t j0 = (int64_t)blockIdx.y * CH;
    const int64_t j1 = (j0 + CH) < n ? (j0 + CH) : n;
    float psi = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
    for (int64_t base = j0; base < j1; base += BT) {
        const int64_t j = base + tid;
        if (j < j1) {
            tile[3 * tid] = rec[3 * j];
            tile[3 * tid + 1] = rec[3 * j + 1];
            tile[3 * tid + 2] = rec[3 * j + 2];
        }
        __syncthreads();
        const int cnt = (int)((j1 - base) < BT ? (j1 - base) : BT);
        for (int jj = 0; jj < cnt; ++jj) {
            const float4 s0 = tile[3 * jj], s1 = tile[3 * jj + 1], s2 = tile[3 * jj + 2];
            const float dxv = (t0.x - s0.x) + (t0.z - s0.z), dyv = (t0.y - s0.y) + (t0.w - s0.w);
            w.cx = s1.y; w.cy = s1.z; w.cz = s1.w;
            w.ex = s2.x; w.ey = s2.y; w.ez = s2.z;
            w.S1 = fmaf(w.ay, w.cy, w.ax * w.cx) + fmaf(w.by, w.ey, w.bx * w.ex);
            w.S3 = fmaf(w.bz, w.ez, w.az * w.cz);
            if (!PER) {
                contract<WALL>(dxv, dyv, t1.x - s1.x, t1.x, s1.x, pc, w, psi, g);
            } else {
                const float dxm = dxv - pc.Lx * rintf(dxv * pc.iLx), dym = dyv - pc.Ly * rintf(dyv * pc.iLy);
#pragma unroll
                for (int ia = -1; ia <= 1; ++ia)
#pragma unroll
                    for (int ib = -1; ib <= 1; ++ib)
                        contract<WALL>(dxm + (float)ia * pc.Lx, dym + (float)ib * pc.Ly, t1.x - s1.x, t1.x, s1.x, pc, w,
                                       psi, g);
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

// g_k from the chunk partials, FP64, chunks in order
__global__ void reduce_kernel(int64_t n, int nch, const float* __restrict__ part, const double* __restrict__ r,
                              double a, int wall, double s_min, double inv8pieta, double* __restrict__ grad)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < nch; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += (double)part[((int64_t)c * 4 + q) * n + k];
    const RegBlob b = reg_blob(r, n, k, a, wall, s_min);
    grad[k] = inv8pieta * b.s * acc[1];
    grad[n + k] = inv8pieta * b.s * acc[2];
    grad[2 * n + k] = inv8pieta * (b.s * acc[3] * b.dzt + b.ds * acc[0]);
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

static int adjoint_entry(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F, double* grad,
                         void* stream, bool f32)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || (n > 0 && (!r || !u || !F || !grad))) return set_error(h, RPBD_BAD_ARG, "adjoint: bad arguments");
    if (n == 0) return RPBD_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const unsigned grid = (unsigned)((n + 127) / 128);
    const double a = h->p.a, sm = h->p.s_min, Lx = h->p.Lx, Ly = h->p.Ly;
    const bool per = Lx > 0.0;
    if (f32) {
        using namespace adjf32;
        float4* rec;
        float* part;
        const int nch = (int)((n + CH - 1) / CH);
        RPBD_TRY(ensure_t(h, BUF_PACK, (size_t)3 * n, &rec));
        RPBD_TRY(ensure_t(h, BUF_PARTIAL, (size_t)nch * 4 * n, &part));
        const int wall = h->p.wall ? 1 : 0;
        pack_kernel<<<grid, 128, 0, st>>>(n, r, u, F, a, wall, sm, rec);
        count_launch();
        const PairConst<float> pc = PairConst<float>::make(a, Lx, Ly);
        const dim3 g2(grid, (unsigned)nch);
        if (per) adjoint_f32_kernel<true, true><<<g2, BT, 0, st>>>(n, rec, u, F, pc, part);
        else if (wall) adjoint_f32_kernel<true, false><<<g2, BT, 0, st>>>(n, rec, u, F, pc, part);
        else adjoint_f32_kernel<false, false><<<g2, BT, 0, st>>>(n, rec, u, F, pc, part);
        count_launch();
        reduce_kernel<<<grid, 128, 0, st>>>(n, nch, part, r, a, wall, sm, inv8pieta, grad);
    } else {
        if (per) adjoint_kernel<true, true, double><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else if (h->p.wall) adjoint_kernel<true, false, double><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else adjoint_kernel<false, false, double><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
    }
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_mobility_adjoint(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F, double* grad,
                          void* stream)
{
    return adjoint_entry(h, n, r, u, F, grad, stream, false);
}

int rpbd_mobility_adjoint_f32(rpbd_handle* h, int64_t n, const double* r, const double* u, const double* F,
                              double* grad, void* stream)
{
    return adjoint_entry(h, n, r, u, F, grad, stream, true);
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
