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
        if (per) adjoint_kernel<true, true, float><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else if (h->p.wall) adjoint_kernel<true, false, float><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
        else adjoint_kernel<false, false, float><<<grid, 128, 0, st>>>(n, r, u, F, a, sm, Lx, Ly, inv8pieta, grad);
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
