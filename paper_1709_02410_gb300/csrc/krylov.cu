// Krylov solvers of the hot path, FP64 vectors on the device:
//
//  Lanczos M^{1/2} W (Sec. 2.2): Lanczos on G = L^-1 M L^-T (L the block
//    Cholesky preconditioner) from v_1 = W/|W| with full (classical, twice)
//    reorthogonalisation; f(G) W ~ |W| V_m T_m^{1/2} e_1, T_m^{1/2} e_1 from a
//    one-warp (round-robin parallel) Jacobi eigendecomposition of T_m; stop
//    when |y_m - y_{m-1}| / |y_m| < tol (evaluated in the small space, V is
//    orthonormal); output L y_m.
//  GMRES (Sec. 2.1, eq. saddle): right-preconditioned restarted GMRES(m) on
//    [M -K; -K^T 0] with the exact body-block solve of Sec. 2.2 as
//    preconditioner; Arnoldi by classical Gram-Schmidt applied twice, Givens
//    rotations and the Hessenberg least-squares solve in a device kernel.
//
// The host drives the iteration and reads one FP64 scalar per iteration (the
// residual estimate or the Lanczos change) to decide whether to stop; every
// arithmetic step runs in the kernels below.
#include <cuda_runtime.h>

#include <cmath>

#include "rpbd_internal.cuh"
#include "tridiag_sqrt.cuh"

namespace rpbd {

constexpr int DOT_BLOCKS = 256;
constexpr int LANCZOS_MAX = 80;

// ---------------------------------------------------------------------------
// vector kernels

// partial[i * gridDim.x + bx] = sum over the block's slice of V_i . w
__global__ void multidot_kernel(int64_t n, const double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                                double* __restrict__ partial)
{
    const int i = blockIdx.y;
    const double* v = V + (int64_t)i * ld;
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        s += v[e] * w[e];
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
    }
}

// out[i] (+)= sum_b partial[i * nb + b]; one block per i
__global__ void reduce_partials_kernel(int nblocks, const double* __restrict__ partial, double* __restrict__ out,
                                       int accumulate)
{
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)i * nblocks + b];
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[i] = accumulate ? out[i] + s : s;
    }
}

// w -= sum_i h[i] V_i
__global__ void multiaxpy_kernel(int64_t n, const double* __restrict__ V, int64_t ld, int nv,
                                 const double* __restrict__ h, double* __restrict__ w)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = w[e];
        for (int i = 0; i < nv; ++i) s -= h[i] * V[(int64_t)i * ld + e];
        w[e] = s;
    }
}

// out = scale * sum_i y[i] V_i   (scale = *scale_dev when scale_dev != NULL)
__global__ void lincomb_kernel(int64_t n, const double* __restrict__ V, int64_t ld, int nv,
                               const double* __restrict__ y, double scale, const double* __restrict__ scale_dev,
                               double* __restrict__ out)
{
    const double sc = scale_dev ? scale * scale_dev[0] : scale;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < nv; ++i) s += y[i] * V[(int64_t)i * ld + e];
        out[e] = sc * s;
    }
}

// out = x / sqrt(*nrm2)  (or 0 when the norm vanishes)
__global__ void normalize_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ nrm2,
                                 double* __restrict__ out)
{
    const double nv = sqrt(nrm2[0]);
    const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = x[e] * inv;
}

__global__ void add_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] += x[e];
}

// saddle operator pieces: lamout -= K U ; Uout = -K^T lam (done with launch_KT then negate)
__global__ void K_sub_kernel(int64_t nb, int nper, const double* __restrict__ r, const double* __restrict__ q,
                             const double* __restrict__ U, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = nb * nper;
    if (i >= n) return;
    const int64_t p = i / nper;
    const double d0 = r[i] - q[3 * p], d1 = r[n + i] - q[3 * p + 1], d2 = r[2 * n + i] - q[3 * p + 2];
    const double* u = U + 6 * p;
    out[i] -= u[0] + (u[4] * d2 - u[5] * d1);
    out[n + i] -= u[1] + (u[5] * d0 - u[3] * d2);
    out[2 * n + i] -= u[2] + (u[3] * d1 - u[4] * d0);
}

__global__ void negate_kernel(int64_t n, double* __restrict__ x)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = -x[e];
}

static unsigned vgrid(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

// h[0..nv) = V^T w (accumulate != 0: h += V^T w)
static int multidot(rpbd_handle* h, int64_t n, const double* V, int64_t ld, int nv, const double* w, double* out,
                    int accumulate, double* partial, cudaStream_t st)
{
    multidot_kernel<<<dim3(DOT_BLOCKS, nv), 256, 0, st>>>(n, V, ld, w, partial); count_launch();
    reduce_partials_kernel<<<nv, 256, 0, st>>>(DOT_BLOCKS, partial, out, accumulate); count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

// ---------------------------------------------------------------------------
// small GMRES kernels (one thread)

// H column j from hcol[0..j] and hcol[j+1] = |w|^2; rotations; residual estimate
__global__ void gmres_column_kernel(int j, int mdim, const double* __restrict__ hcol, double* __restrict__ H,
                                    double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                                    const double* __restrict__ bnorm, double* __restrict__ res)
{
    double* col = H + (int64_t)j * (mdim + 1);
    for (int i = 0; i <= j; ++i) col[i] = hcol[i];
    col[j + 1] = sqrt(hcol[j + 1]);
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    if (den > 0.0) {
        cs[j] = col[j] / den;
        sn[j] = col[j + 1] / den;
    } else {
        cs[j] = 1.0;
        sn[j] = 0.0;
    }
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    res[0] = fabs(g[j + 1]) / bnorm[0];
}

// y = H(0:k,0:k)^-1 g(0:k), upper triangular back substitution
__global__ void gmres_backsolve_kernel(int k, int mdim, const double* __restrict__ H, const double* __restrict__ g,
                                       double* __restrict__ y)
{
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= H[(int64_t)c * (mdim + 1) + i] * y[c];
        const double d = H[(int64_t)i * (mdim + 1) + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// g = [sqrt(nrm2), 0, ...]; bnorm (when first) = sqrt(nrm2); res = sqrt(nrm2)/bnorm
__global__ void gmres_start_kernel(int mdim, const double* __restrict__ nrm2, double* __restrict__ g,
                                   double* __restrict__ bnorm, int first, double* __restrict__ res)
{
    const double b = sqrt(nrm2[0]);
    for (int i = 0; i <= mdim; ++i) g[i] = 0.0;
    g[0] = b;
    if (first) bnorm[0] = b;
    res[0] = bnorm[0] > 0.0 ? b / bnorm[0] : 0.0;
}

// ---------------------------------------------------------------------------
// Lanczos small kernels

// alpha/beta bookkeeping: alpha[m] = h[m] (after both passes), beta[m] = |w|
__global__ void lanczos_coef_kernel(int m, const double* __restrict__ h, const double* __restrict__ nrm2,
                                    double* __restrict__ alpha, double* __restrict__ beta)
{
    alpha[m] = h[m];
    beta[m] = sqrt(nrm2[0]);
}

// One warp: c = T^{1/2} e_1 of the (m+1) x (m+1) tridiagonal T
// (tridiag_sqrt.cuh), change = |c - [c_prev; 0]| / |c|.
__global__ void lanczos_sqrt_kernel(int m1, const double* __restrict__ alpha, const double* __restrict__ beta,
                                    double* __restrict__ c, double* __restrict__ c_prev, double* __restrict__ change)
{
    extern __shared__ double sm[];
    const int lane = threadIdx.x;
    tridiag_sqrt_e1(m1, alpha, beta, sm, c);
    double nc = 0.0, nd = 0.0;
    for (int i = lane; i < m1; i += 32) {
        const double v = c[i];
        const double prev = i < m1 - 1 ? c_prev[i] : 0.0;
        nc += v * v;
        nd += (v - prev) * (v - prev);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    __syncwarp();
    for (int i = lane; i < m1; i += 32) c_prev[i] = c[i];
    if (lane == 0) change[0] = nc > 0.0 ? sqrt(nd / nc) : 0.0;
}

// ---------------------------------------------------------------------------
// host helpers

static int check_flag(rpbd_handle* h, cudaStream_t st)
{
    int flag = 0;
    RPBD_CU(h, cudaMemcpyAsync(&flag, h->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RPBD_CU(h, cudaStreamSynchronize(st));
    if (flag == 1) return set_error(h, RPBD_TIMEOUT, "a pair kernel's bounded wait expired");
    return RPBD_OK;
}

// small device scratch layout (doubles)
struct Small {
    double* base;
    int mdim;
    double* H() { return base; }                                   // (mdim+1) * mdim
    double* cs() { return H() + (int64_t)(mdim + 1) * mdim; }      // mdim
    double* sn() { return cs() + mdim; }                           // mdim
    double* g() { return sn() + mdim; }                            // mdim + 1
    double* y() { return g() + mdim + 1; }                         // mdim + 1
    double* hcol() { return y() + mdim + 1; }                      // mdim + 2
    double* scal() { return hcol() + mdim + 2; }                   // 8 scalars
    double* partial() { return scal() + 8; }                       // DOT_BLOCKS * (mdim + 2)
    static size_t count(int mdim)
    {
        return (size_t)(mdim + 1) * mdim + 2 * mdim + 3 * (mdim + 1) + 1 + 8 + (size_t)DOT_BLOCKS * (mdim + 2);
    }
};

// ---------------------------------------------------------------------------
// Lanczos

// Several Lanczos processes (different W, same M and preconditioner) advance
// in lockstep: each iteration gathers the active processes' vectors into one
// multi-RHS matvec and reads every process's scalars with one
// synchronisation.  Each process keeps its own basis, tridiagonal matrix and
// stopping test, so the answers are those of separate runs.
struct LanczosProc {
    const double* W;
    double* out;
    double *V, *z, *y, *w, *alpha, *beta, *cvec, *cprev, *sc;  // sc: [0] |W|^2, [1] |w|^2, [2] change
    Small S{nullptr, 0};
    double W2 = 0.0, change = INFINITY;
    int m = 0, matvecs = 0, status = RPBD_NOT_CONVERGED;
    bool active = false;
};

int lanczos_multi_impl(rpbd_handle* h, int64_t n, const double* r, int nsys, const double* const* W,
                       double* const* out, double tol, int max_iter, int dtype, int use_precond, rpbd_stats* stats,
                       cudaStream_t st)
{
    if (n <= 0) return set_error(h, RPBD_BAD_ARG, "lanczos: n <= 0");
    if (nsys < 1 || nsys > 4) return set_error(h, RPBD_BAD_ARG, "lanczos: 1..4 vectors");
    if (max_iter < 1 || max_iter > LANCZOS_MAX) return set_error(h, RPBD_BAD_ARG, "lanczos: max_iter must be in 1..80");
    if (use_precond && (!h->prec_valid || h->prec_nb * h->prec_nper != n))
        return set_error(h, RPBD_BAD_ARG, "lanczos: preconditioner not built for these blobs");
    if (!r) return set_error(h, RPBD_BAD_ARG, "lanczos: null positions");
    RPBD_TRY(check_finite(h, 3 * n, r, st));
    const int64_t len = 3 * n;
    const int mdim = LANCZOS_MAX + 1;
    const size_t small_count = Small::count(mdim) + 4 * (size_t)mdim;
    double *Vall, *vall, *small, *mv = nullptr;
    RPBD_TRY(ensure_t(h, BUF_KRYLOV, (size_t)nsys * (max_iter + 1) * len, &Vall));
    RPBD_TRY(ensure_t(h, BUF_VEC, (size_t)nsys * 3 * len, &vall));
    RPBD_TRY(ensure_t(h, BUF_SMALL, (size_t)nsys * small_count, &small));
    if (nsys > 1) RPBD_TRY(ensure_t(h, BUF_GMRES_MV, (size_t)2 * nsys * len, &mv));
    if (once_per_device(h, reinterpret_cast<const void*>(lanczos_sqrt_kernel)))
        RPBD_CU(h, cudaFuncSetAttribute(lanczos_sqrt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        tridiag_sqrt_smem_doubles(LANCZOS_MAX + 1) * (int)sizeof(double)));
    RPBD_CU(h, cudaMemsetAsync(h->dev_flag, 0, sizeof(int), st));
    const unsigned g = vgrid(len);
    LanczosProc P[4];
    for (int s = 0; s < nsys; ++s) {
        LanczosProc& p = P[s];
        if (!W[s] || !out[s]) return set_error(h, RPBD_BAD_ARG, "lanczos: null pointer");
        p.W = W[s];
        p.out = out[s];
        p.V = Vall + (int64_t)s * (max_iter + 1) * len;
        p.z = vall + (int64_t)s * 3 * len;
        p.y = p.z + len;
        p.w = p.z + 2 * len;
        p.S = Small{small + (int64_t)s * small_count, mdim};
        p.alpha = p.S.partial() + (size_t)DOT_BLOCKS * (mdim + 2);
        p.beta = p.alpha + mdim;
        p.cvec = p.beta + mdim;
        p.cprev = p.cvec + mdim;
        p.sc = p.S.scal();
        RPBD_CU(h, cudaMemsetAsync(p.cprev, 0, sizeof(double) * mdim, st));
        RPBD_TRY(multidot(h, len, p.W, 0, 1, p.W, &p.sc[0], 0, p.S.partial(), st));
        normalize_kernel<<<g, 256, 0, st>>>(len, p.W, &p.sc[0], p.V); count_launch();
        RPBD_CU(h, cudaMemcpyAsync(h->host_small + s, &p.sc[0], sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    RPBD_LAUNCH_CHECK(h);
    RPBD_CU(h, cudaStreamSynchronize(st));
    for (int s = 0; s < nsys; ++s) {
        P[s].W2 = h->host_small[s];
        if (P[s].W2 > 0.0) {
            P[s].active = true;
        } else {
            RPBD_CU(h, cudaMemsetAsync(P[s].out, 0, sizeof(double) * len, st));
            P[s].status = RPBD_OK;
        }
    }
    for (;;) {
        int act[4], k = 0;
        for (int s = 0; s < nsys; ++s)
            if (P[s].active) act[k++] = s;
        if (k == 0) break;
        // w = G v_m for every active process, one k-RHS matvec
        for (int a = 0; a < k; ++a) {
            LanczosProc& p = P[act[a]];
            const double* vm = p.V + (int64_t)p.m * len;
            double* dst = k == 1 ? p.z : mv + (int64_t)a * len;
            if (use_precond) RPBD_TRY(precond_apply_impl(h, 2, vm, dst, st));
            else RPBD_CU(h, cudaMemcpyAsync(dst, vm, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
        }
        if (k == 1) {
            LanczosProc& p = P[act[0]];
            RPBD_TRY(mobility_apply_impl(h, n, r, p.z, p.y, 1, dtype, true, st));
        } else {
            RPBD_TRY(mobility_apply_impl(h, n, r, mv, mv + (int64_t)k * len, k, dtype, true, st));
        }
        for (int a = 0; a < k; ++a) {
            LanczosProc& p = P[act[a]];
            const double* my = k == 1 ? p.y : mv + (int64_t)(k + a) * len;
            if (use_precond) RPBD_TRY(precond_apply_impl(h, 1, my, p.w, st));
            else RPBD_CU(h, cudaMemcpyAsync(p.w, my, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
            ++p.matvecs;
            // full reorthogonalisation, classical Gram-Schmidt twice
            const int m = p.m;
            RPBD_TRY(multidot(h, len, p.V, len, m + 1, p.w, p.S.hcol(), 0, p.S.partial(), st));
            multiaxpy_kernel<<<g, 256, 0, st>>>(len, p.V, len, m + 1, p.S.hcol(), p.w); count_launch();
            RPBD_TRY(multidot(h, len, p.V, len, m + 1, p.w, p.S.y(), 0, p.S.partial(), st));
            multiaxpy_kernel<<<g, 256, 0, st>>>(len, p.V, len, m + 1, p.S.y(), p.w); count_launch();
            add_kernel<<<1, 128, 0, st>>>(m + 1, p.S.y(), p.S.hcol()); count_launch();
            RPBD_TRY(multidot(h, len, p.w, 0, 1, p.w, &p.sc[1], 0, p.S.partial(), st));
            lanczos_coef_kernel<<<1, 1, 0, st>>>(m, p.S.hcol(), &p.sc[1], p.alpha, p.beta); count_launch();
            const int m1 = m + 1;
            lanczos_sqrt_kernel<<<1, 32, tridiag_sqrt_smem_doubles(m1) * sizeof(double), st>>>(
                m1, p.alpha, p.beta, p.cvec, p.cprev, &p.sc[2]);
            count_launch();
            normalize_kernel<<<g, 256, 0, st>>>(len, p.w, &p.sc[1], p.V + (int64_t)(m + 1) * len); count_launch();
            RPBD_CU(h, cudaMemcpyAsync(h->host_small + 2 * a, &p.sc[1], 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        RPBD_LAUNCH_CHECK(h);
        RPBD_CU(h, cudaStreamSynchronize(st));
        for (int a = 0; a < k; ++a) {
            LanczosProc& p = P[act[a]];
            const double w2 = h->host_small[2 * a], ch = h->host_small[2 * a + 1];
            bool stop = false;
            if (p.m >= 1) {
                p.change = ch;
                if (ch < tol) { p.status = RPBD_OK; stop = true; }
            }
            if (!stop && !(w2 > 1e-300 * p.W2)) { p.status = RPBD_OK; stop = true; }  // invariant subspace: exact
            if (!stop && p.m + 1 >= max_iter) stop = true;
            if (stop) {
                p.active = false;
                // y = |W| V c, out = L y
                const int nv = p.m + 1;
                lincomb_kernel<<<g, 256, 0, st>>>(len, p.V, len, nv, p.cvec, std::sqrt(p.W2), nullptr,
                                                  use_precond ? p.y : p.out);
                count_launch();
                if (use_precond) RPBD_TRY(precond_apply_impl(h, 0, p.y, p.out, st));
            } else {
                ++p.m;
            }
        }
        RPBD_LAUNCH_CHECK(h);
    }
    RPBD_TRY(check_flag(h, st));
    bool all_ok = true;
    for (int s = 0; s < nsys; ++s) {
        const LanczosProc& p = P[s];
        if (stats)
            stats[s] = p.W2 > 0.0 ? rpbd_stats{p.m + 1, p.matvecs, p.m >= 1 ? p.change : 0.0, p.status}
                                  : rpbd_stats{0, 0, 0.0, RPBD_OK};
        all_ok = all_ok && p.status == RPBD_OK;
    }
    return all_ok ? RPBD_OK : RPBD_NOT_CONVERGED;
}

int lanczos_impl(rpbd_handle* h, int64_t n, const double* r, const double* W, double* out, double tol, int max_iter,
                 int dtype, int use_precond, rpbd_stats* stats, cudaStream_t st)
{
    return lanczos_multi_impl(h, n, r, 1, &W, &out, tol, max_iter, dtype, use_precond, stats, st);
}

// ---------------------------------------------------------------------------
// GMRES on the saddle system
//
// Each GMRES process is a small state machine; a driver advances several
// processes that share the positions (same M, K and preconditioner) in
// lockstep, so that their matvecs go out as one multi-RHS launch (k =
// number of processes needing one), and reads every process's residual with
// one host synchronisation per iteration.

// out = [M lam - K U; -K^T lam] given Mlam = M lam already in out[0:3n]
static void saddle_finish(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* x,
                          double* out, cudaStream_t st)
{
    const int64_t n = nb * nper;
    K_sub_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nb, nper, r, q, x + 3 * n, out); count_launch();
    launch_KT(nb, nper, r, q, x, out + 3 * n, st);
    negate_kernel<<<vgrid(6 * nb), 256, 0, st>>>(6 * nb, out + 3 * n); count_launch();
}

struct GmresProc {
    GmresProblem pb;
    double *V, *x, *b, *w, *z, *sc;
    Small S{nullptr, 0};
    enum Phase { NEED_RESID, NEED_ARNOLDI, READ_START, READ_ITER, DONE } phase = DONE;
    int j = 0, total = 0, matvecs = 0, status = RPBD_NOT_CONVERGED;
    double res = 1.0;
    const double* req = nullptr;  // vector whose saddle product is wanted
};

int gmres_multi_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, int nsys,
                     const GmresProblem* probs, int restart, int dtype, int build_precond, rpbd_stats* stats,
                     cudaStream_t st)
{
    if (nb <= 0 || nper <= 0) return set_error(h, RPBD_BAD_ARG, "gmres: no bodies");
    if (restart < 1 || restart > 200) return set_error(h, RPBD_BAD_ARG, "gmres: bad restart");
    if (nsys < 1 || nsys > 4) return set_error(h, RPBD_BAD_ARG, "gmres: 1..4 systems");
    for (int s = 0; s < nsys; ++s)
        if (probs[s].max_iter < 1 || !probs[s].lambda || !probs[s].U)
            return set_error(h, RPBD_BAD_ARG, "gmres: bad max_iter or null output");
    const int64_t n = nb * nper;
    if (!r || !q) return set_error(h, RPBD_BAD_ARG, "gmres: null positions");
    RPBD_TRY(check_finite(h, 3 * (int64_t)nb * nper, r, st));
    if (build_precond) RPBD_TRY(precond_build_impl(h, nb, nper, r, q, st));
    if (!h->prec_valid || h->prec_nb != nb || h->prec_nper != nper)
        return set_error(h, RPBD_BAD_ARG, "gmres: preconditioner not built for these bodies");
    const int64_t len = 3 * n + 6 * nb;
    const int mdim = restart;
    double *Vall, *vall, *small, *mv = nullptr;
    RPBD_TRY(ensure_t(h, BUF_KRYLOV, (size_t)nsys * (mdim + 1) * len, &Vall));
    RPBD_TRY(ensure_t(h, BUF_VEC, (size_t)nsys * 4 * len, &vall));
    RPBD_TRY(ensure_t(h, BUF_SMALL, (size_t)nsys * Small::count(mdim), &small));
    if (nsys > 1) RPBD_TRY(ensure_t(h, BUF_GMRES_MV, (size_t)2 * nsys * 3 * n, &mv));
    GmresProc P[4];
    const unsigned g = vgrid(len);
    RPBD_CU(h, cudaMemsetAsync(h->dev_flag, 0, sizeof(int), st));

    // r0 = w: |r0|, g, residual estimate, v_0 (first: |b| = |r0|)
    auto begin_cycle = [&](GmresProc& p, int first) -> int {
        RPBD_TRY(multidot(h, len, p.w, 0, 1, p.w, &p.sc[0], 0, p.S.partial(), st));
        gmres_start_kernel<<<1, 1, 0, st>>>(mdim, &p.sc[0], p.S.g(), &p.sc[1], first, &p.sc[2]); count_launch();
        normalize_kernel<<<g, 256, 0, st>>>(len, p.w, &p.sc[0], p.V); count_launch();
        RPBD_LAUNCH_CHECK(h);
        p.phase = GmresProc::READ_START;
        return RPBD_OK;
    };
    // x += P^-1 V y over the cycle's jn Arnoldi vectors
    auto end_cycle = [&](GmresProc& p, int jn) -> int {
        gmres_backsolve_kernel<<<1, 1, 0, st>>>(jn, mdim, p.S.H(), p.S.g(), p.S.y()); count_launch();
        lincomb_kernel<<<g, 256, 0, st>>>(len, p.V, len, jn, p.S.y(), 1.0, nullptr, p.w); count_launch();
        RPBD_TRY(precond_saddle_impl(h, p.w, p.w + 3 * n, p.z, p.z + 3 * n, st));
        add_kernel<<<g, 256, 0, st>>>(len, p.z, p.x); count_launch();
        RPBD_LAUNCH_CHECK(h);
        return RPBD_OK;
    };
    auto want_arnoldi = [&](GmresProc& p) -> int {
        RPBD_TRY(precond_saddle_impl(h, p.V + (int64_t)p.j * len, p.V + (int64_t)p.j * len + 3 * n, p.z, p.z + 3 * n, st));
        p.req = p.z;
        p.phase = GmresProc::NEED_ARNOLDI;
        return RPBD_OK;
    };

    for (int s = 0; s < nsys; ++s) {
        GmresProc& p = P[s];
        p.pb = probs[s];
        p.V = Vall + (int64_t)s * (mdim + 1) * len;
        p.x = vall + (int64_t)s * 4 * len;
        p.b = p.x + len;
        p.w = p.x + 2 * len;
        p.z = p.x + 3 * len;
        p.S = Small{small + (int64_t)s * Small::count(mdim), mdim};
        p.sc = p.S.scal();  // [0] |.|^2, [1] |b|, [2] residual estimate
        // b = [-slip; -FT]
        if (p.pb.slip) launch_scale_copy(3 * n, -1.0, p.pb.slip, p.b, st);
        else RPBD_CU(h, cudaMemsetAsync(p.b, 0, sizeof(double) * 3 * n, st));
        if (p.pb.FT) launch_scale_copy(6 * nb, -1.0, p.pb.FT, p.b + 3 * n, st);
        else RPBD_CU(h, cudaMemsetAsync(p.b + 3 * n, 0, sizeof(double) * 6 * nb, st));
        if (p.pb.warm) {
            // x0 = [lambda; U] as given; |b| is the scale of the stopping test, as for x0 = 0
            RPBD_CU(h, cudaMemcpyAsync(p.x, p.pb.lambda, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
            RPBD_CU(h, cudaMemcpyAsync(p.x + 3 * n, p.pb.U, sizeof(double) * 6 * nb, cudaMemcpyDeviceToDevice, st));
            RPBD_TRY(multidot(h, len, p.b, 0, 1, p.b, &p.sc[0], 0, p.S.partial(), st));
            gmres_start_kernel<<<1, 1, 0, st>>>(mdim, &p.sc[0], p.S.g(), &p.sc[1], 1, &p.sc[2]); count_launch();
            p.req = p.x;
            p.phase = GmresProc::NEED_RESID;
        } else {
            RPBD_CU(h, cudaMemsetAsync(p.x, 0, sizeof(double) * len, st));
            launch_scale_copy(len, 1.0, p.b, p.w, st);
            RPBD_TRY(begin_cycle(p, 1));
        }
    }

    for (;;) {
        // residuals of every process waiting for one: one synchronisation
        int nread = 0;
        for (int s = 0; s < nsys; ++s)
            if (P[s].phase == GmresProc::READ_START || P[s].phase == GmresProc::READ_ITER) {
                RPBD_CU(h, cudaMemcpyAsync(h->host_small + 2 * s, &P[s].sc[1], 2 * sizeof(double),
                                           cudaMemcpyDeviceToHost, st));
                ++nread;
            }
        if (nread) RPBD_CU(h, cudaStreamSynchronize(st));
        for (int s = 0; s < nsys; ++s) {
            GmresProc& p = P[s];
            const double bn = h->host_small[2 * s], res = h->host_small[2 * s + 1];
            if (p.phase == GmresProc::READ_START) {
                p.res = res;
                if (!(bn > 0.0)) {  // zero right-hand side: zero solution
                    RPBD_CU(h, cudaMemsetAsync(p.x, 0, sizeof(double) * len, st));
                    p.res = 0.0;
                    p.status = RPBD_OK;
                    p.phase = GmresProc::DONE;
                } else if (res <= p.pb.tol) {
                    p.status = RPBD_OK;
                    p.phase = GmresProc::DONE;
                } else if (p.total >= p.pb.max_iter) {
                    p.phase = GmresProc::DONE;
                } else {
                    p.j = 0;
                    RPBD_TRY(want_arnoldi(p));
                }
            } else if (p.phase == GmresProc::READ_ITER) {
                p.res = res;
                ++p.total;
                const int jn = p.j + 1;
                if (res <= p.pb.tol || jn == mdim || p.total >= p.pb.max_iter) {
                    RPBD_TRY(end_cycle(p, jn));
                    if (res <= p.pb.tol) {
                        p.status = RPBD_OK;
                        p.phase = GmresProc::DONE;
                    } else if (p.total >= p.pb.max_iter) {
                        p.phase = GmresProc::DONE;
                    } else {
                        p.req = p.x;  // restart: r0 = b - A x
                        p.phase = GmresProc::NEED_RESID;
                    }
                } else {
                    p.j = jn;
                    RPBD_TRY(want_arnoldi(p));
                }
            }
        }
        // one matvec for every process that needs one
        int act[4], k = 0;
        for (int s = 0; s < nsys; ++s)
            if (P[s].phase == GmresProc::NEED_RESID || P[s].phase == GmresProc::NEED_ARNOLDI) act[k++] = s;
        if (k == 0) break;
        if (k == 1) {
            GmresProc& p = P[act[0]];
            RPBD_TRY(mobility_apply_impl(h, n, r, p.req, p.w, 1, dtype, true, st));
        } else {
            double* Fm = mv;
            double* Um = mv + (int64_t)k * 3 * n;
            for (int a = 0; a < k; ++a)
                RPBD_CU(h, cudaMemcpyAsync(Fm + (int64_t)a * 3 * n, P[act[a]].req, sizeof(double) * 3 * n,
                                           cudaMemcpyDeviceToDevice, st));
            RPBD_TRY(mobility_apply_impl(h, n, r, Fm, Um, k, dtype, true, st));
            for (int a = 0; a < k; ++a)
                RPBD_CU(h, cudaMemcpyAsync(P[act[a]].w, Um + (int64_t)a * 3 * n, sizeof(double) * 3 * n,
                                           cudaMemcpyDeviceToDevice, st));
        }
        for (int a = 0; a < k; ++a) {
            GmresProc& p = P[act[a]];
            saddle_finish(h, nb, nper, r, q, p.req, p.w, st);
            ++p.matvecs;
            if (p.phase == GmresProc::NEED_RESID) {
                launch_axpby(len, 1.0, p.b, -1.0, p.w, p.w, st);
                RPBD_TRY(begin_cycle(p, 0));
            } else {
                // Arnoldi: classical Gram-Schmidt twice, Givens, residual estimate
                const int j = p.j;
                RPBD_TRY(multidot(h, len, p.V, len, j + 1, p.w, p.S.hcol(), 0, p.S.partial(), st));
                multiaxpy_kernel<<<g, 256, 0, st>>>(len, p.V, len, j + 1, p.S.hcol(), p.w); count_launch();
                RPBD_TRY(multidot(h, len, p.V, len, j + 1, p.w, p.S.y(), 0, p.S.partial(), st));
                multiaxpy_kernel<<<g, 256, 0, st>>>(len, p.V, len, j + 1, p.S.y(), p.w); count_launch();
                add_kernel<<<1, 256, 0, st>>>(j + 1, p.S.y(), p.S.hcol()); count_launch();
                RPBD_TRY(multidot(h, len, p.w, 0, 1, p.w, p.S.hcol() + j + 1, 0, p.S.partial(), st));
                normalize_kernel<<<g, 256, 0, st>>>(len, p.w, p.S.hcol() + j + 1, p.V + (int64_t)(j + 1) * len);
                count_launch();
                gmres_column_kernel<<<1, 1, 0, st>>>(j, mdim, p.S.hcol(), p.S.H(), p.S.cs(), p.S.sn(), p.S.g(),
                                                      &p.sc[1], &p.sc[2]);
                count_launch();
                RPBD_LAUNCH_CHECK(h);
                p.phase = GmresProc::READ_ITER;
            }
        }
    }
    RPBD_TRY(check_flag(h, st));
    bool all_ok = true;
    for (int s = 0; s < nsys; ++s) {
        GmresProc& p = P[s];
        RPBD_CU(h, cudaMemcpyAsync(p.pb.lambda, p.x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
        RPBD_CU(h, cudaMemcpyAsync(p.pb.U, p.x + 3 * n, sizeof(double) * 6 * nb, cudaMemcpyDeviceToDevice, st));
        if (stats) stats[s] = rpbd_stats{p.total, p.matvecs, p.res, p.status};
        all_ok = all_ok && p.status == RPBD_OK;
    }
    return all_ok ? RPBD_OK : RPBD_NOT_CONVERGED;
}

int gmres_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* slip,
               const double* FT, double* lambda, double* U, double tol, int max_iter, int restart, int dtype,
               int build_precond, int warm, rpbd_stats* stats, cudaStream_t st)
{
    const GmresProblem pb{slip, FT, lambda, U, tol, max_iter, warm};
    return gmres_multi_impl(h, nb, nper, r, q, 1, &pb, restart, dtype, build_precond, stats, st);
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

int rpbd_lanczos_sqrt_apply(rpbd_handle* h, int64_t n, const double* r, const double* W, double* out, double tol,
                            int max_iter, int dtype, int use_precond, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!r || !W || !out) return set_error(h, RPBD_BAD_ARG, "lanczos: null pointer");
    if (!(tol > 0)) return set_error(h, RPBD_BAD_ARG, "lanczos: tol must be > 0");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "lanczos: bad dtype");
    return lanczos_impl(h, n, r, W, out, tol, max_iter, dtype, use_precond, stats,
                        reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_lanczos_sqrt_apply_multi(rpbd_handle* h, int64_t n, const double* r, int nsys, const double* const* W,
                                  double* const* out, double tol, int max_iter, int dtype, int use_precond,
                                  rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!r || !W || !out) return set_error(h, RPBD_BAD_ARG, "lanczos_multi: null pointer");
    if (!(tol > 0)) return set_error(h, RPBD_BAD_ARG, "lanczos_multi: tol must be > 0");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "lanczos_multi: bad dtype");
    return lanczos_multi_impl(h, n, r, nsys, W, out, tol, max_iter, dtype, use_precond, stats,
                              reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_gmres_rigid_solve_multi(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, int nsys,
                                 const double* const* slip, const double* const* FT, double* const* lambda,
                                 double* const* U, double tol, int max_iter, int restart, int dtype,
                                 int build_precond, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!r || !q || nsys < 1 || nsys > 4 || !slip || !FT || !lambda || !U)
        return set_error(h, RPBD_BAD_ARG, "gmres_multi: bad arguments");
    if (!(tol > 0)) return set_error(h, RPBD_BAD_ARG, "gmres_multi: tol must be > 0");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "gmres_multi: bad dtype");
    GmresProblem pb[4];
    for (int s = 0; s < nsys; ++s) {
        if (!lambda[s] || !U[s]) return set_error(h, RPBD_BAD_ARG, "gmres_multi: null output");
        pb[s] = GmresProblem{slip[s], FT[s], lambda[s], U[s], tol, max_iter, 0};
    }
    return gmres_multi_impl(h, nb, nper, r, q, nsys, pb, restart, dtype, build_precond, stats,
                            reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_gmres_rigid_solve(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* slip,
                           const double* FT, double* lambda, double* U, double tol, int max_iter, int restart,
                           int dtype, int build_precond, int warm_start, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!r || !q || !lambda || !U) return set_error(h, RPBD_BAD_ARG, "gmres: null pointer");
    if (!(tol > 0)) return set_error(h, RPBD_BAD_ARG, "gmres: tol must be > 0");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "gmres: bad dtype");
    return gmres_impl(h, nb, nper, r, q, slip, FT, lambda, U, tol, max_iter, restart, dtype, build_precond,
                      warm_start ? 1 : 0, stats, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
