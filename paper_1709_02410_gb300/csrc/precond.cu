// Body-block-diagonal preconditioner (Sec. 2.2).
//
// Interactions between distinct bodies are dropped: M~(pq) = delta_pq M(pp),
// with M(pp) the dense FP64 blob mobility of body p's blobs alone (wall and
// overlap regularisation included).  One CTA per body builds, in shared
// memory:
//   L_p      Cholesky factor, M(pp) = L_p L_p^T      (Lanczos: L = M~^{1/2})
//   L_p^-1   its inverse (triangular)
//   M(pp)^-1 = L_p^-T L_p^-1
//   M(pp)^-1 K_p and N_p = (K_p^T M(pp)^-1 K_p)^-1  (exact body-block solve
//            of the saddle system, eqs. saddle and N_def per body)
// and stores them column-major (element (i, j) at j*m + i, m = 3 nper, blob-
// interleaved rows 3b + c).
#include <cuda_runtime.h>

#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"

namespace rpbd {

constexpr int PREC_THREADS = 128;
constexpr int PREC_MAX_M = 96;  // 3 * nper <= 96

template <bool WALL, bool PER>
__global__ void __launch_bounds__(PREC_THREADS) prec_build_kernel(int nper, int64_t n, const double* __restrict__ r,
                                                                  const double* __restrict__ q, double a, double s_min,
                                                                  double Lx, double Ly,
                                                                  double inv8pieta, double* __restrict__ gL,
                                                                  double* __restrict__ gLinv, double* __restrict__ gMinv,
                                                                  double* __restrict__ gMinvK, double* __restrict__ gN,
                                                                  int* __restrict__ err)
{
    extern __shared__ double sm[];
    const int m = 3 * nper;
    const int64_t p = blockIdx.x;
    const int tid = threadIdx.x;
    double* A = sm;              // m*m: M(pp) -> L (lower)
    double* X = A + m * m;       // m*m: L^-1
    double* B = X + m * m;       // m*6: K_p, then M^-1 K
    double* bx = B + 6 * m;      // nper * 5: x, y, zt, s, (z - q)
    __shared__ double S6[36];
    __shared__ double NN[36];
    __shared__ int spd_fail;
    if (tid == 0) spd_fail = 0;
    for (int b = tid; b < nper; b += blockDim.x) {
        const int64_t i = p * nper + b;
        const double z = r[2 * n + i];
        double zt = z, s = 1.0;
        if (WALL) {
            zt = z > a ? z : a;
            const double t = z / a;
            s = t >= 1.0 ? 1.0 : (t <= s_min ? s_min : t);
        }
        bx[5 * b + 0] = r[i];
        bx[5 * b + 1] = r[n + i];
        bx[5 * b + 2] = zt;
        bx[5 * b + 3] = s;
        bx[5 * b + 4] = z;
    }
    __syncthreads();
    // 1. dense M(pp)
    const PairConst<double> pc = PairConst<double>::make(a, Lx, Ly);
    for (int pr = tid; pr < nper * nper; pr += blockDim.x) {
        const int bi = pr / nper, bj = pr % nper;
        const double* ti = bx + 5 * bi;
        const double* tj = bx + 5 * bj;
        double M[9];
        pair_block_images<double, double, WALL, PER>(ti[0] - tj[0], ti[1] - tj[1], ti[2] - tj[2], ti[2], tj[2], pc, M[0], M[1],
                                         M[2], M[4], M[5], M[6], M[7], M[8]);
        M[3] = M[1];
        const double sc = ti[3] * tj[3] * inv8pieta;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) A[(3 * bj + d) * m + 3 * bi + c] = sc * M[c * 3 + d];
    }
    __syncthreads();
    // 2. Cholesky (right-looking, lower triangle, column-major)
    for (int k = 0; k < m; ++k) {
        if (tid == 0) {
            const double dkk = A[k * m + k];
            if (!(dkk > 0.0)) spd_fail = 1;
            A[k * m + k] = sqrt(dkk > 0.0 ? dkk : 1e-300);
        }
        __syncthreads();
        const double lkk = A[k * m + k];
        for (int i = k + 1 + tid; i < m; i += blockDim.x) A[k * m + i] /= lkk;
        __syncthreads();
        const int rem = m - k - 1;
        for (int e = tid; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j <= i) A[j * m + i] -= A[k * m + i] * A[k * m + j];
        }
        __syncthreads();
    }
    // zero the strict upper triangle
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        if (j > i) A[e] = 0.0;
    }
    __syncthreads();
    // 3. X = L^-1: thread j solves L x = e_j by forward substitution
    for (int j = tid; j < m; j += blockDim.x) {
        for (int i = 0; i < m; ++i) {
            if (i < j) { X[j * m + i] = 0.0; continue; }
            double v = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) v -= A[k * m + i] * X[j * m + k];
            X[j * m + i] = v / A[i * m + i];
        }
    }
    __syncthreads();
    // 4. store L and L^-1; M^-1 = X^T X
    double* L_out = gL + p * m * m;
    double* Li_out = gLinv + p * m * m;
    double* Mi_out = gMinv + p * m * m;
    for (int e = tid; e < m * m; e += blockDim.x) {
        L_out[e] = A[e];
        Li_out[e] = X[e];
    }
    __syncthreads();
    // reuse A for M^-1
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e % m, j = e / m;
        const int k0 = i > j ? i : j;
        double v = 0.0;
        for (int k = k0; k < m; ++k) v += X[i * m + k] * X[j * m + k];
        A[e] = v;
    }
    __syncthreads();
    // 5. K_p (m x 6), column-major
    const double q0 = q[3 * p], q1 = q[3 * p + 1], q2 = q[3 * p + 2];
    for (int b = tid; b < nper; b += blockDim.x) {
        const int64_t i = p * nper + b;
        const double d0 = r[i] - q0, d1 = r[n + i] - q1, d2 = r[2 * n + i] - q2;
        // rows 3b + c; u part identity, omega part -[d]_x
        const double Kr[3][6] = {{1, 0, 0, 0, d2, -d1}, {0, 1, 0, -d2, 0, d0}, {0, 0, 1, d1, -d0, 0}};
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int e = 0; e < 6; ++e) X[e * m + 3 * b + c] = Kr[c][e];  // X reused for K
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) Mi_out[e] = A[e];
    // B = M^-1 K
    for (int e = tid; e < 6 * m; e += blockDim.x) {
        const int i = e % m, c = e / m;
        double v = 0.0;
        for (int k = 0; k < m; ++k) v += A[k * m + i] * X[c * m + k];
        B[c * m + i] = v;
    }
    __syncthreads();
    for (int e = tid; e < 6 * m; e += blockDim.x) gMinvK[p * 6 * m + e] = B[e];
    // S6 = K^T M^-1 K
    for (int e = tid; e < 36; e += blockDim.x) {
        const int a6 = e % 6, b6 = e / 6;
        double v = 0.0;
        for (int k = 0; k < m; ++k) v += X[a6 * m + k] * B[b6 * m + k];
        S6[e] = v;
    }
    __syncthreads();
    // 6. N_p = S6^-1 by Gauss-Jordan with partial pivoting (one thread)
    if (tid == 0) {
        double Aug[6][12];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                Aug[i][j] = 0.5 * (S6[j * 6 + i] + S6[i * 6 + j]);
                Aug[i][6 + j] = (i == j) ? 1.0 : 0.0;
            }
        for (int c = 0; c < 6; ++c) {
            int piv = c;
            for (int i = c + 1; i < 6; ++i)
                if (fabs(Aug[i][c]) > fabs(Aug[piv][c])) piv = i;
            if (piv != c)
                for (int j = 0; j < 12; ++j) {
                    const double t = Aug[c][j];
                    Aug[c][j] = Aug[piv][j];
                    Aug[piv][j] = t;
                }
            const double d = Aug[c][c];
            if (!(fabs(d) > 0.0)) { spd_fail = 1; continue; }
            for (int j = 0; j < 12; ++j) Aug[c][j] /= d;
            for (int i = 0; i < 6; ++i)
                if (i != c) {
                    const double f = Aug[i][c];
                    for (int j = 0; j < 12; ++j) Aug[i][j] -= f * Aug[c][j];
                }
        }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) NN[j * 6 + i] = Aug[i][6 + j];
        if (spd_fail) atomicExch(err, 2);
    }
    __syncthreads();
    for (int e = tid; e < 36; e += blockDim.x) gN[p * 36 + e] = NN[e];
}

// out = A_p x_p per body, A_p one of the stored factors.
// mode 0: L (lower), 1: L^-1 (lower), 2: L^-T, 3: M^-1.  With `active`
// (batches: systems at blob offsets off[0..n_sys]), bodies of inactive
// systems are skipped and their out left as it is.
__global__ void __launch_bounds__(PREC_THREADS) prec_apply_kernel(int mode, int nper, int64_t n,
                                                                  const double* __restrict__ Mat,
                                                                  const double* __restrict__ x, double* __restrict__ out,
                                                                  const int* __restrict__ active,
                                                                  const int64_t* __restrict__ off, int n_sys)
{
    extern __shared__ double sm[];
    const int m = 3 * nper;
    const int64_t p = blockIdx.x;
    if (active) {
        const int64_t i = p * nper;  // the body's first blob; bodies never straddle systems
        int lo = 0, hi = n_sys;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid;
        }
        if (!active[lo]) return;
    }
    double* A = sm;
    double* v = sm + m * m;
    const double* src = Mat + p * m * m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A[e] = src[e];
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const int b = e / 3, c = e % 3;
        v[e] = x[c * n + p * nper + b];
    }
    __syncthreads();
    // row i's sum over its column range [j0, j1) split into `parts` pieces
    // over the CTA's threads, then added in order
    double* part = v + m;  // parts * span
    const int span = (m + 31) & ~31, parts = PREC_THREADS / span;
    const int q = threadIdx.x / span, i = threadIdx.x % span;
    if (q < parts && i < m) {
        const int j0 = mode == 2 ? i : 0, j1 = mode == 2 || mode == 3 ? m : i + 1;
        const int per = (j1 - j0 + parts - 1) / parts;
        const int a0 = j0 + q * per, a1 = a0 + per < j1 ? a0 + per : j1;
        double acc = 0.0;
        if (mode == 2)  // (L^-1)^T: sum_j Linv(j, i) v_j, j >= i
            for (int j = a0; j < a1; ++j) acc += A[i * m + j] * v[j];
        else            // M^-1, or lower triangular (j <= i)
            for (int j = a0; j < a1; ++j) acc += A[j * m + i] * v[j];
        part[q * span + i] = acc;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double acc = part[threadIdx.x];
        for (int q2 = 1; q2 < parts; ++q2) acc += part[q2 * span + threadIdx.x];
        const int b = threadIdx.x / 3, c = threadIdx.x % 3;
        out[c * n + p * nper + b] = acc;
    }
}

// exact body-block saddle solve: [M(pp) -K_p; -K_p^T 0][lam; U] = [a; b]
//   t = (M^-1 K)^T a + b,  U = -N t,  lam = M^-1 a + (M^-1 K) U
// One CTA per body.  M^-1 and M^-1 K are read straight from global memory
// (each entry once, coalesced along the row index); the six dot products of
// t use one warp each with a shuffle reduction, and the m-row product is split
// into column halves over the CTA's threads, then added.
__global__ void __launch_bounds__(PREC_THREADS) prec_saddle_kernel(int nper, int64_t n, const double* __restrict__ Minv,
                                                                   const double* __restrict__ MinvK,
                                                                   const double* __restrict__ N,
                                                                   const double* __restrict__ a,
                                                                   const double* __restrict__ b,
                                                                   double* __restrict__ lam, double* __restrict__ U)
{
    extern __shared__ double sm[];
    const int m = 3 * nper;
    const int64_t p = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = PREC_THREADS / 32;
    const int span = (m + 31) & ~31;           // threads per column part
    const int parts = PREC_THREADS / span;     // >= 1 since m <= PREC_MAX_M <= PREC_THREADS
    double* va = sm;                           // m
    double* part = va + m;                     // parts * span
    __shared__ double t6[6], u6[6];
    const double* A = Minv + p * m * m;        // column-major: (i, j) at j * m + i
    const double* MK = MinvK + p * 6 * m;      // (M^-1 K)^T rows: column c at c * m
    for (int e = tid; e < m; e += PREC_THREADS) {
        const int bb = e / 3, c = e % 3;
        va[e] = a ? a[c * n + p * nper + bb] : 0.0;
    }
    __syncthreads();
    for (int e = warp; e < 6; e += NW) {
        double v = 0.0;
        for (int k = lane; k < m; k += 32) v += MK[e * m + k] * va[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) t6[e] = v + (b ? b[6 * p + e] : 0.0);
    }
    __syncthreads();
    if (tid < 6) {
        double v = 0.0;
        for (int c = 0; c < 6; ++c) v -= N[p * 36 + c * 6 + tid] * t6[c];
        u6[tid] = v;
        U[6 * p + tid] = v;
    }
    __syncthreads();
    const int q = tid / span, i = tid % span;
    if (q < parts && i < m) {
        const int per = (m + parts - 1) / parts;
        const int j0 = q * per, j1 = j0 + per < m ? j0 + per : m;
        double v = 0.0;
        for (int j = j0; j < j1; ++j) v += A[j * m + i] * va[j];
        if (q == 0)
            for (int c = 0; c < 6; ++c) v += MK[c * m + i] * u6[c];
        part[q * span + i] = v;
    }
    __syncthreads();
    if (tid < m) {
        double v = part[tid];
        for (int q2 = 1; q2 < parts; ++q2) v += part[q2 * span + tid];
        const int bb = tid / 3, c = tid % 3;
        lam[c * n + p * nper + bb] = v;
    }
}

int precond_build_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, cudaStream_t st)
{
    if (nb <= 0) return set_error(h, RPBD_BAD_ARG, "precond_build: no bodies");
    const int m = 3 * nper;
    if (nper <= 0 || m > PREC_MAX_M) return set_error(h, RPBD_BAD_ARG, "precond_build: need 1 <= nper <= 32");
    const int64_t n = nb * nper;
    double *L, *Li, *Mi, *MK, *N;
    RPBD_TRY(ensure_t(h, BUF_PREC_L, (size_t)nb * m * m, &L));
    RPBD_TRY(ensure_t(h, BUF_PREC_LINV, (size_t)nb * m * m, &Li));
    RPBD_TRY(ensure_t(h, BUF_PREC_MINV, (size_t)nb * m * m, &Mi));
    RPBD_TRY(ensure_t(h, BUF_PREC_MINVK, (size_t)nb * 6 * m, &MK));
    RPBD_TRY(ensure_t(h, BUF_PREC_N, (size_t)nb * 36, &N));
    const size_t smem = (size_t)(2 * m * m + 6 * m + 5 * nper) * sizeof(double);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    if (once_per_device(h, reinterpret_cast<const void*>(prec_apply_kernel))) {
        const int mx = (2 * PREC_MAX_M * PREC_MAX_M + 6 * PREC_MAX_M + 5 * 32) * (int)sizeof(double);
        RPBD_CU(h, cudaFuncSetAttribute(prec_build_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        RPBD_CU(h, cudaFuncSetAttribute(prec_build_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        RPBD_CU(h, cudaFuncSetAttribute(prec_build_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        const int mx2 = (PREC_MAX_M * PREC_MAX_M + 7 * PREC_MAX_M) * (int)sizeof(double);
        RPBD_CU(h, cudaFuncSetAttribute(prec_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx2));
        RPBD_CU(h, cudaFuncSetAttribute(prec_saddle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx2));
    }
    RPBD_CU(h, cudaMemsetAsync(h->dev_flag, 0, sizeof(int), st));
    const double Lx = h->p.Lx, Ly = h->p.Ly;
    if (Lx > 0.0)
        prec_build_kernel<true, true><<<(unsigned)nb, PREC_THREADS, smem, st>>>(nper, n, r, q, h->p.a, h->p.s_min, Lx, Ly,
                                                                              inv8pieta, L, Li, Mi, MK, N, h->dev_flag);
    else if (h->p.wall)
        prec_build_kernel<true, false><<<(unsigned)nb, PREC_THREADS, smem, st>>>(nper, n, r, q, h->p.a, h->p.s_min, Lx,
                                                                               Ly, inv8pieta, L, Li, Mi, MK, N, h->dev_flag);
    else
        prec_build_kernel<false, false><<<(unsigned)nb, PREC_THREADS, smem, st>>>(nper, n, r, q, h->p.a, h->p.s_min, Lx,
                                                                                Ly, inv8pieta, L, Li, Mi, MK, N, h->dev_flag);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    h->prec_nb = nb;
    h->prec_nper = nper;
    h->prec_valid = true;
    return RPBD_OK;
}

int precond_apply_impl(rpbd_handle* h, int mode, const double* x, double* out, cudaStream_t st, const int* active,
                       const int64_t* off, int n_sys)
{
    if (!h->prec_valid) return set_error(h, RPBD_BAD_ARG, "preconditioner not built");
    if (mode < 0 || mode > 3 || !x || !out) return set_error(h, RPBD_BAD_ARG, "precond_apply: bad arguments");
    const int m = 3 * h->prec_nper;
    const double* Mat = mode == 0 ? (const double*)h->buf[BUF_PREC_L]
                        : mode == 3 ? (const double*)h->buf[BUF_PREC_MINV]
                                    : (const double*)h->buf[BUF_PREC_LINV];
    const size_t smem = (size_t)(m * m + m + PREC_THREADS) * sizeof(double);
    prec_apply_kernel<<<(unsigned)h->prec_nb, PREC_THREADS, smem, st>>>(
        mode, h->prec_nper, h->prec_nb * h->prec_nper, Mat, x, out, active, off, n_sys);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int precond_saddle_impl(rpbd_handle* h, const double* a, const double* b, double* lam, double* U, cudaStream_t st)
{
    if (!h->prec_valid) return set_error(h, RPBD_BAD_ARG, "preconditioner not built");
    const int m = 3 * h->prec_nper;
    const size_t smem = (size_t)(m + PREC_THREADS) * sizeof(double);
    prec_saddle_kernel<<<(unsigned)h->prec_nb, PREC_THREADS, smem, st>>>(
        h->prec_nper, h->prec_nb * h->prec_nper, (const double*)h->buf[BUF_PREC_MINV],
        (const double*)h->buf[BUF_PREC_MINVK], (const double*)h->buf[BUF_PREC_N], a, b, lam, U); count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

int rpbd_precond_build(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!r || !q) return set_error(h, RPBD_BAD_ARG, "precond_build: null pointer");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    RPBD_TRY(precond_build_impl(h, nb, nper, r, q, st));
    int flag = 0;
    RPBD_CU(h, cudaMemcpyAsync(&flag, h->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RPBD_CU(h, cudaStreamSynchronize(st));
    if (flag) {
        h->prec_valid = false;
        return set_error(h, RPBD_BAD_INPUT, "precond_build: a body block is not positive definite");
    }
    return RPBD_OK;
}

int rpbd_precond_apply(rpbd_handle* h, int mode, const double* x, double* out, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    return precond_apply_impl(h, mode, x, out, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
