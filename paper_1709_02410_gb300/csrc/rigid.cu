// Rigid-body kinematics, forces, random numbers and FP64 vector helpers.
//
//  - blob geometry r_i = q_p + R(theta_p) s_i (Sec. 2.1 multiblob model,
//    unit quaternions of App. B.1)
//  - K U = u_p + omega_p x (r_i - q_p) and K^T lambda = (sum lambda_i,
//    sum (r_i - q_p) x lambda_i) (eq. K and the force/torque balance)
//  - Rotate(theta, phi) = [cos(|phi|/2), sin(|phi|/2) phi/|phi|] (x) theta
//    (App. B.1, eq. rotate) for configuration updates Q + s U
//  - forces of Sec. 4: gravity, blob-wall Yukawa repulsion, constant torque
//  - Philox4x32-10 (Salmon et al., SC'11) + Box-Muller normals
#include <cuda_runtime.h>

#include <type_traits>

#include "rpbd_internal.cuh"

namespace rpbd {

__device__ __forceinline__ void quat_rot(const double* th, double R[3][3])
{
    const double s = th[0], p0 = th[1], p1 = th[2], p2 = th[3];
    const double d = s * s - (p0 * p0 + p1 * p1 + p2 * p2);
    R[0][0] = d + 2 * p0 * p0;      R[0][1] = 2 * p0 * p1 - 2 * s * p2; R[0][2] = 2 * p0 * p2 + 2 * s * p1;
    R[1][0] = 2 * p1 * p0 + 2 * s * p2; R[1][1] = d + 2 * p1 * p1;  R[1][2] = 2 * p1 * p2 - 2 * s * p0;
    R[2][0] = 2 * p2 * p0 - 2 * s * p1; R[2][1] = 2 * p2 * p1 + 2 * s * p0; R[2][2] = d + 2 * p2 * p2;
}

__global__ void blobs_kernel(int64_t nb, int nper, const double* __restrict__ shape, const double* __restrict__ q,
                             const double* __restrict__ theta, double* __restrict__ r)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = nb * nper;
    if (i >= n) return;
    const int64_t p = i / nper;
    const int k = (int)(i - p * nper);
    double R[3][3];
    quat_rot(theta + 4 * p, R);
    const double s0 = shape[3 * k], s1 = shape[3 * k + 1], s2 = shape[3 * k + 2];
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c * n + i] = q[3 * p + c] + R[c][0] * s0 + R[c][1] * s1 + R[c][2] * s2;
}

void launch_blobs(int64_t nb, int nper, const double* shape, const double* q, const double* theta, double* r,
                  cudaStream_t st)
{
    const int64_t n = nb * nper;
    if (n <= 0) return;
    blobs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nb, nper, shape, q, theta, r); count_launch();
}

__global__ void K_kernel(int64_t nb, int nper, const double* __restrict__ r, const double* __restrict__ q,
                         const double* __restrict__ U, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = nb * nper;
    if (i >= n) return;
    const int64_t p = i / nper;
    const double d0 = r[i] - q[3 * p], d1 = r[n + i] - q[3 * p + 1], d2 = r[2 * n + i] - q[3 * p + 2];
    const double* u = U + 6 * p;
    out[i] = u[0] + (u[4] * d2 - u[5] * d1);
    out[n + i] = u[1] + (u[5] * d0 - u[3] * d2);
    out[2 * n + i] = u[2] + (u[3] * d1 - u[4] * d0);
}

void launch_K(int64_t nb, int nper, const double* r, const double* q, const double* U, double* out, cudaStream_t st)
{
    const int64_t n = nb * nper;
    if (n <= 0) return;
    K_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(nb, nper, r, q, U, out); count_launch();
}

// one warp per body: lanes stride over its blobs, shuffle-reduce 6 sums
__global__ void KT_kernel(int64_t nb, int nper, const double* __restrict__ r, const double* __restrict__ q,
                          const double* __restrict__ lam, double* __restrict__ out)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nb) return;
    const int64_t n = nb * nper;
    double s[6] = {0, 0, 0, 0, 0, 0};
    const double q0 = q[3 * w], q1 = q[3 * w + 1], q2 = q[3 * w + 2];
    for (int k = lane; k < nper; k += 32) {
        const int64_t i = w * nper + k;
        const double l0 = lam[i], l1 = lam[n + i], l2 = lam[2 * n + i];
        const double d0 = r[i] - q0, d1 = r[n + i] - q1, d2 = r[2 * n + i] - q2;
        s[0] += l0; s[1] += l1; s[2] += l2;
        s[3] += d1 * l2 - d2 * l1;
        s[4] += d2 * l0 - d0 * l2;
        s[5] += d0 * l1 - d1 * l0;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        double v = s[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        s[c] = v;
    }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) out[6 * w + c] = s[c];
}

void launch_KT(int64_t nb, int nper, const double* r, const double* q, const double* lam, double* out,
               cudaStream_t st)
{
    if (nb <= 0) return;
    const int64_t threads = nb * 32;
    KT_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(nb, nper, r, q, lam, out); count_launch();
}

// q1 = q0 + s u; theta1 = Rotate(theta0, s omega)
__global__ void advance_kernel(int64_t nb, const double* __restrict__ q0, const double* __restrict__ th0,
                               const double* __restrict__ U, double s, double* __restrict__ q1,
                               double* __restrict__ th1)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nb) return;
    const double* u = U + 6 * p;
#pragma unroll
    for (int c = 0; c < 3; ++c) q1[3 * p + c] = q0[3 * p + c] + s * u[c];
    const double f0 = s * u[3], f1 = s * u[4], f2 = s * u[5];
    const double ang = sqrt(f0 * f0 + f1 * f1 + f2 * f2);
    double c = 1.0, k = 0.5;  // sin(ang/2)/ang -> 1/2 as ang -> 0
    if (ang > 0.0) {
        double sn;
        sincos(0.5 * ang, &sn, &c);
        k = sn / ang;
    }
    const double a0 = c, a1 = k * f0, a2 = k * f1, a3 = k * f2;  // rotation quaternion
    const double b0 = th0[4 * p], b1 = th0[4 * p + 1], b2 = th0[4 * p + 2], b3 = th0[4 * p + 3];
    // (a0, a) (x) (b0, b) = (a0 b0 - a.b, a0 b + b0 a + a x b)
    th1[4 * p] = a0 * b0 - (a1 * b1 + a2 * b2 + a3 * b3);
    th1[4 * p + 1] = a0 * b1 + b0 * a1 + (a2 * b3 - a3 * b2);
    th1[4 * p + 2] = a0 * b2 + b0 * a2 + (a3 * b1 - a1 * b3);
    th1[4 * p + 3] = a0 * b3 + b0 * a3 + (a1 * b2 - a2 * b1);
}

void launch_advance(int64_t nb, const double* q0, const double* th0, const double* U, double s, double* q1,
                    double* th1, cudaStream_t st)
{
    if (nb <= 0) return;
    advance_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, q0, th0, U, s, q1, th1); count_launch();
}

__global__ void blob_forces_kernel(int64_t n, const double* __restrict__ r, rpbd_forces f, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double z = r[2 * n + i];
    const double h = z > f.h_floor ? z : f.h_floor;
    double fz = -f.weight;
    if (f.wall_gamma != 0.0) fz += f.wall_gamma * exp(-h / f.wall_b) * (1.0 / (f.wall_b * h) + 1.0 / (h * h));
    out[i] = 0.0;
    out[n + i] = 0.0;
    out[2 * n + i] = fz;
}

// Blob-blob Yukawa repulsion between blobs of different bodies (Sec. 4.1,
// U = gamma exp(-r/b)/r), added to out.  The force is evaluated at
// max(r, r_floor); pairs beyond r_cut (when > 0) and coincident blobs are
// skipped.  One thread per target blob, sources split into chunks of
// STERIC_CH (grid.y) so small suspensions still fill the GPU; each chunk's
// sum goes to its own partial and a second kernel adds the chunks in a fixed
// order (deterministic).  Source tiles are staged through shared memory.
// FP64: FP64 throughout.  FP32: positions split into hi + lo floats so
// separations keep FP64-level accuracy (as in the pair kernels), force in
// FP32 with one rsqrt and one fast exp (__expf) per pair.
constexpr int STERIC_T = 256;
constexpr int STERIC_CH = 2048;

// force on the target from one source at separation (dx, dy, dz), r2 = |d|^2
template <typename T>
__device__ __forceinline__ void steric_pair(T dx, T dy, T dz, T gamma, T invb, T rfloor, T ifl, T rfl2, T rcut2,
                                            T& fx, T& fy, T& fz)
{
    const T r2 = dx * dx + dy * dy + dz * dz;
    if ((rcut2 > T(0) && r2 > rcut2) || !(r2 > T(0))) return;
    T inv, rr, e;
    const bool fl = r2 < rfl2;
    if constexpr (std::is_same<T, float>::value) {
        inv = rsqrtf(r2);
        rr = r2 * inv;
        e = __expf(-(fl ? rfloor : rr) * invb);
    } else {
        rr = sqrt(r2);
        inv = 1.0 / rr;
        e = exp(-(fl ? rfloor : rr) * invb);
    }
    const T ire = fl ? ifl : inv;
    const T c = gamma * e * ire * (invb + ire) * inv;
    fx += dx * c;
    fy += dy * c;
    fz += dz * c;
}

template <typename T>
__global__ void __launch_bounds__(STERIC_T) steric_kernel(int64_t n, int nper, const double* __restrict__ r, T gamma,
                                                          T b, T rfloor, T rcut2, T* __restrict__ part)
{
    constexpr bool F32 = std::is_same<T, float>::value;
    // FP32: (x, y, z) hi and lo parts as two float4 per source; FP64: (x, y, z, 0)
    using V4 = typename std::conditional<F32, float4, double4>::type;
    __shared__ V4 sh[STERIC_T];
    __shared__ float4 sl[F32 ? STERIC_T : 1];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ii = i < n ? i : n - 1;
    const double xi = r[ii], yi = r[n + ii], zi = r[2 * n + ii];
    const T txh = (T)xi, tyh = (T)yi, tzh = (T)zi;
    const float txl = F32 ? (float)(xi - (double)txh) : 0.0f, tyl = F32 ? (float)(yi - (double)tyh) : 0.0f,
                tzl = F32 ? (float)(zi - (double)tzh) : 0.0f;
    const int64_t b0 = (ii / nper) * nper, b1 = b0 + nper;  // own body's blobs
    const T invb = T(1) / b, ifl = T(1) / rfloor;
    const T rfl2 = rfloor * rfloor;
    T fx = 0, fy = 0, fz = 0;
    const int64_t j0 = (int64_t)blockIdx.y * STERIC_CH;
    const int64_t j1 = (j0 + STERIC_CH) < n ? (j0 + STERIC_CH) : n;
    for (int64_t t0 = j0; t0 < j1; t0 += STERIC_T) {
        const int64_t j = t0 + threadIdx.x;
        if (j < j1) {
            const double x = r[j], y = r[n + j], z = r[2 * n + j];
            V4 hv;
            hv.x = (T)x;
            hv.y = (T)y;
            hv.z = (T)z;
            hv.w = T(0);
            sh[threadIdx.x] = hv;
            if constexpr (F32)
                sl[threadIdx.x] = make_float4((float)(x - (double)hv.x), (float)(y - (double)hv.y),
                                              (float)(z - (double)hv.z), 0.0f);
        }
        __syncthreads();
        const int cnt = (int)((j1 - t0) < STERIC_T ? (j1 - t0) : STERIC_T);
        // own-body sources of this tile: [lo, hi) in tile indices
        const int64_t lo64 = b0 - t0, hi64 = b1 - t0;
        const int lo = (int)(lo64 < 0 ? 0 : (lo64 > cnt ? cnt : lo64));
        const int hi = (int)(hi64 < 0 ? 0 : (hi64 > cnt ? cnt : hi64));
        for (int jj = 0; jj < cnt; ++jj) {
            if (jj >= lo && jj < hi) continue;
            const V4 sv = sh[jj];
            T dx = txh - sv.x, dy = tyh - sv.y, dz = tzh - sv.z;
            if constexpr (F32) {
                const float4 lv = sl[jj];
                dx += txl - lv.x;
                dy += tyl - lv.y;
                dz += tzl - lv.z;
            }
            steric_pair<T>(dx, dy, dz, gamma, invb, rfloor, ifl, rfl2, rcut2, fx, fy, fz);
        }
        __syncthreads();
    }
    if (i < n) {
        T* o = part + (int64_t)blockIdx.y * 3 * n;
        o[i] = fx;
        o[n + i] = fy;
        o[2 * n + i] = fz;
    }
}

template <typename T>
__global__ void steric_reduce_kernel(int64_t n, int nch, const T* __restrict__ part, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nch; ++k) acc += (double)part[((int64_t)k * 3 + c) * n + i];
        out[c * n + i] += acc;
    }
}

template <typename T>
static int launch_steric(rpbd_handle* h, int64_t n, int nper, const double* r, const rpbd_forces& f, double* out,
                         cudaStream_t st)
{
    const int nch = (int)((n + STERIC_CH - 1) / STERIC_CH);
    T* part;
    RPBD_TRY(ensure_t(h, BUF_AUX, (size_t)nch * 3 * n, &part));
    const T rc2 = f.r_cut > 0.0 ? (T)(f.r_cut * f.r_cut) : T(0);
    const dim3 grid((unsigned)((n + STERIC_T - 1) / STERIC_T), (unsigned)nch);
    steric_kernel<T><<<grid, STERIC_T, 0, st>>>(n, nper, r, (T)f.steric_gamma, (T)f.steric_b, (T)f.r_floor, rc2,
                                                part);
    count_launch();
    steric_reduce_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, nch, part, out);
    count_launch();
    return RPBD_OK;
}

int launch_blob_forces(rpbd_handle* h, int64_t n, int nper, const double* r, const rpbd_forces& f, int dtype,
                       double* out, cudaStream_t st)
{
    if (n <= 0) return RPBD_OK;
    blob_forces_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, r, f, out); count_launch();
    if (f.steric_gamma != 0.0 && nper > 0) {
        if (dtype == RPBD_F32) RPBD_TRY(launch_steric<float>(h, n, nper, r, f, out, st));
        else RPBD_TRY(launch_steric<double>(h, n, nper, r, f, out, st));
    }
    return RPBD_OK;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 and Box-Muller

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
    const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

__global__ void normals_kernel(uint64_t seed, uint32_t step, uint32_t sid, int64_t n, double* __restrict__ out)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // counter index
    if (g * 4 >= n) return;
    uint32_t c[4] = {(uint32_t)g, step, sid, 0u};
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const double TWO_M32 = 2.3283064365386963e-10;  // 2^-32
    const double TWO_PI = 6.283185307179586476925;
    double z[4];
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const double ua = ((double)c[2 * pr] + 0.5) * TWO_M32;
        const double ub = ((double)c[2 * pr + 1] + 0.5) * TWO_M32;
        const double rad = sqrt(-2.0 * log(ua));
        double sn, cs;
        sincos(TWO_PI * ub, &sn, &cs);
        z[2 * pr] = rad * cs;
        z[2 * pr + 1] = rad * sn;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (g * 4 + w < n) out[g * 4 + w] = z[w];
}

void launch_normals(uint64_t seed, uint32_t step, uint32_t sid, int64_t n, double* out, cudaStream_t st)
{
    if (n <= 0) return;
    const int64_t nc = (n + 3) / 4;
    normals_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(seed, step, sid, n, out); count_launch();
}

// ---------------------------------------------------------------------------
// FP64 vector helpers

__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

static unsigned grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (unsigned)g;
}

void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t st)
{
    if (n <= 0) return;
    axpby_kernel<<<grid_for(n), 256, 0, st>>>(n, a, x, b, y, out); count_launch();
}

void launch_scale_copy(int64_t n, double a, const double* x, double* out, cudaStream_t st)
{
    launch_axpby(n, a, x, 0.0, nullptr, out, st);
}

__global__ void finite_kernel(int64_t n, const double* __restrict__ x, int* __restrict__ bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) atomicExch(bad, 1);
}

int check_finite(rpbd_handle* h, int64_t n, const double* x, cudaStream_t st)
{
    if (n <= 0) return RPBD_OK;
    int* flag;
    RPBD_TRY(ensure_t(h, BUF_AUX, 1, &flag));
    RPBD_CU(h, cudaMemsetAsync(flag, 0, sizeof(int), st));
    finite_kernel<<<grid_for(n), 256, 0, st>>>(n, x, flag); count_launch();
    RPBD_LAUNCH_CHECK(h);
    int bad = 0;
    RPBD_CU(h, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RPBD_CU(h, cudaStreamSynchronize(st));
    if (bad) return set_error(h, RPBD_BAD_INPUT, "non-finite values in positions");
    return RPBD_OK;
}

}  // namespace rpbd
