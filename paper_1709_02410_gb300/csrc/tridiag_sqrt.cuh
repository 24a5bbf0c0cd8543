// T^{1/2} e_1 for the Lanczos square root (Sec. 2.2): the symmetric
// tridiagonal T_m (diagonal alpha, off-diagonal beta) is diagonalised by
// cyclic Jacobi on one warp, T = Q diag(lambda) Q^T, and
//   c = T^{1/2} e_1 = Q diag(sqrt(max(lambda, 0))) Q^T e_1.
//
// The rotations of one sweep are ordered as a round-robin tournament: in each
// of the N - 1 rounds (N = m1 rounded up to even) the indices form N/2
// disjoint pairs, so the round's rotations commute and are applied together
// (all column updates, then all row updates, the lanes splitting the
// entries).  A sweep therefore costs N - 1 dependent steps instead of
// m1 (m1 - 1) / 2.  Each pair's 2x2 block is then set from the closed form
// (diagonal app - t apq, aqq + t apq, off-diagonal exactly zero).
#pragma once

#include <cuda_runtime.h>

namespace rpbd {

constexpr int TRIDIAG_MAX_PAIRS = 48;

// shared memory (doubles) the routine needs for order m1
__host__ __device__ inline int tridiag_sqrt_smem_doubles(int m1) { return 2 * m1 * m1 + 6 * TRIDIAG_MAX_PAIRS; }

// One warp (all 32 lanes call it).  sm: tridiag_sqrt_smem_doubles(m1)
// doubles of shared memory; m1 <= 2 * TRIDIAG_MAX_PAIRS.  On return c[i]
// (global or shared, i < m1) holds T^{1/2} e_1; the return value is valid
// in every lane.
__device__ inline void tridiag_sqrt_e1(int m1, const double* __restrict__ alpha, const double* __restrict__ beta,
                                       double* sm, double* __restrict__ c)
{
    const int lane = threadIdx.x & 31;
    double* A = sm;                    // m1 x m1, row-major
    double* Q = A + m1 * m1;           // eigenvectors (columns)
    double* rc = Q + m1 * m1;          // per pair: cos, sin, t, apq, app, aqq
    double* rs = rc + TRIDIAG_MAX_PAIRS;
    double* rt = rs + TRIDIAG_MAX_PAIRS;
    double* rpq = rt + TRIDIAG_MAX_PAIRS;
    double* rpp = rpq + TRIDIAG_MAX_PAIRS;
    double* rqq = rpp + TRIDIAG_MAX_PAIRS;
    for (int e = lane; e < m1 * m1; e += 32) {
        const int i = e / m1, j = e % m1;
        double v = 0.0;
        if (i == j) v = alpha[i];
        else if (j == i + 1) v = beta[i];
        else if (i == j + 1) v = beta[j];
        A[e] = v;
        Q[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncwarp();
    double fro = 0.0;
    for (int e = lane; e < m1 * m1; e += 32) fro += A[e] * A[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
    const int N = (m1 + 1) & ~1;  // even number of slots; slot m1 (odd m1) sits out
    const int np = N / 2;
    // pair p of round r: slot N-1 against r, then (r + p, r - p) mod (N - 1)
    auto pair_of = [&](int r, int p, int& i, int& j) {
        int a, b;
        if (p == 0) {
            a = N - 1;
            b = r;
        } else {
            a = (r + p) % (N - 1);
            b = (r - p + (N - 1)) % (N - 1);
        }
        i = a < b ? a : b;
        j = a < b ? b : a;
    };
    for (int sweep = 0; sweep < 60 && m1 > 1; ++sweep) {
        double off = 0.0;
        for (int e = lane; e < m1 * m1; e += 32)
            if (e / m1 != e % m1) off += A[e] * A[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
        if (off <= 1e-32 * fro) break;
        for (int r = 0; r < N - 1; ++r) {
            // 1: one lane per pair computes its rotation (identity when skipped)
            for (int p = lane; p < np; p += 32) {
                int i, j;
                pair_of(r, p, i, j);
                double cc = 1.0, sn = 0.0, t = 0.0, apq = 0.0, app = 0.0, aqq = 0.0;
                if (j < m1) {
                    apq = A[i * m1 + j];
                    app = A[i * m1 + i];
                    aqq = A[j * m1 + j];
                    if (fabs(apq) > 1e-300 && !(fabs(apq) < 1e-19 * sqrt(fabs(app * aqq)))) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        t = tau != 0.0 ? copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau)) : 1.0;
                        cc = 1.0 / sqrt(1.0 + t * t);
                        sn = t * cc;
                    }
                }
                rc[p] = cc;
                rs[p] = sn;
                rt[p] = t;
                rpq[p] = apq;
                rpp[p] = app;
                rqq[p] = aqq;
            }
            __syncwarp();
            // 2: columns of A and Q: X <- X J
            for (int e = lane; e < np * m1; e += 32) {
                const int p = e / m1, k = e % m1;
                if (rs[p] == 0.0) continue;
                int i, j;
                pair_of(r, p, i, j);
                const double cc = rc[p], sn = rs[p];
                const double aki = A[k * m1 + i], akj = A[k * m1 + j];
                A[k * m1 + i] = cc * aki - sn * akj;
                A[k * m1 + j] = sn * aki + cc * akj;
                const double qki = Q[k * m1 + i], qkj = Q[k * m1 + j];
                Q[k * m1 + i] = cc * qki - sn * qkj;
                Q[k * m1 + j] = sn * qki + cc * qkj;
            }
            __syncwarp();
            // 3: rows of A: A <- J^T A
            for (int e = lane; e < np * m1; e += 32) {
                const int p = e / m1, k = e % m1;
                if (rs[p] == 0.0) continue;
                int i, j;
                pair_of(r, p, i, j);
                const double cc = rc[p], sn = rs[p];
                const double aik = A[i * m1 + k], ajk = A[j * m1 + k];
                A[i * m1 + k] = cc * aik - sn * ajk;
                A[j * m1 + k] = sn * aik + cc * ajk;
            }
            __syncwarp();
            // 4: each rotated pair's 2x2 block from the closed form
            for (int p = lane; p < np; p += 32) {
                if (rs[p] == 0.0) continue;
                int i, j;
                pair_of(r, p, i, j);
                A[i * m1 + i] = rpp[p] - rt[p] * rpq[p];
                A[j * m1 + j] = rqq[p] + rt[p] * rpq[p];
                A[i * m1 + j] = 0.0;
                A[j * m1 + i] = 0.0;
            }
            __syncwarp();
        }
    }
    __syncwarp();
    for (int i = lane; i < m1; i += 32) {
        double v = 0.0;
        for (int k = 0; k < m1; ++k) {
            const double lam = A[k * m1 + k];
            v += Q[i * m1 + k] * sqrt(lam > 0.0 ? lam : 0.0) * Q[k];  // Q[0][k]
        }
        c[i] = v;
    }
    __syncwarp();
}

}  // namespace rpbd
