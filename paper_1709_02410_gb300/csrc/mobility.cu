// Wall-RPY blob-mobility matvec U = M(r) F (Sec. 2.1; the dense GPU sum
// the paper uses for every application of M, Sec. 2.1 and Sec. 4.2).
//
// Pipeline of one apply:
//   1. pack:   per blob, one 16-byte aligned record holding its position
//              (FP32: hi/lo split of x, y; FP64: plain) and its k force
//              vectors pre-scaled by the wall-overlap scale s_j.
//   2. pairs:  grid (target tiles) x (source chunks).  Each CTA streams its
//              chunk of source records through shared memory with 1-D TMA
//              bulk copies (cp.async.bulk + mbarrier, NST-deep ring); each
//              thread owns one target blob, forms the 3x3 block of every
//              pair once and applies it to all k right-hand sides from
//              registers.  FP32 kernels keep FP32 sums over one chunk.
//   3. reduce: sums the chunk partials in a fixed order (FP64 partials
//              in FP64, FP32 partials as compensated float pairs, about
//              48 bits; the result is deterministic), multiplies by
//              s_i / (8 pi eta) and writes U in the caller's type.
// FP32 applies through the handle accumulate in fixed point instead
// (fixed_point.cuh): each CTA adds its chunk sums to one 64-bit integer per
// blob and component, so memory is O(n k) rather than O(n^2 k / 2048), and a
// small kernel finishes U; the result is the same bit for bit on every run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "accum.cuh"
#include "fixed_point.cuh"
#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"

namespace rpbd {

// ---------------------------------------------------------------------------
// record layouts

template <class R, int K>
struct Rec;
// FP32, k = 1: [x_hi, y_hi, x_lo, y_lo][z~, F(0,x), F(0,y), F(0,z)].
// FP32, k >= 2 (even): the right-hand sides interleaved in pairs, so one
// 8-byte lane pair holds the same component of two of them:
//   [x_hi, y_hi, x_lo, y_lo][z~, 0, F(0,x), F(1,x), F(0,y), F(1,y), F(0,z), F(1,z), F(2,x), F(3,x) ...]
// padded to 4 floats.
template <int K>
struct Rec<float, K> {
    static constexpr int TAIL = K == 1 ? 4 : ((2 + 3 * K) + 3) / 4 * 4;
    static constexpr int LEN = 4 + TAIL;  // floats
};
// FP64: [x, y, z~, F(0,x), F(0,y), F(0,z), ...] padded to 2 doubles
template <int K>
struct Rec<double, K> {
    static constexpr int LEN = ((3 + 3 * K) + 1) / 2 * 2;  // doubles
};

// partial sums: FP32 kernels store float chunk sums, FP64 kernels double
template <class R>
struct PartialT { using type = R; };

// FP32 fixed-point accumulation (acc != nullptr): [3K][n_pad] accumulators and
// fmax_bits (largest |force|, non-finite flag); cap as in fixed_exponent
struct FixedAcc {
    unsigned long long* acc;
    unsigned* fmax_bits;
    double cap;
};

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier + 1-D TMA bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: `limit` SM clock cycles at most (default ~2 s); false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = 4000000000LL)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// 1. pack

template <class R, int K, class In>
__global__ void pack_kernel(int64_t n, int64_t n_pad, int k, const double* __restrict__ r,
                            const In* __restrict__ F, double a, int wall, double s_min,
                            R* __restrict__ rec, double* __restrict__ scale, unsigned* __restrict__ fmax_bits = nullptr)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    constexpr int LEN = Rec<R, K>::LEN;
    R* o = rec + i * LEN;
    double x, y, zt, s;
    if (i < n) {
        x = r[i];
        y = r[n + i];
        const double z = r[2 * n + i];
        if (wall) {
            zt = z > a ? z : a;
            const double t = z / a;
            s = t >= 1.0 ? 1.0 : (t <= s_min ? s_min : t);
        } else {
            zt = z;
            s = 1.0;
        }
        scale[i] = s;
    } else {  // padding source: far away, zero force
        x = 1.0e7;
        y = 1.0e7;
        zt = a;
        s = 0.0;
    }
    if constexpr (sizeof(R) == 4) {
        const float xh = (float)x, yh = (float)y;
        o[0] = xh;
        o[1] = yh;
        o[2] = (float)(x - (double)xh);
        o[3] = (float)(y - (double)yh);
        o[4] = (float)zt;
        constexpr int TAIL = Rec<R, K>::TAIL;
#pragma unroll
        for (int q = 1; q < TAIL; ++q) o[4 + q] = 0.0f;
        float fm = 0.0f;  // largest |stored force| of this blob (+inf: not finite)
        if (i < n)
            for (int m = 0; m < k; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float v = (float)(s * (double)F[((int64_t)m * 3 + c) * n + i]);
                    if constexpr (K == 1) o[5 + c] = v;
                    else o[6 + 6 * (m / 2) + 2 * c + (m & 1)] = v;
                    fm = isfinite(v) ? fmaxf(fm, fabsf(v)) : INFINITY;
                }
        if (fmax_bits) fixed_force_max(fmax_bits, fm);
    } else {
        o[0] = x;
        o[1] = y;
        o[2] = zt;
#pragma unroll
        for (int q = 3; q < LEN; ++q) o[q] = 0.0;
        if (i < n)
            for (int m = 0; m < k; ++m)
#pragma unroll
                for (int c = 0; c < 3; ++c) o[3 + 3 * m + c] = s * (double)F[((int64_t)m * 3 + c) * n + i];
    }
}

// ---------------------------------------------------------------------------
// 2. pair kernel

template <class R, int K, int BT, int TS, int NST, bool WALL, bool PER, bool FX>
__device__ __forceinline__ void pair_body(const R* __restrict__ rec, int64_t n, int64_t n_pad, int tiles_per_chunk,
                                          int n_tiles, PairConst<R> pc, typename PartialT<R>::type* __restrict__ partial,
                                          int* __restrict__ err_flag, RingTest rt, FixedAcc fx)
{
    constexpr int LEN = Rec<R, K>::LEN;
    constexpr uint32_t TILE_BYTES = TS * LEN * sizeof(R);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    R* stage = reinterpret_cast<R*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NST * TILE_BYTES);

    const int tid = threadIdx.x;
    const int chunk = blockIdx.y;
    const int tile0 = chunk * tiles_per_chunk;
    const int ntile = min(tiles_per_chunk, n_tiles - tile0);
    const int64_t i = blockIdx.x * (int64_t)BT + tid;
    const int64_t ii = i < n ? i : n - 1;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        // (failure-path test: stage 0 gets no copy, so its wait runs out)
        for (int s = rt.skip_first ? 1 : 0; s < NST && s < ntile; ++s) {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * TS * LEN, rec + (size_t)(tile0 + s) * TS * LEN, TILE_BYTES, &bar[s]);
        }
    }

    // target position
    const R* me = rec + ii * LEN;
    R xh, yh, xl = R(0), yl = R(0), zi;
    if constexpr (sizeof(R) == 4) {
        const float4 p = *reinterpret_cast<const float4*>(me);
        xh = p.x; yh = p.y; xl = p.z; yl = p.w;
        zi = me[4];
    } else {
        xh = me[0]; yh = me[1]; zi = me[2];
    }

    // FP32 with k >= 2: accumulators of right-hand-side pairs (2p, 2p+1) in
    // the .x / .y lanes, updated by two-wide FMAs against the broadcast block
    constexpr bool PK = sizeof(R) == 4 && K >= 2;
    constexpr int NA = PK ? 3 * K : 1;  // scalar accumulators, or float2 pairs below
    R acc[PK ? 1 : 3 * K];
    float2 acc2[PK ? 3 * K / 2 : 1];
#pragma unroll
    for (int q = 0; q < (PK ? 1 : 3 * K); ++q) acc[q] = R(0);
#pragma unroll
    for (int q = 0; q < (PK ? 3 * K / 2 : 1); ++q) acc2[q] = make_float2(0.0f, 0.0f);
    (void)NA;

    int t = 0;
    bool bad = false;
    for (; t < ntile; ++t) {
        const int s = t % NST;
        const uint32_t par = (t / NST) & 1;
        const bool ok = mbar_wait_bounded(&bar[s], par, rt.limit);
        if (ok) {
            const R* st = stage + (size_t)s * TS * LEN;
#pragma unroll(K <= 4 ? 2 : 1)
            for (int jj = 0; jj < TS; ++jj) {
                const R* rj = st + jj * LEN;
                R dx, dy, zj;
                R f[3 * K];
                if constexpr (sizeof(R) == 4) {
                    const float4 p = *reinterpret_cast<const float4*>(rj);
                    dx = (xh - p.x) + (xl - p.z);
                    dy = (yh - p.y) + (yl - p.w);
                    constexpr int TAIL = Rec<R, K>::TAIL;
                    float tail[TAIL];
#pragma unroll
                    for (int q = 0; q < TAIL / 4; ++q) {
                        const float4 v = reinterpret_cast<const float4*>(rj + 4)[q];
                        tail[4 * q + 0] = v.x; tail[4 * q + 1] = v.y;
                        tail[4 * q + 2] = v.z; tail[4 * q + 3] = v.w;
                    }
                    zj = tail[0];
#pragma unroll
                    for (int q = 0; q < 3 * K; ++q) f[q] = tail[(K == 1 ? 1 : 2) + q];
                } else {
                    dx = xh - rj[0];
                    dy = yh - rj[1];
                    zj = rj[2];
#pragma unroll
                    for (int q = 0; q < 3 * K; ++q) f[q] = rj[3 + q];
                }
                const R dz = zi - zj;
                R Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz;
                pair_block_images<R, R, WALL, PER>(dx, dy, dz, zi, zj, pc, Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz);
                if constexpr (PK) {
                    // two right-hand sides per instruction: f[6p + 2c + e] = F(2p + e, c)
                    const float2 bxx = make_float2(Mxx, Mxx), bxy = make_float2(Mxy, Mxy), bxz = make_float2(Mxz, Mxz);
                    const float2 byy = make_float2(Myy, Myy), byz = make_float2(Myz, Myz), bzx = make_float2(Mzx, Mzx);
                    const float2 bzy = make_float2(Mzy, Mzy), bzz = make_float2(Mzz, Mzz);
#pragma unroll
                    for (int pp = 0; pp < K / 2; ++pp) {
                        const float2 fx = make_float2(f[6 * pp], f[6 * pp + 1]);
                        const float2 fy = make_float2(f[6 * pp + 2], f[6 * pp + 3]);
                        const float2 fz = make_float2(f[6 * pp + 4], f[6 * pp + 5]);
                        acc2[3 * pp + 0] = __ffma2_rn(bxz, fz, __ffma2_rn(bxy, fy, __ffma2_rn(bxx, fx, acc2[3 * pp + 0])));
                        acc2[3 * pp + 1] = __ffma2_rn(byz, fz, __ffma2_rn(byy, fy, __ffma2_rn(bxy, fx, acc2[3 * pp + 1])));
                        acc2[3 * pp + 2] = __ffma2_rn(bzz, fz, __ffma2_rn(bzy, fy, __ffma2_rn(bzx, fx, acc2[3 * pp + 2])));
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        // three FMA chains: 9 FMA per right-hand side
                        const R fx = f[3 * m], fy = f[3 * m + 1], fz = f[3 * m + 2];
                        acc[3 * m + 0] = fma(Mxz, fz, fma(Mxy, fy, fma(Mxx, fx, acc[3 * m + 0])));
                        acc[3 * m + 1] = fma(Myz, fz, fma(Myy, fy, fma(Mxy, fx, acc[3 * m + 1])));
                        acc[3 * m + 2] = fma(Mzz, fz, fma(Mzy, fy, fma(Mzx, fx, acc[3 * m + 2])));
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        if (tid == 0 && t + NST < ntile) {
            fence_proxy_async();
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * TS * LEN, rec + (size_t)(tile0 + t + NST) * TS * LEN, TILE_BYTES,
                        &bar[s]);
        }
    }
    if (bad) {
        // record the timeout, then let copies still in flight land (bounded)
        if (tid == 0) {
            atomicExch(err_flag, 1);
            for (int u = t + 1; u < ntile && u < t + NST; ++u)
                mbar_wait_bounded(&bar[u % NST], (u / NST) & 1);
        }
        return;
    }
    if (i < n) {
        if constexpr (FX) {  // FP32: the chunk sums into the fixed-point accumulators
            const int S = fixed_exponent(__uint_as_float(__ldg(fx.fmax_bits)), n, fx.cap);
            unsigned* const flag = fx.fmax_bits + 1;
            if constexpr (PK) {
#pragma unroll
                for (int pp = 0; pp < K / 2; ++pp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        fixed_add(fx.acc + (int64_t)(3 * (2 * pp) + c) * n_pad + i, (float)acc2[3 * pp + c].x, S, flag);
                        fixed_add(fx.acc + (int64_t)(3 * (2 * pp + 1) + c) * n_pad + i, (float)acc2[3 * pp + c].y, S,
                                  flag);
                    }
            } else {
#pragma unroll
                for (int q = 0; q < 3 * K; ++q) fixed_add(fx.acc + (int64_t)q * n_pad + i, (float)acc[q], S, flag);
            }
        } else if constexpr (PK) {
#pragma unroll
            for (int pp = 0; pp < K / 2; ++pp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    partial[((int64_t)chunk * 3 * K + 3 * (2 * pp) + c) * n_pad + i] = acc2[3 * pp + c].x;
                    partial[((int64_t)chunk * 3 * K + 3 * (2 * pp + 1) + c) * n_pad + i] = acc2[3 * pp + c].y;
                }
        } else {
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) partial[((int64_t)chunk * 3 * K + q) * n_pad + i] = acc[q];
        }
    }
}

template <class R, int K, int BT, int TS, int NST, bool WALL, bool PER, bool FX = false>
__global__ void __launch_bounds__(BT) pair_kernel(const R* __restrict__ rec, int64_t n, int64_t n_pad,
                                                  int tiles_per_chunk, int n_tiles, PairConst<R> pc,
                                                  typename PartialT<R>::type* __restrict__ partial,
                                                  int* __restrict__ err_flag, RingTest rt, FixedAcc fx)
{
    pair_body<R, K, BT, TS, NST, WALL, PER, FX>(rec, n, n_pad, tiles_per_chunk, n_tiles, pc, partial, err_flag, rt, fx);
}

// FP32, 16 right-hand sides: registers capped so five CTAs share an SM
template <class R, int K, int BT, int TS, int NST, bool WALL, bool PER, bool FX = false>
__global__ void __launch_bounds__(BT, 5) pair_kernel_k16(const R* __restrict__ rec, int64_t n, int64_t n_pad,
                                                         int tiles_per_chunk, int n_tiles, PairConst<R> pc,
                                                         typename PartialT<R>::type* __restrict__ partial,
                                                         int* __restrict__ err_flag, RingTest rt, FixedAcc fx)
{
    pair_body<R, K, BT, TS, NST, WALL, PER, FX>(rec, n, n_pad, tiles_per_chunk, n_tiles, pc, partial, err_flag, rt, fx);
}

template <class R, int K, int BT, int TS, int NST, bool WALL, bool PER, bool FX>
static auto pick_pair_kernel()
{
    if constexpr (sizeof(R) == 4 && K == 16) return pair_kernel_k16<R, K, BT, TS, NST, WALL, PER, FX>;
    else return pair_kernel<R, K, BT, TS, NST, WALL, PER, FX>;
}

// ---------------------------------------------------------------------------
// 3. reduce

// one thread per (blob, component q = blockIdx.y < 3k): the chunk partials
// summed in chunk order (deterministic), four chunks' loads issued together
template <class P, class Out>
__global__ void reduce_kernel(int64_t n, int64_t n_pad, int k, int kt, int n_chunks,
                              const P* __restrict__ partial, const double* __restrict__ scale,
                              double inv8pieta, Out* __restrict__ U)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= n || q >= 3 * k) return;
    const P* src = partial + (int64_t)q * n_pad + i;
    const int64_t stride = (int64_t)3 * kt * n_pad;
    double sum = 0.0;
    int c = 0;
    if constexpr (sizeof(P) == 4) {  // FP32 partials: compensated FP32 pair
        float hs = 0.0f, hc = 0.0f;
        for (; c + 4 <= n_chunks; c += 4) {
            const float v0 = src[c * stride], v1 = src[(c + 1) * stride], v2 = src[(c + 2) * stride],
                        v3 = src[(c + 3) * stride];
            two_sum_acc(hs, hc, v0);
            two_sum_acc(hs, hc, v1);
            two_sum_acc(hs, hc, v2);
            two_sum_acc(hs, hc, v3);
        }
        for (; c < n_chunks; ++c) two_sum_acc(hs, hc, src[c * stride]);
        sum = two_sum_value(hs, hc);
    } else {
        for (; c < n_chunks; ++c) sum += (double)src[c * stride];
    }
    U[(int64_t)q * n + i] = (Out)(scale[i] * inv8pieta * sum);
}

// ---------------------------------------------------------------------------
// launch

struct Tile {
    int BT, TS, NST;
};

template <class R, int K>
constexpr Tile default_tile()
{
    if constexpr (sizeof(R) == 4) return Tile{128, 64, 3};
    else return Tile{128, 32, 3};
}

template <class R, int K, bool WALL, bool PER, class In, class Out>
static int apply_k(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    constexpr Tile T = default_tile<R, K>();
    constexpr int BT = T.BT, TS = T.TS, NST = T.NST;
    constexpr int LEN = Rec<R, K>::LEN;
    const int64_t n_pad = (n + TS - 1) / TS * TS;
    const int n_tiles = (int)(n_pad / TS);
    const int64_t tgt_tiles = (n + BT - 1) / BT;
    // chunk: enough CTAs to fill the GPU several times over, at most
    // MAX_CHUNK sources summed in the kernel's own precision
    const int max_chunk_tiles = (sizeof(R) == 4 ? 2048 : 4096) / TS;
    const int64_t want_ctas = (int64_t)h->sm_count * 8;
    int64_t S = (want_ctas + tgt_tiles - 1) / tgt_tiles;
    if (S < 1) S = 1;
    int tiles_per_chunk = (int)((n_tiles + S - 1) / S);
    if (tiles_per_chunk > max_chunk_tiles) tiles_per_chunk = max_chunk_tiles;
    if (tiles_per_chunk < 1) tiles_per_chunk = 1;
    const int n_chunks = (n_tiles + tiles_per_chunk - 1) / tiles_per_chunk;

    R* rec;
    double* scale;
    typename PartialT<R>::type* partial = nullptr;
    RPBD_TRY(ensure_t(h, BUF_PACK, (size_t)n_pad * LEN, &rec));
    RPBD_TRY(ensure_t(h, BUF_SCALE, (size_t)n_pad, &scale));
    // FP32: fixed-point accumulators unless per-chunk partials are requested
    // (RPBD_OPT_SYM_PARTIALS); block entries are at most 4 / (3 a) (8 pi eta
    // M in lengths of the caller), nine images in the periodic cell
    const bool fixed = sizeof(R) == 4 && !h->sym_partials;
    FixedAcc fx{nullptr, nullptr, (PER ? 36.0 : 4.0) / h->p.a};
    if (fixed) {
        RPBD_TRY(ensure_t(h, BUF_PARTIAL, (size_t)3 * K * n_pad + 1, &fx.acc));
        RPBD_CU(h, cudaMemsetAsync(fx.acc, 0, sizeof(unsigned long long) * (3 * K * n_pad + 1), st));
        fx.fmax_bits = reinterpret_cast<unsigned*>(fx.acc + 3 * K * n_pad);
    } else {
        RPBD_TRY(ensure_t(h, BUF_PARTIAL, (size_t)n_chunks * 3 * K * n_pad, &partial));
    }

    const PairConst<R> pc = PairConst<R>::make(h->p.a, h->p.Lx, h->p.Ly);
    pack_kernel<R, K, In><<<(unsigned)((n_pad + 255) / 256), 256, 0, st>>>(n, n_pad, k, r, F, h->p.a, h->p.wall,
                                                                           h->p.s_min, rec, scale, fx.fmax_bits);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    const size_t smem = (size_t)NST * TS * LEN * sizeof(R) + NST * sizeof(uint64_t);
    // FX: a separate instantiation, so the partials kernel keeps its own register allocation
    auto kern = pick_pair_kernel<R, K, BT, TS, NST, WALL, PER, false>();
    if constexpr (sizeof(R) == 4)
        if (fixed) kern = pick_pair_kernel<R, K, BT, TS, NST, WALL, PER, true>();
    if (once_per_device(h, reinterpret_cast<const void*>(kern)))
        RPBD_CU(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)tgt_tiles, (unsigned)n_chunks);
    if (h->profile) prof_begin(h, st);
    kern<<<grid, BT, smem, st>>>(rec, n, n_pad, tiles_per_chunk, n_tiles, pc, partial, h->dev_flag, ring_test(h),
                                 fx);
    count_launch();
    if (h->profile) prof_end(h, st, sizeof(R) == 4 ? RPBD_F32 : RPBD_F64, K, (double)n * (double)n);
    RPBD_LAUNCH_CHECK(h);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const dim3 rgrid((unsigned)((n + 255) / 256), (unsigned)(3 * k));
    if (fixed)
        finish_fixed_kernel<Out><<<rgrid, 256, 0, st>>>(n, n_pad, k, fx.cap, fx.acc, fx.fmax_bits, scale, inv8pieta, U);
    else
        reduce_kernel<typename PartialT<R>::type, Out><<<rgrid, 256, 0, st>>>(n, n_pad, k, K, n_chunks, partial, scale,
                                                                              inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

template <class R, bool WALL, bool PER, class In, class Out>
static int apply_dispatch(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    if (k <= 1) return apply_k<R, 1, WALL, PER>(h, n, r, F, U, k, st);
    if (k <= 2) return apply_k<R, 2, WALL, PER>(h, n, r, F, U, k, st);
    if (k <= 4) return apply_k<R, 4, WALL, PER>(h, n, r, F, U, k, st);
    if (k <= 8) return apply_k<R, 8, WALL, PER>(h, n, r, F, U, k, st);
    return apply_k<R, 16, WALL, PER>(h, n, r, F, U, k, st);
}

template <class In, class Out>
static int apply_typed(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, int dtype,
                       cudaStream_t st)
{
    const bool wall = h->p.wall != 0;
    const bool per = h->p.Lx > 0.0;  // periodic runs only with the wall (as in Sec. 4.2)
    if (dtype == RPBD_F32)
        return per ? apply_dispatch<float, true, true>(h, n, r, F, U, k, st)
                   : wall ? apply_dispatch<float, true, false>(h, n, r, F, U, k, st)
                          : apply_dispatch<float, false, false>(h, n, r, F, U, k, st);
    return per ? apply_dispatch<double, true, true>(h, n, r, F, U, k, st)
               : wall ? apply_dispatch<double, true, false>(h, n, r, F, U, k, st)
                      : apply_dispatch<double, false, false>(h, n, r, F, U, k, st);
}

int mobility_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k, int dtype,
                        bool io_double, cudaStream_t st)
{
    if (n <= 0) return RPBD_OK;
    if (k < 1 || k > 16) return set_error(h, RPBD_BAD_ARG, "k must be in 1..16");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "bad dtype");
    if (!r || !F || !U) return set_error(h, RPBD_BAD_ARG, "null pointer");
    // the one-home symmetric kernel keeps one visitor partial per (home tile,
    // blob): about n^2 / 256 * 3k floats, plus FP64 segment sums (one per 16
    // home tiles); beyond 16 GiB it gives way to the one-direction kernel, whose
    // partials grow as n^2 / 2048.  The packed kernel accumulates in fixed
    // point per blob (memory O(n)) and takes any n.
    const double np_ = (double)(n + 255);
    const double sym_bytes =
        (np_ / 256.0 + np_ / 2048.0 + 2.0 * np_ / 4096.0 + 4.0) * 3.0 * (k <= 2 ? k : 4) * np_ * 4.0;
    if (dtype == RPBD_F32 && h->p.wall && h->far_field) {
        // cancellation-free far field: the packed symmetric kernel, up to four
        // right-hand sides per launch
        if (!h->use_packed) return set_error(h, RPBD_BAD_ARG, "far-field mode needs the packed symmetric kernel");
        const size_t esz = io_double ? sizeof(double) : sizeof(float);
        for (int m0 = 0; m0 < k; m0 += 4) {
            const int kc = k - m0 < 4 ? k - m0 : 4;
            const size_t off = (size_t)m0 * 3 * (size_t)n * esz;
            RPBD_TRY(sym_apply_impl(h, n, r, static_cast<const char*>(F) + off, static_cast<char*>(U) + off, kc,
                                    io_double, st));
        }
        return RPBD_OK;
    }
    // the packed symmetric kernel takes any n (past the partials' limit it sums in FP64
    // atomics); the one-home kernel only while its partials fit
    const bool packed_sym = h->use_packed && h->p.wall;
    if (dtype == RPBD_F32 && k <= 4 && h->use_sym[sym_class(k)] && (packed_sym || sym_bytes <= 16.0 * (1ull << 30)))
        return sym_apply_impl(h, n, r, F, U, k, io_double, st);
    // one direction with the wall in the open cell: the packed tile (two
    // targets per thread) for k = 1, 3, 4; k = 2 keeps its own K = 2 tile
    if (dtype == RPBD_F32 && h->use_packed && h->p.wall && !(h->p.Lx > 0.0) && k <= 4 && k != 2)
        return single_packed_apply_impl(h, n, r, F, U, k, io_double, st);
    if (io_double || dtype == RPBD_F64)
        return apply_typed<double, double>(h, n, r, (const double*)F, (double*)U, k, dtype, st);
    return apply_typed<float, float>(h, n, r, (const float*)F, (float*)U, k, dtype, st);
}

}  // namespace rpbd

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP32 multi-RHS matvec.
//
// Its scratch (packed source records, overlap scales, chunk partials and the
// wait-timeout flag) lives in one file-scope device array instead of the
// handle's workspace, so the call needs neither a handle nor cudaMalloc.
// Sizes are fixed by that array: n <= NOALLOC_MAX_N blobs, 1 <= k <= 16.

namespace rpbd {
namespace noalloc {

constexpr int64_t NOALLOC_MAX_N = 16384;
constexpr int MAX_CHUNK_SOURCES = 2048;  // FP32 chunk length, as in the workspace path
constexpr int64_t MAX_CHUNKS = NOALLOC_MAX_N / MAX_CHUNK_SOURCES;
constexpr size_t REC_BYTES = (size_t)NOALLOC_MAX_N * Rec<float, 16>::LEN * sizeof(float);
constexpr size_t SCALE_BYTES = (size_t)NOALLOC_MAX_N * sizeof(double);
constexpr size_t PARTIAL_BYTES = (size_t)MAX_CHUNKS * 3 * 16 * NOALLOC_MAX_N * sizeof(float);
constexpr size_t FLAG_BYTES = 256;
constexpr size_t SCRATCH_BYTES = REC_BYTES + SCALE_BYTES + PARTIAL_BYTES + FLAG_BYTES;  // 27.6 MiB

}  // namespace noalloc
}  // namespace rpbd

// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[rpbd::noalloc::SCRATCH_BYTES];

namespace rpbd {
namespace noalloc {

constexpr int MAX_DEVICES = 64;
static void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device; looked up once
// per device (host code may not use the symbol itself as a pointer).
static int scratch_address(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return RPBD_CUDA;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RPBD_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return RPBD_OK;
}

// A pair kernel whose bounded wait ran out skips its partial sums, so the
// reduction has summed stale values from an earlier call: the whole result
// is overwritten with NaN so that it cannot pass for a valid one.
__global__ void poison_on_timeout_kernel(int64_t count, const int* __restrict__ flag, float* __restrict__ U)
{
    if (*flag == 0) return;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) U[e] = __int_as_float(0x7fc00000);
}

template <int K, bool WALL>
static int apply(int sm_count, const rpbd_params& p, int64_t n, const double* r, const float* F, float* U, int k,
                 cudaStream_t st)
{
    constexpr Tile T = default_tile<float, K>();
    constexpr int BT = T.BT, TS = T.TS, NST = T.NST;
    constexpr int LEN = Rec<float, K>::LEN;
    unsigned char* base = nullptr;
    if (scratch_address(&base) != RPBD_OK) return RPBD_CUDA;
    float* rec = reinterpret_cast<float*>(base);
    double* scale = reinterpret_cast<double*>(base + REC_BYTES);
    float* partial = reinterpret_cast<float*>(base + REC_BYTES + SCALE_BYTES);
    int* flag = reinterpret_cast<int*>(base + REC_BYTES + SCALE_BYTES + PARTIAL_BYTES);

    const int64_t n_pad = (n + TS - 1) / TS * TS;
    const int n_tiles = (int)(n_pad / TS);
    const int64_t tgt_tiles = (n + BT - 1) / BT;
    const int max_chunk_tiles = MAX_CHUNK_SOURCES / TS;
    const int64_t want_ctas = (int64_t)sm_count * 8;
    int64_t S = (want_ctas + tgt_tiles - 1) / tgt_tiles;
    if (S < 1) S = 1;
    int tiles_per_chunk = (int)((n_tiles + S - 1) / S);
    if (tiles_per_chunk > max_chunk_tiles) tiles_per_chunk = max_chunk_tiles;
    if (tiles_per_chunk < 1) tiles_per_chunk = 1;
    // no more chunks than the partial region holds (at n = NOALLOC_MAX_N and
    // K = 16 this is exactly the 2048-source chunk)
    const int64_t fit = (int64_t)(PARTIAL_BYTES / ((size_t)3 * K * n_pad * sizeof(float)));
    const int min_tiles = (int)((n_tiles + fit - 1) / fit);
    if (tiles_per_chunk < min_tiles) tiles_per_chunk = min_tiles;
    const int n_chunks = (n_tiles + tiles_per_chunk - 1) / tiles_per_chunk;
    // the layout below must fit the array (guaranteed by n <= NOALLOC_MAX_N)
    if ((size_t)n_pad * LEN * sizeof(float) > REC_BYTES || (size_t)n_pad * sizeof(double) > SCALE_BYTES ||
        (size_t)n_chunks * 3 * K * n_pad * sizeof(float) > PARTIAL_BYTES)
        return RPBD_BAD_ARG;

    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return RPBD_CUDA;
    const PairConst<float> pc = PairConst<float>::make(p.a);
    pack_kernel<float, K, float><<<(unsigned)((n_pad + 255) / 256), 256, 0, st>>>(n, n_pad, k, r, F, p.a, p.wall,
                                                                               p.s_min, rec, scale);
    count_launch();
    const size_t smem = (size_t)NST * TS * LEN * sizeof(float) + NST * sizeof(uint64_t);
    static_assert((size_t)NST * TS * Rec<float, 16>::LEN * sizeof(float) + NST * sizeof(uint64_t) <= 48 * 1024,
                  "the no-alloc kernels must fit the default dynamic shared memory limit");
    pair_kernel<float, K, BT, TS, NST, WALL, false><<<dim3((unsigned)tgt_tiles, (unsigned)n_chunks), BT, smem, st>>>(
        rec, n, n_pad, tiles_per_chunk, n_tiles, pc, partial, flag, RingTest{4000000000LL, 0}, FixedAcc{});
    count_launch();
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * p.eta);
    reduce_kernel<float, float><<<dim3((unsigned)((n + 255) / 256), (unsigned)(3 * k)), 256, 0, st>>>(
        n, n_pad, k, K, n_chunks, partial, scale, inv8pieta, U);
    count_launch();
    const int64_t count = (int64_t)3 * k * n;
    poison_on_timeout_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, flag, U);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RPBD_OK : RPBD_CUDA;
}

template <bool WALL>
static int dispatch(int sm, const rpbd_params& p, int64_t n, const double* r, const float* F, float* U, int k,
                    cudaStream_t st)
{
    if (k <= 1) return apply<1, WALL>(sm, p, n, r, F, U, k, st);
    if (k <= 2) return apply<2, WALL>(sm, p, n, r, F, U, k, st);
    if (k <= 4) return apply<4, WALL>(sm, p, n, r, F, U, k, st);
    if (k <= 8) return apply<8, WALL>(sm, p, n, r, F, U, k, st);
    return apply<16, WALL>(sm, p, n, r, F, U, k, st);
}

}  // namespace noalloc
}  // namespace rpbd

extern "C" int rpbd_mobility_apply_f32_noalloc(const rpbd_params* p, int64_t n, const double* r, const float* F,
                                               float* U, int k, void* stream)
{
    using namespace rpbd::noalloc;
    if (!p || !(p->eta > 0) || !(p->a > 0) || !(p->s_min > 0) || p->s_min > 1) return RPBD_BAD_ARG;
    if (p->Lx != 0.0 || p->Ly != 0.0) return RPBD_BAD_ARG;  // open systems only
    if (n < 0 || k < 1) return RPBD_BAD_ARG;
    if (n > NOALLOC_MAX_N || k > 16) return RPBD_TOO_LARGE;  // beyond the fixed scratch array
    if (n == 0) return RPBD_OK;
    if (!r || !F || !U) return RPBD_BAD_ARG;
    int dev = 0, sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RPBD_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return p->wall ? dispatch<true>(sm, *p, n, r, F, U, k, st) : dispatch<false>(sm, *p, n, r, F, U, k, st);
}
