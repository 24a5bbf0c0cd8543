// Many independent suspensions of uneven size in one launch.
//
// Systems are concatenated: system s owns blobs [off_s, off_{s+1}) of every
// SoA array; blobs interact only inside their system (each system is its own
// wall-bounded suspension, Sec. 4).  The work is a list of items (system,
// target tile, source chunk), longest first; a persistent grid (one wave of
// resident CTAs) pulls items from an atomic counter -- no CTA ever waits for
// another, so the queue cannot hang.  Each item streams its chunk of source
// records through shared memory with the same TMA bulk ring as the single-
// system kernel and writes FP32 chunk partials that a reduce kernel sums in
// FP64 per target (deterministic).
//
// Tile shapes (targets per CTA, sources per stage) come from a small set of
// compiled variants; rpbd_autotune_batched times them on the caller's batch
// and keeps the fastest.  The batched Lanczos M^{1/2} W (Sec. 2.2) runs all
// systems in lockstep with per-system coefficients and stop flags; its
// iteration loop is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "accum.cuh"
#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"
#include "wall_rpy_x2.cuh"

namespace rpbd {

// same PTX helpers as the single-system kernel (file-local copies)
namespace bt {
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 4000000000LL) return false;
    return true;
}
}  // namespace bt

// FP32 record: [x_hi, y_hi, x_lo, y_lo][z~, F(0..K-1)] padded to 4 floats
template <int K>
struct BRec {
    static constexpr int TAIL = ((1 + 3 * K) + 3) / 4 * 4;
    static constexpr int LEN = 4 + TAIL;
};

struct Item {
    int sys;         // system
    int tgt0;        // first target (system-local index)
    int tile0;       // first source tile (system-local)
    int ntile;       // source tiles in the chunk
    int slot;        // chunk index inside the system (partial slot)
};

// per-system tables on the device
struct SysTab {
    const int64_t* off;      // blob offsets [n_sys + 1]
    const int64_t* rec_off;  // record offsets (padded to the stage tile) [n_sys + 1]
    const int* nslots;       // chunk slots per system [n_sys]
};

__device__ __forceinline__ int find_sys(const int64_t* off, int n_sys, int64_t i)
{
    int lo = 0, hi = n_sys;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// pack records of all systems (padded per system); index over padded records
template <int K, class In>
__global__ void bpack_kernel(int n_sys, int64_t n_tot, int64_t rec_tot, int k, SysTab tab, const double* __restrict__ r,
                             const In* __restrict__ F, double a, int wall, double s_min, float* __restrict__ rec,
                             double* __restrict__ scale)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= rec_tot) return;
    const int s = find_sys(tab.rec_off, n_sys, g);
    const int64_t local = g - tab.rec_off[s];
    const int64_t i = tab.off[s] + local;
    const bool real = i < tab.off[s + 1];
    constexpr int LEN = BRec<K>::LEN;
    float* o = rec + g * LEN;
    double x = 1.0e7, y = 1.0e7, zt = a, sc = 0.0;
    if (real) {
        x = r[i];
        y = r[n_tot + i];
        const double z = r[2 * n_tot + i];
        if (wall) {
            zt = z > a ? z : a;
            const double t = z / a;
            sc = t >= 1.0 ? 1.0 : (t <= s_min ? s_min : t);
        } else {
            zt = z;
            sc = 1.0;
        }
        scale[i] = sc;
    }
    const float xh = (float)x, yh = (float)y;
    o[0] = xh;
    o[1] = yh;
    o[2] = (float)(x - (double)xh);
    o[3] = (float)(y - (double)yh);
    o[4] = (float)zt;
#pragma unroll
    for (int q = 1; q < BRec<K>::TAIL; ++q) o[4 + q] = 0.0f;
    if (real)
        for (int m = 0; m < k; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) o[5 + 3 * m + c] = (float)(sc * (double)F[((int64_t)m * 3 + c) * n_tot + i]);
}

template <int K, int BT, int TS, int NST, bool WALL>
__global__ void __launch_bounds__(BT) bpair_kernel(const float* __restrict__ rec, SysTab tab, const Item* __restrict__ items,
                                                   int n_items, int* __restrict__ queue,
                                                   const int* __restrict__ active, PairConst<float> pc,
                                                   float* __restrict__ partial, int64_t n_tot, int* __restrict__ err_flag)
{
    constexpr int LEN = BRec<K>::LEN;
    constexpr uint32_t TILE_BYTES = TS * LEN * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NST * TILE_BYTES);
    __shared__ int s_item;
    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) bt::mbar_init(&bar[s], 1);
        bt::fence_mbar_init();
    }
    __syncthreads();
    uint32_t g = 0;  // tiles consumed by this CTA: ring stage g % NST, parity (g / NST) & 1
    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const Item w = items[it];
        if (active && !active[w.sys]) continue;  // system already converged
        const int64_t off = tab.off[w.sys];
        const int64_t n_s = tab.off[w.sys + 1] - off;
        const float* srec = rec + tab.rec_off[w.sys] * LEN;
        const int64_t li = (int64_t)w.tgt0 + tid;                 // system-local target
        const int64_t lii = li < n_s ? li : n_s - 1;
        if (tid == 0) {
            for (int s = 0; s < NST && s < w.ntile; ++s) {
                const uint32_t st = (g + s) % NST;
                bt::mbar_expect_tx(&bar[st], TILE_BYTES);
                bt::tma_load_1d(stage + (size_t)st * TS * LEN, srec + (size_t)(w.tile0 + s) * TS * LEN, TILE_BYTES,
                                &bar[st]);
            }
        }
        const float* me = srec + lii * LEN;
        const float4 pme = *reinterpret_cast<const float4*>(me);
        const float xh = pme.x, yh = pme.y, xl = pme.z, yl = pme.w, zi = me[4];
        float acc[3 * K];
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) acc[q] = 0.0f;
        bool bad = false;
        int t = 0;
        for (; t < w.ntile; ++t) {
            const uint32_t st = (g + t) % NST;
            const uint32_t par = ((g + t) / NST) & 1;
            const bool ok = bt::mbar_wait_bounded(&bar[st], par);
            if (ok) {
                const float* sp = stage + (size_t)st * TS * LEN;
#pragma unroll(K <= 4 ? 2 : 1)
                for (int jj = 0; jj < TS; ++jj) {
                    const float* rj = sp + jj * LEN;
                    const float4 p = *reinterpret_cast<const float4*>(rj);
                    const float dx = (xh - p.x) + (xl - p.z);
                    const float dy = (yh - p.y) + (yl - p.w);
                    float tail[BRec<K>::TAIL];
#pragma unroll
                    for (int q = 0; q < BRec<K>::TAIL / 4; ++q) {
                        const float4 v = reinterpret_cast<const float4*>(rj + 4)[q];
                        tail[4 * q] = v.x; tail[4 * q + 1] = v.y; tail[4 * q + 2] = v.z; tail[4 * q + 3] = v.w;
                    }
                    const float zj = tail[0];
                    float Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz;
                    pair_block<float, float, WALL>(dx, dy, zi - zj, zi, zj, pc, Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz);
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        const float fx = tail[1 + 3 * m], fy = tail[2 + 3 * m], fz = tail[3 + 3 * m];
                        acc[3 * m + 0] = fmaf(Mxz, fz, fmaf(Mxy, fy, fmaf(Mxx, fx, acc[3 * m + 0])));
                        acc[3 * m + 1] = fmaf(Myz, fz, fmaf(Myy, fy, fmaf(Mxy, fx, acc[3 * m + 1])));
                        acc[3 * m + 2] = fmaf(Mzz, fz, fmaf(Mzy, fy, fmaf(Mzx, fx, acc[3 * m + 2])));
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && t + NST < w.ntile) {
                bt::fence_proxy_async();
                bt::mbar_expect_tx(&bar[st], TILE_BYTES);
                bt::tma_load_1d(stage + (size_t)st * TS * LEN, srec + (size_t)(w.tile0 + t + NST) * TS * LEN,
                                TILE_BYTES, &bar[st]);
            }
        }
        if (bad) {
            if (tid == 0) {
                atomicExch(err_flag, 1);
                for (int u = t + 1; u < w.ntile && u < t + NST; ++u)
                    bt::mbar_wait_bounded(&bar[(g + u) % NST], ((g + u) / NST) & 1);
            }
            return;
        }
        g += w.ntile;
        if (li < n_s) {
            const int64_t i = off + li;
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) partial[((int64_t)w.slot * 3 * K + q) * n_tot + i] = acc[q];
        }
    }
}

// Packed variant (wall only): each thread owns two targets (t and t + BT of
// the item) and meets every source with both at once in packed two-wide FP32
// instructions (wall_rpy_x2.cuh, lengths in units of a).  Source records
// duplicate every field so a 16-byte load gives two packed operands:
// [x_hi x_hi y_hi y_hi][x_lo x_lo y_lo y_lo][z z F0x F0x][F0y F0y F0z F0z]...
template <int K>
struct BRec2 {
    static constexpr int LEN = (2 * (5 + 3 * K) + 3) / 4 * 4;
};

template <int K, class In>
__global__ void bpack2_kernel(int n_sys, int64_t n_tot, int64_t rec_tot, int k, SysTab tab,
                              const double* __restrict__ r, const In* __restrict__ F, double a, double s_min,
                              float* __restrict__ rec, double* __restrict__ scale)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= rec_tot) return;
    const int s = find_sys(tab.rec_off, n_sys, g);
    const int64_t local = g - tab.rec_off[s];
    const int64_t i = tab.off[s] + local;
    const bool real = i < tab.off[s + 1];
    constexpr int LEN = BRec2<K>::LEN;
    float* o = rec + g * LEN;
    double x = 1.0e7, y = 1.0e7, zt = a, sc = 0.0;
    if (real) {
        x = r[i];
        y = r[n_tot + i];
        const double z = r[2 * n_tot + i];
        zt = z > a ? z : a;
        const double t = z / a;
        sc = t >= 1.0 ? 1.0 : (t <= s_min ? s_min : t);
        scale[i] = sc;
    }
    const double ia = 1.0 / a;  // lengths in units of a
    x *= ia;
    y *= ia;
    zt *= ia;
    float v[LEN / 2];
#pragma unroll
    for (int q = 0; q < LEN / 2; ++q) v[q] = 0.0f;
    const float xh = (float)x, yh = (float)y;
    v[0] = xh;
    v[1] = yh;
    v[2] = (float)(x - (double)xh);
    v[3] = (float)(y - (double)yh);
    v[4] = (float)zt;
    if (real)
        for (int m = 0; m < k; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) v[5 + 3 * m + c] = (float)(sc * (double)F[((int64_t)m * 3 + c) * n_tot + i]);
#pragma unroll
    for (int q = 0; q < LEN / 2; ++q) {
        o[2 * q] = v[q];
        o[2 * q + 1] = v[q];
    }
}

template <int K, int BT, int TS, int NST>
__global__ void __launch_bounds__(BT) bpair2_kernel(const float* __restrict__ rec, SysTab tab,
                                                    const Item* __restrict__ items, int n_items,
                                                    int* __restrict__ queue, const int* __restrict__ active,
                                                    float* __restrict__ partial, int64_t n_tot,
                                                    int* __restrict__ err_flag)
{
    constexpr int LEN = BRec2<K>::LEN;
    constexpr uint32_t TILE_BYTES = TS * LEN * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NST * TILE_BYTES);
    __shared__ int s_item;
    const int tid = threadIdx.x;
    const PairConstX2 pc = PairConstX2::make_unit();
    const float2 m1 = pc.m1;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) bt::mbar_init(&bar[s], 1);
        bt::fence_mbar_init();
    }
    __syncthreads();
    uint32_t g = 0;  // tiles consumed by this CTA: ring stage g % NST, parity (g / NST) & 1
    for (;;) {
        if (tid == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) break;
        const Item w = items[it];
        if (active && !active[w.sys]) continue;  // system already converged
        const int64_t off = tab.off[w.sys];
        const int64_t n_s = tab.off[w.sys + 1] - off;
        const float* srec = rec + tab.rec_off[w.sys] * LEN;
        const int64_t l0 = (int64_t)w.tgt0 + tid, l1 = l0 + BT;  // system-local targets
        const int64_t c0 = l0 < n_s ? l0 : n_s - 1, c1 = l1 < n_s ? l1 : n_s - 1;
        if (tid == 0) {
            for (int s = 0; s < NST && s < w.ntile; ++s) {
                const uint32_t st = (g + s) % NST;
                bt::mbar_expect_tx(&bar[st], TILE_BYTES);
                bt::tma_load_1d(stage + (size_t)st * TS * LEN, srec + (size_t)(w.tile0 + s) * TS * LEN, TILE_BYTES,
                                &bar[st]);
            }
        }
        const float* r0 = srec + c0 * LEN;
        const float* r1 = srec + c1 * LEN;
        const float2 xh = make_float2(r0[0], r1[0]), yh = make_float2(r0[2], r1[2]);
        const float2 xl = make_float2(r0[4], r1[4]), yl = make_float2(r0[6], r1[6]);
        const float2 zi = make_float2(r0[8], r1[8]);
        float2 acc[3 * K];
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) acc[q] = make_float2(0.0f, 0.0f);
        bool bad = false;
        int t = 0;
        for (; t < w.ntile; ++t) {
            const uint32_t st = (g + t) % NST;
            const uint32_t par = ((g + t) / NST) & 1;
            const bool ok = bt::mbar_wait_bounded(&bar[st], par);
            if (ok) {
                const float* sp = stage + (size_t)st * TS * LEN;
#pragma unroll(K <= 4 ? 2 : 1)
                for (int jj = 0; jj < TS; ++jj) {
                    const float4* rj = reinterpret_cast<const float4*>(sp + jj * LEN);
                    const float4 p0 = rj[0], p1 = rj[1], p2 = rj[2];
                    const float2 dx = add2(fma2(m1, make_float2(p0.x, p0.y), xh), fma2(m1, make_float2(p1.x, p1.y), xl));
                    const float2 dy = add2(fma2(m1, make_float2(p0.z, p0.w), yh), fma2(m1, make_float2(p1.z, p1.w), yl));
                    const float2 zj = make_float2(p2.x, p2.y);
                    const float2 dz = fma2(m1, zj, zi);
                    float2 al, be, gx, gz, mzz;
                    pair_factors_x2<false>(dx, dy, dz, zi, zj, pc, al, be, gx, gz, mzz);
                    // forces F(m, c) at float index 10 + 2 (3m + c) of the record
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        const float* fp = sp + jj * LEN + 10 + 6 * m;
                        const float2 fx = make_float2(fp[0], fp[1]), fy = make_float2(fp[2], fp[3]);
                        const float2 fz = make_float2(fp[4], fp[5]);
                        const float2 P = fma2(dy, fy, mul2(dx, fx));
                        const float2 Q = fma2(be, P, mul2(gx, fz));
                        acc[3 * m + 0] = fma2(dx, Q, fma2(al, fx, acc[3 * m + 0]));
                        acc[3 * m + 1] = fma2(dy, Q, fma2(al, fy, acc[3 * m + 1]));
                        acc[3 * m + 2] = fma2(mzz, fz, fma2(gz, P, acc[3 * m + 2]));
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            if (tid == 0 && t + NST < w.ntile) {
                bt::fence_proxy_async();
                bt::mbar_expect_tx(&bar[st], TILE_BYTES);
                bt::tma_load_1d(stage + (size_t)st * TS * LEN, srec + (size_t)(w.tile0 + t + NST) * TS * LEN,
                                TILE_BYTES, &bar[st]);
            }
        }
        if (bad) {
            if (tid == 0) {
                atomicExch(err_flag, 1);
                for (int u = t + 1; u < w.ntile && u < t + NST; ++u)
                    bt::mbar_wait_bounded(&bar[(g + u) % NST], ((g + u) / NST) & 1);
            }
            return;
        }
        g += w.ntile;
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) {
            if (l0 < n_s) partial[((int64_t)w.slot * 3 * K + q) * n_tot + off + l0] = acc[q].x;
            if (l1 < n_s) partial[((int64_t)w.slot * 3 * K + q) * n_tot + off + l1] = acc[q].y;
        }
    }
}

template <class Out>
__global__ void breduce_kernel(int n_sys, int64_t n_tot, int k, int kt, SysTab tab, const float* __restrict__ partial,
                               const double* __restrict__ scale, const int* __restrict__ active, double inv8pieta,
                               Out* __restrict__ U)
{
    // one thread per (blob, component q = blockIdx.y < 3k); slots summed in
    // order as a compensated FP32 pair, four slots' loads issued together
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= n_tot || q >= 3 * k) return;
    const int s = find_sys(tab.off, n_sys, i);
    if (active && !active[s]) return;
    const int ns = tab.nslots[s];
    const float* src = partial + (int64_t)q * n_tot + i;
    const int64_t stride = (int64_t)3 * kt * n_tot;
    float hs = 0.0f, hc = 0.0f;
    int c = 0;
    for (; c + 4 <= ns; c += 4) {
        const float v0 = src[c * stride], v1 = src[(c + 1) * stride], v2 = src[(c + 2) * stride],
                    v3 = src[(c + 3) * stride];
        two_sum_acc(hs, hc, v0);
        two_sum_acc(hs, hc, v1);
        two_sum_acc(hs, hc, v2);
        two_sum_acc(hs, hc, v3);
    }
    for (; c < ns; ++c) two_sum_acc(hs, hc, src[c * stride]);
    U[(int64_t)q * n_tot + i] = (Out)(scale[i] * inv8pieta * two_sum_value(hs, hc));
}

// ---------------------------------------------------------------------------
// host side: plan (work list) per tile variant

struct Variant {
    int BT, TS;
    bool packed;  // two targets per thread (wall only)
    int targets() const { return packed ? 2 * BT : BT; }
};
static const Variant VARIANTS[] = {{128, 64, false}, {64, 64, false}, {256, 32, false}, {128, 64, true}};
constexpr int N_VARIANTS = 4;
constexpr int B_NST = 3;
constexpr int B_MAX_CHUNK = 2048;

struct BatchPlan {
    std::vector<int64_t> off;
    int variant = -1;
    int k = 0;
    int64_t rec_tot = 0;
    int n_items = 0;
    int max_slots = 0;
    // device copies
    int64_t* d_off = nullptr;
    int64_t* d_rec_off = nullptr;
    int* d_nslots = nullptr;
    Item* d_items = nullptr;
    int* d_queue = nullptr;
    int grid = 0;
};

static void free_plan(BatchPlan* p)
{
    if (!p) return;
    cudaFree(p->d_off);
    cudaFree(p->d_rec_off);
    cudaFree(p->d_nslots);
    cudaFree(p->d_items);
    cudaFree(p->d_queue);
    delete p;
}

template <int K, int BT, int TS>
static int occupancy2(int* blocks)
{
    constexpr int LEN = BRec2<K>::LEN;
    const size_t smem = (size_t)B_NST * TS * LEN * sizeof(float) + B_NST * sizeof(uint64_t);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, bpair2_kernel<K, BT, TS, B_NST>, BT, smem) ==
                   cudaSuccess
               ? RPBD_OK
               : RPBD_CUDA;
}

template <int K, int BT, int TS, bool WALL>
static int occupancy(int* blocks)
{
    constexpr int LEN = BRec<K>::LEN;
    const size_t smem = (size_t)B_NST * TS * LEN * sizeof(float) + B_NST * sizeof(uint64_t);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, bpair_kernel<K, BT, TS, B_NST, WALL>, BT, smem) ==
                   cudaSuccess
               ? RPBD_OK
               : RPBD_CUDA;
}

static int build_plan(rpbd_handle* h, const int64_t* off_host, int n_sys, int k, int variant, BatchPlan** out)
{
    const Variant V = VARIANTS[variant];
    BatchPlan* p = new BatchPlan();
    p->off.assign(off_host, off_host + n_sys + 1);
    p->variant = variant;
    p->k = k;
    std::vector<int64_t> rec_off(n_sys + 1, 0);
    std::vector<int> nslots(n_sys, 0);
    std::vector<Item> items;
    const int max_chunk_tiles = B_MAX_CHUNK / V.TS;
    for (int s = 0; s < n_sys; ++s) {
        const int64_t n_s = off_host[s + 1] - off_host[s];
        const int64_t ntiles = (n_s + V.TS - 1) / V.TS;
        rec_off[s + 1] = rec_off[s] + ntiles * V.TS;
        const int tpc = (int)std::min<int64_t>(max_chunk_tiles, std::max<int64_t>(1, ntiles));
        const int nch = (int)((ntiles + tpc - 1) / tpc);
        nslots[s] = nch;
        p->max_slots = std::max(p->max_slots, nch);
        for (int64_t t0 = 0; t0 < n_s; t0 += V.targets())
            for (int c = 0; c < nch; ++c) {
                Item it;
                it.sys = s;
                it.tgt0 = (int)t0;
                it.tile0 = c * tpc;
                it.ntile = (int)std::min<int64_t>(tpc, ntiles - (int64_t)c * tpc);
                it.slot = c;
                items.push_back(it);
            }
    }
    // longest items first: the dynamic queue then balances the tail
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.ntile > b.ntile; });
    p->rec_tot = rec_off[n_sys];
    p->n_items = (int)items.size();
    auto up = [&](void** d, const void* src, size_t bytes) -> int {
        if (cudaMalloc(d, bytes ? bytes : 16) != cudaSuccess) return RPBD_NO_MEM;
        if (bytes && src && cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return RPBD_CUDA;
        if (bytes && !src && cudaMemset(*d, 0, bytes) != cudaSuccess) return RPBD_CUDA;
        return RPBD_OK;
    };
    int st = RPBD_OK;
    if ((st = up((void**)&p->d_off, off_host, sizeof(int64_t) * (n_sys + 1))) != RPBD_OK ||
        (st = up((void**)&p->d_rec_off, rec_off.data(), sizeof(int64_t) * (n_sys + 1))) != RPBD_OK ||
        (st = up((void**)&p->d_nslots, nslots.data(), sizeof(int) * n_sys)) != RPBD_OK ||
        (st = up((void**)&p->d_items, items.data(), sizeof(Item) * items.size())) != RPBD_OK ||
        (st = up((void**)&p->d_queue, nullptr, sizeof(int))) != RPBD_OK) {
        free_plan(p);
        return set_error(h, st, "batched: plan upload failed");
    }
    *out = p;
    return RPBD_OK;
}

template <int K, int BT, int TS, bool WALL, class In, class Out>
static int run_variant(rpbd_handle* h, BatchPlan* p, int n_sys, const double* r, const In* F, Out* U, int k,
                       const int* active, int prof_kind, cudaStream_t st)
{
    constexpr int LEN = BRec<K>::LEN;
    const int64_t n_tot = p->off[n_sys];
    float* rec;
    double* scale;
    float* partial;
    RPBD_TRY(ensure_t(h, BUF_BPACK, (size_t)p->rec_tot * LEN, &rec));
    RPBD_TRY(ensure_t(h, BUF_BSCALE, (size_t)n_tot, &scale));
    RPBD_TRY(ensure_t(h, BUF_BPARTIAL, (size_t)p->max_slots * 3 * K * n_tot, &partial));
    SysTab tab{p->d_off, p->d_rec_off, p->d_nslots};
    bpack_kernel<K, In><<<(unsigned)((p->rec_tot + 255) / 256), 256, 0, st>>>(
        n_sys, n_tot, p->rec_tot, k, tab, r, F, h->p.a, h->p.wall, h->p.s_min, rec, scale);
    count_launch();
    const size_t smem = (size_t)B_NST * TS * LEN * sizeof(float) + B_NST * sizeof(uint64_t);
    auto kern = bpair_kernel<K, BT, TS, B_NST, WALL>;
    if (smem > 48 * 1024) RPBD_CU(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (p->grid == 0) {
        int blocks = 0;
        RPBD_TRY((occupancy<K, BT, TS, WALL>(&blocks)));
        p->grid = std::max(1, blocks) * h->sm_count;
    }
    RPBD_CU(h, cudaMemsetAsync(p->d_queue, 0, sizeof(int), st));
    const PairConst<float> pc = PairConst<float>::make(h->p.a);
    if (h->profile) prof_begin(h, st);
    kern<<<p->grid, BT, smem, st>>>(rec, tab, p->d_items, p->n_items, p->d_queue, active, pc, partial, n_tot,
                                    h->dev_flag);
    count_launch();
    if (h->profile) {
        double pairs = 0.0;
        for (int s = 0; s < n_sys; ++s) {
            const double ns = (double)(p->off[s + 1] - p->off[s]);
            pairs += ns * ns;
        }
        prof_end(h, st, prof_kind, K, pairs);
    }
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    breduce_kernel<Out><<<dim3((unsigned)((n_tot + 255) / 256), (unsigned)(3 * k)), 256, 0, st>>>(n_sys, n_tot, k, K, tab, partial, scale,
                                                                         active, inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

template <int K, int BT, int TS, class In, class Out>
static int run_variant2(rpbd_handle* h, BatchPlan* p, int n_sys, const double* r, const In* F, Out* U, int k,
                        const int* active, int prof_kind, cudaStream_t st)
{
    constexpr int LEN = BRec2<K>::LEN;
    const int64_t n_tot = p->off[n_sys];
    float* rec;
    double* scale;
    float* partial;
    RPBD_TRY(ensure_t(h, BUF_BPACK, (size_t)p->rec_tot * LEN, &rec));
    RPBD_TRY(ensure_t(h, BUF_BSCALE, (size_t)n_tot, &scale));
    RPBD_TRY(ensure_t(h, BUF_BPARTIAL, (size_t)p->max_slots * 3 * K * n_tot, &partial));
    SysTab tab{p->d_off, p->d_rec_off, p->d_nslots};
    bpack2_kernel<K, In><<<(unsigned)((p->rec_tot + 255) / 256), 256, 0, st>>>(n_sys, n_tot, p->rec_tot, k, tab, r, F,
                                                                               h->p.a, h->p.s_min, rec, scale);
    count_launch();
    const size_t smem = (size_t)B_NST * TS * LEN * sizeof(float) + B_NST * sizeof(uint64_t);
    auto kern = bpair2_kernel<K, BT, TS, B_NST>;
    if (smem > 48 * 1024) RPBD_CU(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (p->grid == 0) {
        int blocks = 0;
        RPBD_TRY((occupancy2<K, BT, TS>(&blocks)));
        p->grid = std::max(1, blocks) * h->sm_count;
    }
    RPBD_CU(h, cudaMemsetAsync(p->d_queue, 0, sizeof(int), st));
    if (h->profile) prof_begin(h, st);
    kern<<<p->grid, BT, smem, st>>>(rec, tab, p->d_items, p->n_items, p->d_queue, active, partial, n_tot, h->dev_flag);
    count_launch();
    if (h->profile) {
        double pairs = 0.0;
        for (int s = 0; s < n_sys; ++s) {
            const double ns = (double)(p->off[s + 1] - p->off[s]);
            pairs += ns * ns;
        }
        prof_end(h, st, prof_kind, K, pairs);
    }
    // blocks were formed in units of a: M = M(a = 1) / a
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta * h->p.a);
    breduce_kernel<Out><<<dim3((unsigned)((n_tot + 255) / 256), (unsigned)(3 * k)), 256, 0, st>>>(n_sys, n_tot, k, K, tab, partial, scale,
                                                                         active, inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

template <int K, bool WALL, class In, class Out>
static int run_k(rpbd_handle* h, BatchPlan* p, int n_sys, const double* r, const In* F, Out* U, int k,
                 const int* active, int pk, cudaStream_t st)
{
    switch (p->variant) {
    case 1: return run_variant<K, 64, 64, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
    case 2: return run_variant<K, 256, 32, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
    case 3:
        if constexpr (WALL) return run_variant2<K, 128, 64>(h, p, n_sys, r, F, U, k, active, pk, st);
        else return set_error(h, RPBD_BAD_ARG, "batched: the packed variant needs the wall");
    default: return run_variant<K, 128, 64, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
    }
}

template <bool WALL, class In, class Out>
static int run_dispatch(rpbd_handle* h, BatchPlan* p, int n_sys, const double* r, const In* F, Out* U, int k,
                        const int* active, int pk, cudaStream_t st)
{
    if (k <= 1) return run_k<1, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
    if (k <= 4) return run_k<4, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
    return run_k<16, WALL>(h, p, n_sys, r, F, U, k, active, pk, st);
}

// find or build the plan of this batch for the handle's chosen variant
static int get_plan(rpbd_handle* h, int n_sys, const int64_t* off, int k, int variant, BatchPlan** out)
{
    for (BatchPlan* p : h->bplans) {
        if (p->variant == variant && (int)p->off.size() == n_sys + 1 &&
            std::equal(p->off.begin(), p->off.end(), off)) {
            *out = p;
            return RPBD_OK;
        }
    }
    BatchPlan* p = nullptr;
    RPBD_TRY(build_plan(h, off, n_sys, k, variant, &p));
    h->bplans.push_back(p);
    *out = p;
    return RPBD_OK;
}

int batched_apply_impl(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const void* F, void* U, int k,
                       bool io_double, const int* active, cudaStream_t st)
{
    if (n_sys <= 0) return set_error(h, RPBD_BAD_ARG, "batched: n_sys <= 0");
    if (h->p.Lx > 0.0) return set_error(h, RPBD_BAD_ARG, "batched: systems are open in x, y (no periodic cell)");
    if (k < 1 || k > 16) return set_error(h, RPBD_BAD_ARG, "batched: k must be in 1..16");
    for (int s = 0; s < n_sys; ++s)
        if (off[s + 1] < off[s] || (off[s + 1] - off[s]) > (int64_t)1 << 30)
            return set_error(h, RPBD_BAD_ARG, "batched: offsets must be non-decreasing");
    if (off[0] != 0) return set_error(h, RPBD_BAD_ARG, "batched: offsets must start at 0");
    if (off[n_sys] == 0) return RPBD_OK;
    // variant 4: the packed symmetric kernel over the batch (k <= 4 with the wall;
    // the default there: 7.7 vs 11.7 ms for the 64-system boomerang batch)
    const int want = h->batch_variant >= 0 ? h->batch_variant : (h->p.wall ? 4 : 0);
    if (want == 4 && k <= 4) return sym_batched_apply_impl(h, n_sys, off, r, F, U, k, io_double, active, st);
    BatchPlan* p = nullptr;
    // k > 4 on the symmetric variant: the packed one-direction tile (two targets per thread)
    const int variant = want == 4 ? 3 : want;
    RPBD_TRY(get_plan(h, n_sys, off, k, variant, &p));
    const bool wall = h->p.wall != 0;
    if (io_double)
        return wall ? run_dispatch<true>(h, p, n_sys, r, (const double*)F, (double*)U, k, active, 2, st)
                    : run_dispatch<false>(h, p, n_sys, r, (const double*)F, (double*)U, k, active, 2, st);
    return wall ? run_dispatch<true>(h, p, n_sys, r, (const float*)F, (float*)U, k, active, 2, st)
                : run_dispatch<false>(h, p, n_sys, r, (const float*)F, (float*)U, k, active, 2, st);
}

int single_packed_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k,
                             bool io_double, cudaStream_t st)
{
    if (!h->p.wall || h->p.Lx > 0.0 || k < 1 || k > 4 || n <= 0 || n > (int64_t)1 << 30)
        return set_error(h, RPBD_BAD_ARG, "packed one-direction matvec: wall, open cell, 1 <= k <= 4");
    // the work list depends on n only; it is kept apart from the batch plans
    // (which captured graphs may reference) and rebuilt when n changes
    const int64_t off[2] = {0, n};
    if (h->mv_plan && h->mv_plan->off[1] != n) {
        RPBD_CU(h, cudaStreamSynchronize(st));
        free_plan(h->mv_plan);
        h->mv_plan = nullptr;
    }
    if (!h->mv_plan) RPBD_TRY(build_plan(h, off, 1, k, 3, &h->mv_plan));
    BatchPlan* p = h->mv_plan;
    if (io_double)
        return k == 1 ? run_k<1, true>(h, p, 1, r, (const double*)F, (double*)U, k, nullptr, RPBD_F32, st)
                      : run_k<4, true>(h, p, 1, r, (const double*)F, (double*)U, k, nullptr, RPBD_F32, st);
    return k == 1 ? run_k<1, true>(h, p, 1, r, (const float*)F, (float*)U, k, nullptr, RPBD_F32, st)
                  : run_k<4, true>(h, p, 1, r, (const float*)F, (float*)U, k, nullptr, RPBD_F32, st);
}

void batched_free_plans(rpbd_handle* h)
{
    for (BatchPlan* p : h->bplans) free_plan(p);
    h->bplans.clear();
    free_sym2_plans(h);
    free_plan(h->mv_plan);
    h->mv_plan = nullptr;
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

int rpbd_mobility_apply_batched(rpbd_handle* h, int n_sys, const int64_t* offsets, const double* r, const float* F,
                                float* U, int k, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!offsets || !r || !F || !U) return set_error(h, RPBD_BAD_ARG, "batched: null pointer");
    return batched_apply_impl(h, n_sys, offsets, r, F, U, k, false, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_autotune_batched(rpbd_handle* h, int n_sys, const int64_t* offsets, const double* r, int k, double* best_ms,
                          void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!offsets || !r || n_sys <= 0 || k < 1 || k > 16) return set_error(h, RPBD_BAD_ARG, "autotune: bad arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_tot = offsets[n_sys];
    float *F, *U;
    RPBD_TRY(ensure_t(h, BUF_BAUX, (size_t)2 * k * 3 * n_tot, &F));
    U = F + (size_t)k * 3 * n_tot;
    RPBD_CU(h, cudaMemsetAsync(F, 0, sizeof(float) * k * 3 * n_tot, st));
    cudaEvent_t e0, e1;
    RPBD_CU(h, cudaEventCreate(&e0));
    RPBD_CU(h, cudaEventCreate(&e1));
    double best = 1e300;
    int best_v = 0;
    // the tile variants, then (k <= 4 with the wall) the packed symmetric kernel
    for (int v = 0; v <= N_VARIANTS; ++v) {
        if (v < N_VARIANTS && VARIANTS[v].packed && !h->p.wall) continue;
        if (v == N_VARIANTS && (!h->p.wall || k > 4)) continue;
        h->batch_variant = v;
        RPBD_TRY(batched_apply_impl(h, n_sys, offsets, r, F, U, k, false, nullptr, st));  // warm-up, plan
        RPBD_CU(h, cudaEventRecord(e0, st));
        for (int rep = 0; rep < 3; ++rep) RPBD_TRY(batched_apply_impl(h, n_sys, offsets, r, F, U, k, false, nullptr, st));
        RPBD_CU(h, cudaEventRecord(e1, st));
        RPBD_CU(h, cudaEventSynchronize(e1));
        float ms = 0.0f;
        RPBD_CU(h, cudaEventElapsedTime(&ms, e0, e1));
        if (ms / 3.0 < best) {
            best = ms / 3.0;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->batch_variant = best_v;
    if (best_ms) *best_ms = best;
    return best_v;
}

}  // extern "C"
