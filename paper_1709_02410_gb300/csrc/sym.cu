// Symmetric FP32 wall-RPY matvec for few right-hand sides (k <= 4).
//
// M is symmetric blockwise, M_ji = M_ij^T (Sec. 2.1: the blob mobility
// matrix is symmetric), so one evaluation of the 3x3 block of an unordered
// pair {i, j} serves both U_i += M_ij F_j and U_j += M_ij^T F_i.  This kernel
// forms each block once:
//
//  * home tile H: 128 blobs, one per thread (4 warps x 32), positions and
//    forces in registers, accumulating U_i over the item;
//  * visitors: the blobs after the home tile, streamed through shared memory
//    in tiles of 32 records by the TMA bulk ring (as in mobility.cu);
//  * inside a warp, lane l takes visitor (s + l) mod 32 at step s, so the 32
//    lanes work on 32 different visitors; each lane carries the visitor's
//    running sum of M^T F_i and hands it to lane l - 1 by one shuffle per
//    component after every step -- after 32 steps every visitor's sum over
//    the warp's 32 homes is back in lane (visitor index);
//  * the four warps' visitor sums are added in shared memory (double-
//    buffered, so one barrier per tile) and stored as one partial per (home
//    tile, visitor); home sums are stored per chunk;
//  * pairs inside a home tile (and the self block) are done by a diagonal
//    item in the plain one-direction form.
// Two reduce kernels add, for blob i, the visitor partials of every home tile
// before i's tile and the home partials of i's own tile in a fixed order
// (compensated FP32 pairs widened to FP64; deterministic), then apply
// s_i / (8 pi eta).  The packed variant below (two homes per thread) also
// runs over a batch of independent systems: each system padded to whole home
// tiles, with its own partial and segment-sum regions (SymSys).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "accum.cuh"
#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"
#include "fixed_point.cuh"
#include "wall_rpy_x2.cuh"

namespace rpbd {
namespace sym {

constexpr int HT = 128;    // home tile (threads per CTA)
constexpr int VT = 32;     // visitor tile (records per stage)
constexpr int NST = 4;     // TMA ring depth
constexpr int CHUNK = 2048;  // visitors per off-diagonal item (at most; see get_items)

template <int K>
struct Rec {
    static constexpr int TAIL = ((1 + 3 * K) + 3) / 4 * 4;
    static constexpr int LEN = 4 + TAIL;
};

// tuning variants per K: visitor-loop unroll and minimum resident CTAs per SM
// (the latter caps registers: 65536 / (MINB * 128)); chosen so no variant spills
template <int K, int V, bool PER = false>
struct SymVar {
    static constexpr int UNR = V == 1 ? 1 : (V == 3 ? 4 : 2);
    static constexpr int MINB0 = K == 1 ? (V == 2 ? 9 : 8) : (K == 2 ? (V == 2 ? 8 : 7) : (V == 2 ? 5 : 4));
    // the image loop of the periodic cell needs more registers
    static constexpr int PCAP = K == 1 ? 6 : (K == 2 ? 5 : 4);
    static constexpr int MINB = PER && MINB0 > PCAP ? PCAP : MINB0;
};

struct SymItem {
    int home;   // home tile index (global, in records)
    int v0;     // first visitor record (multiple of VT)
    int ntile;  // visitor tiles
    int slot;   // home-partial slot (0: diagonal item)
    int sys;    // system of a batch (0 for a single system)
};

// One system of the packed symmetric kernel's launch.  A single system has
// B = g0 = P1 = S1 = 0; a batch concatenates the systems' records, each
// padded to whole home tiles, and gives each its own partial and segment-sum
// regions, so pairs never cross systems.
struct SymSys {
    int64_t B;      // first record (multiple of the home tile)
    int64_t g0;     // first blob in the caller's concatenated vectors
    int64_t n;      // blobs
    int64_t n_pad;  // records (n rounded up to whole home tiles)
    int64_t P1;     // first float of the visitor/home partials, divided by 3K
    int64_t S1;     // first double of the segment sums, divided by 3K
    int T;          // home tiles
    int chunk;      // visitors per off-diagonal item
};

// system of global index x, given ascending starts base(s) (binary search)
template <class F>
__device__ __forceinline__ int sys_of(int n_sys, int64_t x, F base)
{
    int lo = 0, hi = n_sys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t c)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(c) : "memory");
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
// bounded wait: `limit` SM clock cycles at most (default ~2 s); false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = 4000000000LL)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

template <int K, class In>
__global__ void pack_kernel(int64_t n, int64_t n_pad, int k, const double* __restrict__ r, const In* __restrict__ F,
                            double a, int wall, double s_min, float* __restrict__ rec, double* __restrict__ scale)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    constexpr int LEN = Rec<K>::LEN;
    float* o = rec + i * LEN;
    double x = 1.0e7, y = 1.0e7, zt = a, s = 0.0;
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
    }
    const float xh = (float)x, yh = (float)y;
    o[0] = xh;
    o[1] = yh;
    o[2] = (float)(x - (double)xh);
    o[3] = (float)(y - (double)yh);
    o[4] = (float)zt;
#pragma unroll
    for (int q = 1; q < Rec<K>::TAIL; ++q) o[4 + q] = 0.0f;
    if (i < n)
        for (int m = 0; m < k; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) o[5 + 3 * m + c] = (float)(s * (double)F[((int64_t)m * 3 + c) * n + i]);
}

template <int K>
__device__ __forceinline__ void load_rec(const float* rj, float& xh, float& yh, float& xl, float& yl, float& z,
                                         float* f)
{
    const float4 p = *reinterpret_cast<const float4*>(rj);
    xh = p.x; yh = p.y; xl = p.z; yl = p.w;
    float tail[Rec<K>::TAIL];
#pragma unroll
    for (int q = 0; q < Rec<K>::TAIL / 4; ++q) {
        const float4 v = reinterpret_cast<const float4*>(rj + 4)[q];
        tail[4 * q] = v.x; tail[4 * q + 1] = v.y; tail[4 * q + 2] = v.z; tail[4 * q + 3] = v.w;
    }
    z = tail[0];
#pragma unroll
    for (int q = 0; q < 3 * K; ++q) f[q] = tail[1 + q];
}

template <int K, bool WALL, bool PER, int UNR, int MINB>
__global__ void __launch_bounds__(HT, MINB) sym_kernel(const float* __restrict__ rec, int64_t n, int64_t n_pad,
                                                 const SymItem* __restrict__ items, int n_home_tiles, PairConst<float> pc,
                                                 float* __restrict__ partial, int* __restrict__ err_flag, RingTest rt)
{
    constexpr int LEN = Rec<K>::LEN;
    constexpr uint32_t TILE_BYTES = VT * LEN * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    float* red = reinterpret_cast<float*>(smem_raw + NST * TILE_BYTES);  // [2 buffers][4 warps][VT][3K]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NST * TILE_BYTES + 2 * 4 * VT * 3 * K * sizeof(float));
    const SymItem it = items[blockIdx.x];
    const bool diag = it.slot == 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)it.home * HT + tid;  // home blob (i < n_pad always)
    // one or two right-hand sides in an open cell: skip assembling the block
    constexpr bool FACTORED = K <= 2 && !PER;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)  // (failure-path test: stage 0 gets no copy, so its wait runs out)
        for (int s = rt.skip_first ? 1 : 0; s < NST && s < it.ntile; ++s) {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * VT * LEN, rec + ((size_t)it.v0 + (size_t)s * VT) * LEN, TILE_BYTES, &bar[s]);
        }
    float hxh, hyh, hxl, hyl, hz, hf[3 * K];
    load_rec<K>(rec + i * LEN, hxh, hyh, hxl, hyl, hz, hf);
    float acc[3 * K];
#pragma unroll
    for (int q = 0; q < 3 * K; ++q) acc[q] = 0.0f;

    int t = 0;
    bool bad = false;
    for (; t < it.ntile; ++t) {
        const int s = t % NST;
        const bool ok = mbar_wait_bounded(&bar[s], (t / NST) & 1, rt.limit);
        const float* st = stage + (size_t)s * VT * LEN;
        if (ok && diag) {
            // one direction, all lanes on the same source (broadcast reads)
#pragma unroll 2
            for (int jj = 0; jj < VT; ++jj) {
                float xh, yh, xl, yl, zj, f[3 * K];
                load_rec<K>(st + jj * LEN, xh, yh, xl, yl, zj, f);
                const float dx = (hxh - xh) + (hxl - xl), dy = (hyh - yh) + (hyl - yl);
                float Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz;
                pair_block_images<float, float, WALL, PER>(dx, dy, hz - zj, hz, zj, pc, Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz);
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    const float fx = f[3 * m], fy = f[3 * m + 1], fz = f[3 * m + 2];
                    acc[3 * m + 0] = fmaf(Mxz, fz, fmaf(Mxy, fy, fmaf(Mxx, fx, acc[3 * m + 0])));
                    acc[3 * m + 1] = fmaf(Myz, fz, fmaf(Myy, fy, fmaf(Mxy, fx, acc[3 * m + 1])));
                    acc[3 * m + 2] = fmaf(Mzz, fz, fmaf(Mzy, fy, fmaf(Mzx, fx, acc[3 * m + 2])));
                }
            }
        } else if (ok) {
            // both directions; lane l takes visitor (step + l) mod 32
            float vacc[3 * K];
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) vacc[q] = 0.0f;
#pragma unroll UNR
            for (int step = 0; step < VT; ++step) {
                const int v = (step + lane) & (VT - 1);
                float xh, yh, xl, yl, zj, f[3 * K];
                load_rec<K>(st + v * LEN, xh, yh, xl, yl, zj, f);
                const float dx = (hxh - xh) + (hxl - xl), dy = (hyh - yh) + (hyl - yl);
                if constexpr (FACTORED) {
                    // apply the block in factored form, both directions (no
                    // assembly of the 9 entries)
                    float al, be, gxx, gzz, Mzz;
                    pair_factors<float, float, WALL>(dx, dy, hz - zj, hz, zj, pc, al, be, gxx, gzz, Mzz);
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        const float fx = f[3 * m], fy = f[3 * m + 1], fz = f[3 * m + 2];
                        const float P = fmaf(dy, fy, dx * fx);
                        const float Q = fmaf(be, P, gxx * fz);
                        acc[3 * m + 0] = fmaf(dx, Q, fmaf(al, fx, acc[3 * m + 0]));
                        acc[3 * m + 1] = fmaf(dy, Q, fmaf(al, fy, acc[3 * m + 1]));
                        acc[3 * m + 2] = fmaf(Mzz, fz, fmaf(gzz, P, acc[3 * m + 2]));
                        // M^T applied to the home force
                        const float hx = hf[3 * m], hy = hf[3 * m + 1], hzf = hf[3 * m + 2];
                        const float Pt = fmaf(dy, hy, dx * hx);
                        const float Qt = fmaf(be, Pt, gzz * hzf);
                        vacc[3 * m + 0] = fmaf(dx, Qt, fmaf(al, hx, vacc[3 * m + 0]));
                        vacc[3 * m + 1] = fmaf(dy, Qt, fmaf(al, hy, vacc[3 * m + 1]));
                        vacc[3 * m + 2] = fmaf(Mzz, hzf, fmaf(gxx, Pt, vacc[3 * m + 2]));
                    }
                } else {
                    float Mxx, Mxy, Mxz, Myy, Myz, Mzx, Mzy, Mzz;
                    pair_block_images<float, float, WALL, PER>(dx, dy, hz - zj, hz, zj, pc, Mxx, Mxy, Mxz, Myy, Myz, Mzx,
                                                               Mzy, Mzz);
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        const float fx = f[3 * m], fy = f[3 * m + 1], fz = f[3 * m + 2];
                        acc[3 * m + 0] = fmaf(Mxz, fz, fmaf(Mxy, fy, fmaf(Mxx, fx, acc[3 * m + 0])));
                        acc[3 * m + 1] = fmaf(Myz, fz, fmaf(Myy, fy, fmaf(Mxy, fx, acc[3 * m + 1])));
                        acc[3 * m + 2] = fmaf(Mzz, fz, fmaf(Mzy, fy, fmaf(Mzx, fx, acc[3 * m + 2])));
                        const float gx = hf[3 * m], gy = hf[3 * m + 1], gz = hf[3 * m + 2];
                        // M^T applied to the home force
                        vacc[3 * m + 0] = fmaf(Mzx, gz, fmaf(Mxy, gy, fmaf(Mxx, gx, vacc[3 * m + 0])));
                        vacc[3 * m + 1] = fmaf(Mzy, gz, fmaf(Myy, gy, fmaf(Mxy, gx, vacc[3 * m + 1])));
                        vacc[3 * m + 2] = fmaf(Mzz, gz, fmaf(Myz, gy, fmaf(Mxz, gx, vacc[3 * m + 2])));
                    }
                }
                // hand the visitor sums to the lane that takes that visitor next
#pragma unroll
                for (int q = 0; q < 3 * K; ++q) vacc[q] = __shfl_sync(0xffffffffu, vacc[q], (lane + 1) & 31);
            }
            // lane l now holds visitor l's sum over this warp's homes
            float* rb = red + (t & 1) * (4 * VT * 3 * K);  // double-buffered: one barrier per tile
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) rb[(warp * VT + lane) * 3 * K + q] = vacc[q];
        }
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        if (!diag) {
            // add the four warps' visitor sums of this tile; the next tile writes
            // the other buffer, and the one after that comes only after the
            // next barrier, which every thread reaches after finishing here
            const float* rb = red + (t & 1) * (4 * VT * 3 * K);
            const int64_t vbase = (int64_t)it.v0 + (int64_t)t * VT;
            for (int e = tid; e < VT * 3 * K; e += HT) {
                const int vl = e / (3 * K), q = e % (3 * K);
                const int64_t vg = vbase + vl;
                if (vg < n) {
                    const float sum = rb[(0 * VT + vl) * 3 * K + q] + rb[(1 * VT + vl) * 3 * K + q] +
                                      rb[(2 * VT + vl) * 3 * K + q] + rb[(3 * VT + vl) * 3 * K + q];
                    partial[((int64_t)it.home * 3 * K + q) * n_pad + vg] = sum;
                }
            }
        }
        if (tid == 0 && t + NST < it.ntile) {
            fence_proxy_async();
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * VT * LEN, rec + ((size_t)it.v0 + (size_t)(t + NST) * VT) * LEN, TILE_BYTES,
                        &bar[s]);
        }
    }
    if (bad) {
        if (tid == 0) {
            atomicExch(err_flag, 1);
            for (int u = t + 1; u < it.ntile && u < t + NST; ++u) mbar_wait_bounded(&bar[u % NST], (u / NST) & 1);
        }
        return;
    }
    if (i < n) {
        const int slot = n_home_tiles + it.slot;
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) partial[((int64_t)slot * 3 * K + q) * n_pad + i] = acc[q];
    }
}

// Visitor partials are reduced in two passes so the triangular sum over the
// home tiles before blob i's tile spreads over many threads (several loads in
// flight each): pass 1 sums home tiles [s SEG, (s+1) SEG) for segment s =
// blockIdx.y; pass 2 adds the segments and the home partials, then scales.
// Both passes use a fixed order (deterministic).  The FP32 partials are
// accumulated as compensated float pairs (accum.cuh), widened to FP64 once
// per segment.
constexpr int SEG = 16;  // home tiles per segment

template <int HTT, int KT, class P>
__global__ void reduce_visitors_kernel(int64_t n, int64_t n_pad, int k, const P* __restrict__ partial,
                                       double* __restrict__ segsum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int h = (int)(i / HTT);
    const int H0 = blockIdx.y * SEG;
    const int H1 = (H0 + SEG) < h ? (H0 + SEG) : h;
    if (H0 >= H1) return;
    float s[3 * KT], c[3 * KT];
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q) s[q] = c[q] = 0.0f;
    // four home tiles' loads issued together, then added in home-tile order
    int H = H0;
    for (; H + 4 <= H1; H += 4) {
        P v[4][3 * KT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 3 * KT; ++q)
                v[u][q] = q < 3 * k ? partial[((int64_t)(H + u) * 3 * KT + q) * n_pad + i] : P(0);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 3 * KT; ++q) two_sum_acc(s[q], c[q], v[u][q]);
    }
    for (; H < H1; ++H)
#pragma unroll
        for (int q = 0; q < 3 * KT; ++q)
            if (q < 3 * k) two_sum_acc(s[q], c[q], partial[((int64_t)H * 3 * KT + q) * n_pad + i]);
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q)
        if (q < 3 * k) segsum[((int64_t)blockIdx.y * 3 * KT + q) * n_pad + i] = two_sum_value(s[q], c[q]);
}

template <int HTT, class P, class Out>
__global__ void reduce_kernel(int64_t n, int64_t n_pad, int k, int kt, int n_home_tiles, int chunk,
                              const P* __restrict__ partial, const double* __restrict__ segsum,
                              const double* __restrict__ scale, double inv8pieta, Out* __restrict__ U)
{
    // one thread per (blob, component q = blockIdx.y < 3k)
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= n || q >= 3 * k) return;
    const int h = (int)(i / HTT);
    const int nseg = (h + SEG - 1) / SEG;
    const int64_t vis = n_pad - (int64_t)(h + 1) * HTT;  // visitors of tile h
    const int home_slots = 1 + (int)((vis + chunk - 1) / chunk);
    double sum = 0.0;
    for (int sg = 0; sg < nseg; ++sg) sum += segsum[((int64_t)sg * 3 * kt + q) * n_pad + i];
    float hs = 0.0f, hc = 0.0f;
    for (int c = 0; c < home_slots; ++c)
        two_sum_acc(hs, hc, (float)partial[((int64_t)(n_home_tiles + c) * 3 * kt + q) * n_pad + i]);
    sum += two_sum_value(hs, hc);
    U[(int64_t)q * n + i] = (Out)(scale[i] * inv8pieta * sum);
}

// Work items of the symmetric kernels for home tiles of TILE blobs: per home
// tile one diagonal item (slot 0) and one item per `chunk` visitors after it.
// The chunk is CHUNK, halved (down to one visitor tile) while the items would
// not fill 4 CTAs per SM, so small suspensions still spread over the GPU.
// Cached per n (the one-home kernel; the packed kernel's lists are Sym2Plan).
template <int TILE>
static int get_items(rpbd_handle* h, int64_t n, int64_t n_pad, SymItem** d_items, int* n_items, int* n_home,
                     int* max_slots, int* chunk_out)
{
    SymPlan& pl = h->sym_plan;
    if (pl.n != n) {
        std::vector<SymItem> items;
        const int T = (int)(n_pad / TILE);
        int chunk = CHUNK;
        auto count = [&](int c) {
            int64_t m = T;
            for (int H = 0; H < T; ++H) m += (n_pad - (int64_t)(H + 1) * TILE + c - 1) / c;
            return m;
        };
        while (chunk > VT && count(chunk) < 4 * (int64_t)h->sm_count) chunk /= 2;
        int ms = 1;
        for (int H = 0; H < T; ++H) {
            items.push_back(SymItem{H, H * TILE, TILE / VT, 0, 0});
            int c = 1;
            for (int64_t v0 = (int64_t)(H + 1) * TILE; v0 < n_pad; v0 += chunk, ++c) {
                const int64_t v1 = std::min<int64_t>(n_pad, v0 + chunk);
                items.push_back(SymItem{H, (int)v0, (int)((v1 - v0) / VT), c, 0});
            }
            ms = std::max(ms, c);
        }
        // longest items first so the hardware scheduler fills the tail with short ones
        std::stable_sort(items.begin(), items.end(), [](const SymItem& a, const SymItem& b) { return a.ntile > b.ntile; });
        void* d = nullptr;
        RPBD_TRY(ensure(h, BUF_SYM_ITEMS, items.size() * sizeof(SymItem), &d));
        RPBD_CU(h, cudaMemcpy(d, items.data(), items.size() * sizeof(SymItem), cudaMemcpyHostToDevice));
        pl.n = n;
        pl.n_items = (int)items.size();
        pl.n_home = T;
        pl.max_slots = ms;
        pl.chunk = chunk;
    }
    *d_items = reinterpret_cast<SymItem*>(h->buf[BUF_SYM_ITEMS]);
    *n_items = pl.n_items;
    *n_home = pl.n_home;
    *max_slots = pl.max_slots;
    *chunk_out = pl.chunk;
    return RPBD_OK;
}

template <int K, bool WALL, bool PER, class In, class Out>
static int run(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    constexpr int LEN = Rec<K>::LEN;
    const int64_t n_pad = (n + HT - 1) / HT * HT;
    SymItem* items;
    int n_items, n_home, max_slots;
    int chunk;
    RPBD_TRY(get_items<HT>(h, n, n_pad, &items, &n_items, &n_home, &max_slots, &chunk));
    float* rec;
    double* scale;
    float* partial;
    RPBD_TRY(ensure_t(h, BUF_PACK, (size_t)n_pad * LEN, &rec));
    RPBD_TRY(ensure_t(h, BUF_SCALE, (size_t)n_pad, &scale));
    RPBD_TRY(ensure_t(h, BUF_PARTIAL, (size_t)(n_home + max_slots) * 3 * K * n_pad, &partial));
    pack_kernel<K, In><<<(unsigned)((n_pad + 255) / 256), 256, 0, st>>>(n, n_pad, k, r, F, h->p.a, h->p.wall,
                                                                        h->p.s_min, rec, scale);
    count_launch();
    const size_t smem = (size_t)NST * VT * LEN * sizeof(float) + 2 * 4 * VT * 3 * K * sizeof(float) + NST * sizeof(uint64_t);
    const PairConst<float> pc = PairConst<float>::make(h->p.a, h->p.Lx, h->p.Ly);
    if (h->profile) prof_begin(h, st);
    // variant -1: the measured default per K (k <= 2: unroll 4; otherwise unroll 2)
    const int sv = h->sym_variant[sym_class(K)];
    const int var = sv >= 0 ? sv : (K <= 2 ? 3 : 0);
    const RingTest rt = ring_test(h);
    switch (var) {  // tuning variants: (visitor-loop unroll, min CTAs per SM), see SymVar
    case 1: sym_kernel<K, WALL, PER, SymVar<K, 1, PER>::UNR, SymVar<K, 1, PER>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag, rt); break;
    case 2: sym_kernel<K, WALL, PER, SymVar<K, 2, PER>::UNR, SymVar<K, 2, PER>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag, rt); break;
    case 3: sym_kernel<K, WALL, PER, SymVar<K, 3, PER>::UNR, SymVar<K, 3, PER>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag, rt); break;
    default: sym_kernel<K, WALL, PER, SymVar<K, 0, PER>::UNR, SymVar<K, 0, PER>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag, rt); break;
    }
    count_launch();
    if (h->profile) prof_end(h, st, (K <= 2 && !PER) ? 4 /* symmetric, factored */ : 3 /* symmetric */, K,
                             (double)n * (double)n);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const int nseg = (n_home + SEG - 1) / SEG;
    double* segsum;
    RPBD_TRY(ensure_t(h, BUF_SYM_SEG, (size_t)nseg * 3 * K * n_pad, &segsum));
    reduce_visitors_kernel<HT, K, float><<<dim3((unsigned)((n + 255) / 256), (unsigned)nseg), 256, 0, st>>>(
        n, n_pad, k, partial, segsum);
    count_launch();
    reduce_kernel<HT, float, Out><<<dim3((unsigned)((n + 255) / 256), (unsigned)(3 * k)), 256, 0, st>>>(n, n_pad, k, K, n_home, chunk,
                                                                               partial, segsum, scale, inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

// ---------------------------------------------------------------------------
// Packed variant for k <= 4 with the wall, open or pseudo-periodic cell (k =
// 1, 2: the Krylov matvecs of a time step).  Each thread holds two home blobs (256 per CTA)
// and meets every visitor with both at once: the two pair blocks are formed
// in the .x / .y lanes of float2 values with packed two-wide FP32
// instructions (wall_rpy_x2.cuh), so one instruction stream serves two pairs.
// The visitor's running sums carry both homes' contributions (.x, .y) and are
// added only when the tile's sums go to shared memory.  Source records are
// stored with every field duplicated ([xh xh yh yh][xl xl yl yl][z z fx fx]
// ...) so a 16-byte shared load yields two packed operands, and transposed
// within each 32-record tile (field chunk c of record j at (c * 32 + j) * 4
// floats) so the 32 lanes' loads of different records hit distinct banks.

constexpr int HT2 = 256;  // home blobs per CTA, two per thread
// beyond this many bytes of per-home-tile visitor partials a single system
// always takes the fixed-point accumulation below
constexpr double SYM_PARTIAL_LIMIT = 16.0 * (1ull << 30);

// single-system accumulation in fixed point (fixed_point.cuh): every block
// entry is at most the self term 4/3 in units of a (nine images in the
// periodic cell), so a velocity component is at most 4 n max|F| (x 9)
__host__ __device__ constexpr double fixed_cap(bool per) { return per ? 36.0 : 4.0; }

template <int K>
struct Rec2 {
    static constexpr int NV = 5 + 3 * K;        // values: x_hi, y_hi, x_lo, y_lo, z, forces
    static constexpr int NCH = (NV + 1) / 2;    // 16-byte chunks per record (two values each)
    static constexpr int LEN = 4 * NCH;         // floats per record
};

__host__ __device__ __forceinline__ int64_t rec2_off(int64_t i, int c, int len)
{
    return (i / VT) * VT * len + ((int64_t)c * VT + (i % VT)) * 4;
}

// One thread per record of the launch (all systems, padded to whole home
// tiles); padding records sit far away with zero force.
template <int K, class In>
__global__ void pack2_kernel(int n_sys, const SymSys* __restrict__ sys, int64_t rec_end, int64_t n_tot, int k,
                             const double* __restrict__ r, const In* __restrict__ F, double a, int wall, double s_min,
                             const int* __restrict__ active, float* __restrict__ rec, double* __restrict__ scale,
                             unsigned* __restrict__ fmax_bits = nullptr)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= rec_end) return;
    constexpr int NCH = Rec2<K>::NCH, LEN = Rec2<K>::LEN;
    const int sx = n_sys == 1 ? 0 : sys_of(n_sys, j, [&](int m) { return sys[m].B; });
    if (active && !active[sx]) return;  // a converged system of a batch: its records are not read
    const int64_t l = j - sys[sx].B;
    const bool real = l < sys[sx].n;
    const int64_t i = sys[sx].g0 + l;  // the blob's index in the caller's vectors
    double x = 1.0e7, y = 1.0e7, zt = a, s = 0.0;
    if (real) {
        x = r[i];
        y = r[n_tot + i];
        const double z = r[2 * n_tot + i];
        if (wall) {
            zt = z > a ? z : a;
            const double t = z / a;
            s = t >= 1.0 ? 1.0 : (t <= s_min ? s_min : t);
        } else {
            zt = z;
            s = 1.0;
        }
        scale[i] = s;
    }
    float v[2 * NCH];
#pragma unroll
    for (int q = 0; q < 2 * NCH; ++q) v[q] = 0.0f;
    // lengths in units of a (the packed pair form takes a = 1)
    const double ia = 1.0 / a;
    x *= ia;
    y *= ia;
    zt *= ia;
    const float xh = (float)x, yh = (float)y;
    v[0] = xh;
    v[1] = yh;
    v[2] = (float)(x - (double)xh);
    v[3] = (float)(y - (double)yh);
    v[4] = (float)zt;
    float fm = 0.0f;
    if (real)
        for (int m = 0; m < k; ++m)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[5 + 3 * m + c] = (float)(s * (double)F[((int64_t)m * 3 + c) * n_tot + i]);
                fm = isfinite(v[5 + 3 * m + c]) ? fmaxf(fm, fabsf(v[5 + 3 * m + c])) : INFINITY;
            }
#pragma unroll
    for (int c = 0; c < NCH; ++c)
        *reinterpret_cast<float4*>(rec + rec2_off(j, c, LEN)) = make_float4(v[2 * c], v[2 * c], v[2 * c + 1], v[2 * c + 1]);
    // largest |force| of the record's system and its non-finite flag (a warp never
    // straddles two systems: each is padded to whole 256-record home tiles)
    if (fmax_bits) fixed_force_max(fmax_bits + 2 * sx, fm);
}

// record j of a staged tile -> packed operands (both lanes equal); value m
// sits in chunk m / 2, lanes (0, 1) for even m and (2, 3) for odd m
template <int K>
__device__ __forceinline__ void load_rec2(const float* st, int j, float2& xh, float2& yh, float2& xl, float2& yl,
                                          float2& z, float2* f)
{
    const float4* p = reinterpret_cast<const float4*>(st) + j;
    float2 v[2 * Rec2<K>::NCH];
#pragma unroll
    for (int c = 0; c < Rec2<K>::NCH; ++c) {
        const float4 q = p[c * VT];
        v[2 * c] = make_float2(q.x, q.y);
        v[2 * c + 1] = make_float2(q.z, q.w);
    }
    xh = v[0];
    yh = v[1];
    xl = v[2];
    yl = v[3];
    z = v[4];
#pragma unroll
    for (int q = 0; q < 3 * K; ++q) f[q] = v[5 + q];
}

// Both directions (BOTH) or the home direction only, for one pair separation
// in packed form: acc += M f (visitor forces f), vacc += M^T hf (home forces).
template <int K, bool BOTH, bool FAR>
__device__ __forceinline__ void pair_apply2(float2 dx, float2 dy, float2 dz, float2 hz, float2 zj,
                                            const PairConstX2& pc, const float2* f, const float2* hf, float2* acc,
                                            float2* vacc)
{
    float2 al, be, gx, gz, mzz;
    pair_factors_x2<FAR>(dx, dy, dz, hz, zj, pc, al, be, gx, gz, mzz);
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const float2 fx = f[3 * m], fy = f[3 * m + 1], fz = f[3 * m + 2];
        if constexpr (BOTH) {
            // both directions, written so that consecutive instructions share
            // an operand in the same position (al, dx, dy, be, mzz): the
            // register file feeds such packed FMAs faster than ones that read
            // three fresh register pairs
            const float2 hx = hf[3 * m], hy = hf[3 * m + 1], hzf = hf[3 * m + 2];
            float2 a0 = fma2(al, fx, acc[3 * m + 0]);
            float2 a1 = fma2(al, fy, acc[3 * m + 1]);
            float2 v0 = fma2(al, hx, vacc[3 * m + 0]);
            float2 v1 = fma2(al, hy, vacc[3 * m + 1]);
            float2 P = mul2(dx, fx);
            float2 Pt = mul2(dx, hx);
            P = fma2(dy, fy, P);
            Pt = fma2(dy, hy, Pt);
            float2 Q = mul2(gx, fz);
            float2 Qt = mul2(gz, hzf);
            Q = fma2(be, P, Q);
            Qt = fma2(be, Pt, Qt);
            acc[3 * m + 0] = fma2(dx, Q, a0);
            vacc[3 * m + 0] = fma2(dx, Qt, v0);
            acc[3 * m + 1] = fma2(dy, Q, a1);
            vacc[3 * m + 1] = fma2(dy, Qt, v1);
            float2 a2 = fma2(mzz, fz, acc[3 * m + 2]);
            float2 v2 = fma2(mzz, hzf, vacc[3 * m + 2]);
            acc[3 * m + 2] = fma2(gz, P, a2);
            vacc[3 * m + 2] = fma2(gx, Pt, v2);
        } else {
            const float2 P = fma2(dy, fy, mul2(dx, fx));
            const float2 Q = fma2(be, P, mul2(gx, fz));
            acc[3 * m + 0] = fma2(dx, Q, fma2(al, fx, acc[3 * m + 0]));
            acc[3 * m + 1] = fma2(dy, Q, fma2(al, fy, acc[3 * m + 1]));
            acc[3 * m + 2] = fma2(mzz, fz, fma2(gz, P, acc[3 * m + 2]));
        }
    }
}

// pair_apply2 summed over the minimum image and its 8 nearest periodic images
// in x, y (Sec. 4.2); Lx, Ly in units of a
template <int K, bool BOTH, bool PER, bool FAR>
__device__ __forceinline__ void pair_apply2_images(float2 dx, float2 dy, float2 dz, float2 hz, float2 zj,
                                                   const PairConstX2& pc, float Lx, float Ly, const float2* f,
                                                   const float2* hf, float2* acc, float2* vacc)
{
    if constexpr (!PER) {
        pair_apply2<K, BOTH, FAR>(dx, dy, dz, hz, zj, pc, f, hf, acc, vacc);
    } else {
        const float iLx = 1.0f / Lx, iLy = 1.0f / Ly;
        dx = make_float2(dx.x - Lx * rintf(dx.x * iLx), dx.y - Lx * rintf(dx.y * iLx));
        dy = make_float2(dy.x - Ly * rintf(dy.x * iLy), dy.y - Ly * rintf(dy.y * iLy));
#pragma unroll
        for (int ia = -1; ia <= 1; ++ia)
#pragma unroll
            for (int ib = -1; ib <= 1; ++ib)
                pair_apply2<K, BOTH, FAR>(add2(dx, bc2((float)ia * Lx)), add2(dy, bc2((float)ib * Ly)), dz, hz, zj, pc,
                                     f, hf, acc, vacc);
    }
}

// tuning variants (visitor-loop unroll, min CTAs per SM, packed home pairs
// per thread); chosen per K so no variant spills.  Variants 0-3: two home
// blobs per thread (128 threads); 4-5: four (64 threads).
template <int K, int V, bool PER = false>
struct Sym2Var {
    static constexpr int HP = V >= 4 ? 2 : 1;
    // (the periodic cell's nine-image body is unrolled less, to bound the code size)
    static constexpr int UNR = V == 0 ? 2
                             : (V == 1 ? 1 : (V == 2 ? 2 : (V == 3 ? (K == 1 && !PER ? 16 : 4) : (V == 4 ? 1 : (PER ? 2 : (K == 1 ? 4 : 8))))));
    static constexpr int MINB0 = V >= 4 ? (K == 1 ? 8 : (K == 2 ? 5 : 4))
                                        : (K == 1 ? (V == 1 ? 6 : (V == 2 ? 5 : 4))
                                                  : (K == 2 ? (V == 2 ? 3 : 4) : (V == 1 ? 3 : 2)));
    // the image loop of the periodic cell needs more registers
    static constexpr int PCAP = HP == 1 ? (K == 1 ? 4 : 2) : (K == 1 ? 6 : 4);
    static constexpr int MINB = PER ? (MINB0 > PCAP ? PCAP : MINB0) : MINB0;
    static constexpr int NT = HT2 / (2 * HP);  // threads per CTA
    static size_t smem(int len)
    {
        return (size_t)NST * VT * len * sizeof(float) + 2 * (NT / 32) * VT * 3 * K * sizeof(float) +
               NST * sizeof(uint64_t);
    }
};

// BATCH: items of several systems (layout per item from sys[], converged
// systems skipped); otherwise one system of n blobs, n_pad records and
// n_home_tiles home tiles, given as arguments.  HP: packed home pairs per
// thread (1: two home blobs per thread, 128 threads; 2: four home blobs per
// thread, 64 threads, so each visitor record loaded and each visitor sum
// handed on serves twice the pairs).  Warp w owns homes [64 HP w, 64 HP (w+1))
// of the tile; pair p of a thread holds homes 64 HP w + 64 p + lane (.x) and
// that + 32 (.y).  FAR: the cancellation-free far-field block.  ATOM (one
// system): the visitor and home sums go into the fixed-point accumulators
// (partial = [3K][n_pad] 64-bit integers, fmax_bits after them) instead of
// the per-home-tile partials.
template <int K, bool PER, int UNR, int MINB, bool BATCH, int HP = 1, bool FAR = false, bool ATOM = false>
__global__ void __launch_bounds__(HT2 / (2 * HP), MINB) sym2_kernel(const float* __restrict__ rec,
                                                              const SymItem* __restrict__ items, int64_t n,
                                                              int64_t n_pad, int n_home_tiles,
                                                              const SymSys* __restrict__ sys,
                                                              const int* __restrict__ active, float Lx, float Ly,
                                                              float* __restrict__ partial, int* __restrict__ err_flag,
                                                              RingTest rt, const unsigned* __restrict__ fmax_bits = nullptr,
                                                              int64_t acc_stride = 0)
{
    constexpr int NT = HT2 / (2 * HP);  // threads
    constexpr int NW = NT / 32;          // warps
    constexpr int LEN = Rec2<K>::LEN;
    constexpr uint32_t TILE_BYTES = VT * LEN * sizeof(float);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stage = reinterpret_cast<float*>(smem_raw);
    float* red = reinterpret_cast<float*>(smem_raw + NST * TILE_BYTES);  // [2 buffers][NW warps][VT][3K]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NST * TILE_BYTES + 2 * NW * VT * 3 * K * sizeof(float));
    const SymItem it = items[blockIdx.x];
    if constexpr (BATCH)
        if (active && !active[it.sys]) return;  // a converged system: nothing in flight yet
    // a batch's layout is read again where partials are written (cached
    // loads), so none of it stays live in registers through the pair loop
    const SymSys* const sd = sys + it.sys;
    const bool diag = it.slot == 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ib = (int64_t)it.home * HT2 + warp * 64 * HP + lane;  // home record of pair 0, lane .x
    const PairConstX2 pc = PairConstX2::make_unit();
    const float2 m1 = pc.m1;
    // exponent S of the fixed-point scale 2^S of this item's system (ATOM)
    const int fexp = ATOM ? fixed_exponent(__uint_as_float(__ldg(fmax_bits + (BATCH ? 2 * it.sys : 0))),
                                           BATCH ? __ldg(&sd->n) : n, fixed_cap(PER))
                          : 0;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)  // (failure-path test: stage 0 gets no copy, so its wait runs out)
        for (int s = rt.skip_first ? 1 : 0; s < NST && s < it.ntile; ++s) {
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * VT * LEN, rec + ((size_t)it.v0 + (size_t)s * VT) * LEN, TILE_BYTES, &bar[s]);
        }
    float2 hxh[HP], hyh[HP], hxl[HP], hyl[HP], hz[HP], hf[HP][3 * K];
#pragma unroll
    for (int p = 0; p < HP; ++p) {
        // value m of home blob ib + 64 p in .x, of ib + 64 p + 32 in .y
        float2 hv[2 * Rec2<K>::NCH];
#pragma unroll
        for (int c = 0; c < Rec2<K>::NCH; ++c) {
            const float4 a = *reinterpret_cast<const float4*>(rec + rec2_off(ib + 64 * p, c, LEN));
            const float4 b = *reinterpret_cast<const float4*>(rec + rec2_off(ib + 64 * p + 32, c, LEN));
            hv[2 * c] = make_float2(a.x, b.x);
            hv[2 * c + 1] = make_float2(a.z, b.z);
        }
        hxh[p] = hv[0];
        hyh[p] = hv[1];
        hxl[p] = hv[2];
        hyl[p] = hv[3];
        hz[p] = hv[4];
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) hf[p][q] = hv[5 + q];
    }
    float2 acc[HP][3 * K];
#pragma unroll
    for (int p = 0; p < HP; ++p)
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) acc[p][q] = make_float2(0.0f, 0.0f);

    int t = 0;
    bool bad = false;
    for (; t < it.ntile; ++t) {
        const int s = t % NST;
        const bool ok = mbar_wait_bounded(&bar[s], (t / NST) & 1, rt.limit);
        const float* st = stage + (size_t)s * VT * LEN;
        if (ok && diag) {
            // one direction, every lane on the same source (broadcast reads)
#pragma unroll 2
            for (int jj = 0; jj < VT; ++jj) {
                float2 xh, yh, xl, yl, zj, f[3 * K];
                load_rec2<K>(st, jj, xh, yh, xl, yl, zj, f);
#pragma unroll
                for (int p = 0; p < HP; ++p) {
                    const float2 dx = add2(fma2(m1, xh, hxh[p]), fma2(m1, xl, hxl[p]));
                    const float2 dy = add2(fma2(m1, yh, hyh[p]), fma2(m1, yl, hyl[p]));
                    const float2 dz = fma2(m1, zj, hz[p]);
                    pair_apply2_images<K, false, PER, FAR>(dx, dy, dz, hz[p], zj, pc, Lx, Ly, f, hf[p], acc[p],
                                                           nullptr);
                }
            }
        } else if (ok) {
            // both directions; lane l takes visitor (step + l) mod 32
            float2 vacc[3 * K];
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) vacc[q] = make_float2(0.0f, 0.0f);
#pragma unroll UNR
            for (int step = 0; step < VT; ++step) {
                const int v = (step + lane) & (VT - 1);
                float2 xh, yh, xl, yl, zj, f[3 * K];
                load_rec2<K>(st, v, xh, yh, xl, yl, zj, f);
#pragma unroll
                for (int p = 0; p < HP; ++p) {
                    const float2 dx = add2(fma2(m1, xh, hxh[p]), fma2(m1, xl, hxl[p]));
                    const float2 dy = add2(fma2(m1, yh, hyh[p]), fma2(m1, yl, hyl[p]));
                    const float2 dz = fma2(m1, zj, hz[p]);
                    pair_apply2_images<K, true, PER, FAR>(dx, dy, dz, hz[p], zj, pc, Lx, Ly, f, hf[p], acc[p], vacc);
                }
                // hand the visitor sums to the lane that takes that visitor next
#pragma unroll
                for (int q = 0; q < 3 * K; ++q) {
                    vacc[q].x = __shfl_sync(0xffffffffu, vacc[q].x, (lane + 1) & 31);
                    vacc[q].y = __shfl_sync(0xffffffffu, vacc[q].y, (lane + 1) & 31);
                }
            }
            // lane l now holds visitor l's sums over this warp's 64 HP homes
            float* rb = red + (t & 1) * (NW * VT * 3 * K);  // double-buffered: one barrier per tile
#pragma unroll
            for (int q = 0; q < 3 * K; ++q) rb[(warp * VT + lane) * 3 * K + q] = vacc[q].x + vacc[q].y;
        }
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        if (!diag) {
            const float* rb = red + (t & 1) * (NW * VT * 3 * K);
            const int64_t sB = BATCH ? __ldg(&sd->B) : 0, sn = BATCH ? __ldg(&sd->n) : n;
            const int64_t sn_pad = BATCH ? __ldg(&sd->n_pad) : n_pad;
            float* const part = BATCH ? partial + (int64_t)3 * K * __ldg(&sd->P1) : partial;  // the system's partials
            const int64_t hloc = (int64_t)it.home - sB / HT2;  // home tile within the system
            const int64_t vbase = (int64_t)it.v0 + (int64_t)t * VT - sB;
            for (int e = tid; e < VT * 3 * K; e += NT) {
                const int vl = e / (3 * K), q = e % (3 * K);
                const int64_t vg = vbase + vl;
                if (vg < sn) {
                    float sum = rb[vl * 3 * K + q];
#pragma unroll
                    for (int w = 1; w < NW; ++w) sum += rb[(w * VT + vl) * 3 * K + q];
                    if constexpr (ATOM)  // one fixed-point accumulator per record and component
                        fixed_add(reinterpret_cast<unsigned long long*>(partial) + (int64_t)q * acc_stride + sB + vg,
                                  sum, fexp, const_cast<unsigned*>(fmax_bits) + (BATCH ? 2 * it.sys : 0) + 1);
                    else
                        part[(hloc * 3 * K + q) * sn_pad + vg] = sum;
                }
            }
        }
        if (tid == 0 && t + NST < it.ntile) {
            fence_proxy_async();
            mbar_expect_tx(&bar[s], TILE_BYTES);
            tma_load_1d(stage + (size_t)s * VT * LEN, rec + ((size_t)it.v0 + (size_t)(t + NST) * VT) * LEN, TILE_BYTES,
                        &bar[s]);
        }
    }
    if (bad) {
        if (tid == 0) {
            atomicExch(err_flag, 1);
            for (int u = t + 1; u < it.ntile && u < t + NST; ++u) mbar_wait_bounded(&bar[u % NST], (u / NST) & 1);
        }
        return;
    }
    const int64_t sB = BATCH ? __ldg(&sd->B) : 0, sn = BATCH ? __ldg(&sd->n) : n;
    const int64_t sn_pad = BATCH ? __ldg(&sd->n_pad) : n_pad;
    float* const part = BATCH ? partial + (int64_t)3 * K * __ldg(&sd->P1) : partial;
    const int slot = (BATCH ? __ldg(&sd->T) : n_home_tiles) + it.slot;
#pragma unroll
    for (int p = 0; p < HP; ++p) {
        const int64_t l0 = ib + 64 * p - sB, l1 = l0 + 32;  // the home blobs within the system
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) {
            if constexpr (ATOM) {
                unsigned long long* a64 = reinterpret_cast<unsigned long long*>(partial) + (int64_t)q * acc_stride + sB;
                unsigned* const flag = const_cast<unsigned*>(fmax_bits) + (BATCH ? 2 * it.sys : 0) + 1;
                if (l0 < sn) fixed_add(a64 + l0, acc[p][q].x, fexp, flag);
                if (l1 < sn) fixed_add(a64 + l1, acc[p][q].y, fexp, flag);
            } else {
                if (l0 < sn) part[((int64_t)slot * 3 * K + q) * sn_pad + l0] = acc[p][q].x;
                if (l1 < sn) part[((int64_t)slot * 3 * K + q) * sn_pad + l1] = acc[p][q].y;
            }
        }
    }
}

// U of a batch from its fixed-point accumulators ([3K][records], then two
// words per system: largest |force|, non-finite flag): undo the system's 2^S,
// scale and write; converged systems keep their U.  One thread per (blob,
// component blockIdx.y).
template <class Out>
__global__ void finish_fixed_batch_kernel(int n_sys, const SymSys* __restrict__ sys, int64_t n_tot, int k,
                                          int64_t acc_stride, const int* __restrict__ active,
                                          const unsigned long long* __restrict__ acc,
                                          const unsigned* __restrict__ fmax_bits, const double* __restrict__ scale,
                                          double inv8pieta, Out* __restrict__ U)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (g >= n_tot || q >= 3 * k) return;
    const int sx = sys_of(n_sys, g, [&](int m) { return sys[m].g0; });
    if (active && !active[sx]) return;
    const SymSys d = sys[sx];
    const unsigned* fb = fmax_bits + 2 * sx;
    const int S = fixed_exponent(__uint_as_float(fb[0]), d.n, fixed_cap(false));
    const double v = fb[1] ? __longlong_as_double(0x7ff8000000000000LL)
                           : ldexp((double)(long long)acc[(int64_t)q * acc_stride + d.B + (g - d.g0)], -S);
    U[(int64_t)q * n_tot + g] = (Out)(scale[g] * inv8pieta * v);
}

// Reductions of the packed kernel's partials, per system of the launch (the
// same two passes as reduce_visitors_kernel / reduce_kernel): pass 1 sums the
// visitor partials of home tiles [y SEG, (y+1) SEG) before the blob's tile;
// pass 2 adds the segments and the blob's home partials, scales and writes U.
template <int KT>
__global__ void reduce2_visitors_kernel(int n_sys, const SymSys* __restrict__ sys, int64_t n_tot, int k,
                                        const int* __restrict__ active, const float* __restrict__ partial,
                                        double* __restrict__ segsum)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    const int sx = n_sys == 1 ? 0 : sys_of(n_sys, g, [&](int m) { return sys[m].g0; });
    if (active && !active[sx]) return;
    const SymSys d = sys[sx];
    const int64_t l = g - d.g0;
    const int h = (int)(l / HT2);
    const int H0 = blockIdx.y * SEG;
    const int H1 = (H0 + SEG) < h ? (H0 + SEG) : h;
    if (H0 >= H1) return;
    const float* src = partial + (int64_t)3 * KT * d.P1 + l;
    float s[3 * KT], c[3 * KT];
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q) s[q] = c[q] = 0.0f;
    int H = H0;
    for (; H + 4 <= H1; H += 4) {
        float v[4][3 * KT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 3 * KT; ++q) v[u][q] = q < 3 * k ? src[((int64_t)(H + u) * 3 * KT + q) * d.n_pad] : 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 3 * KT; ++q) two_sum_acc(s[q], c[q], v[u][q]);
    }
    for (; H < H1; ++H)
#pragma unroll
        for (int q = 0; q < 3 * KT; ++q)
            if (q < 3 * k) two_sum_acc(s[q], c[q], src[((int64_t)H * 3 * KT + q) * d.n_pad]);
    double* dst = segsum + (int64_t)3 * KT * d.S1 + l;
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q)
        if (q < 3 * k) dst[((int64_t)blockIdx.y * 3 * KT + q) * d.n_pad] = two_sum_value(s[q], c[q]);
}

template <class Out>
__global__ void reduce2_kernel(int n_sys, const SymSys* __restrict__ sys, int64_t n_tot, int k, int kt,
                               const int* __restrict__ active, const float* __restrict__ partial,
                               const double* __restrict__ segsum, const double* __restrict__ scale, double inv8pieta,
                               Out* __restrict__ U)
{
    // one thread per (blob, component q = blockIdx.y < 3k)
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (g >= n_tot || q >= 3 * k) return;
    const int sx = n_sys == 1 ? 0 : sys_of(n_sys, g, [&](int m) { return sys[m].g0; });
    if (active && !active[sx]) return;
    const SymSys d = sys[sx];
    const int64_t l = g - d.g0;
    const int h = (int)(l / HT2);
    const int nseg = (h + SEG - 1) / SEG;
    const int64_t vis = d.n_pad - (int64_t)(h + 1) * HT2;  // visitors of tile h
    const int home_slots = 1 + (int)((vis + d.chunk - 1) / d.chunk);
    const double* sg = segsum + (int64_t)3 * kt * d.S1 + l;
    const float* pt = partial + (int64_t)3 * kt * d.P1 + l;
    double sum = 0.0;
    for (int y = 0; y < nseg; ++y) sum += sg[((int64_t)y * 3 * kt + q) * d.n_pad];
    float hs = 0.0f, hc = 0.0f;
    for (int c = 0; c < home_slots; ++c) two_sum_acc(hs, hc, pt[((int64_t)(d.T + c) * 3 * kt + q) * d.n_pad]);
    sum += two_sum_value(hs, hc);
    U[(int64_t)q * n_tot + g] = (Out)(scale[g] * inv8pieta * sum);
}

}  // namespace sym

// Work list of the packed symmetric kernel for one launch (one system, or a
// batch of systems given by blob offsets), cached per offsets.
struct Sym2Plan {
    std::vector<int64_t> off;
    std::vector<sym::SymSys> sys;
    sym::SymItem* d_items = nullptr;
    sym::SymSys* d_sys = nullptr;
    int n_items = 0;
    int max_nseg = 1;
    int64_t rec_end = 0;    // records of the launch
    int64_t part_rows = 0;  // sum over systems of (T + slots) n_pad: partial floats / (3K)
    int64_t seg_rows = 0;   // sum over systems of nseg n_pad: segment doubles / (3K)
};

void free_sym2_plans(rpbd_handle* h)
{
    for (Sym2Plan* p : h->sym2_plans) {
        cudaFree(p->d_items);
        cudaFree(p->d_sys);
        delete p;
    }
    h->sym2_plans.clear();
}

namespace sym {

static int get_plan2(rpbd_handle* h, int n_sys, const int64_t* off, Sym2Plan** out)
{
    for (Sym2Plan* p : h->sym2_plans)
        if ((int)p->off.size() == n_sys + 1 && std::equal(p->off.begin(), p->off.end(), off)) {
            *out = p;
            return RPBD_OK;
        }
    Sym2Plan* p = new Sym2Plan();
    p->off.assign(off, off + n_sys + 1);
    // chunk: halved (down to one visitor tile) while the launch would have
    // fewer than 4 items per SM
    auto count = [&](int c) {
        int64_t m = 0;
        for (int s = 0; s < n_sys; ++s) {
            const int64_t np_ = (off[s + 1] - off[s] + HT2 - 1) / HT2 * HT2;
            for (int64_t H = 0; H < np_ / HT2; ++H) m += 1 + (np_ - (H + 1) * HT2 + c - 1) / c;
        }
        return m;
    };
    int chunk = CHUNK;
    while (chunk > VT && count(chunk) < 4 * (int64_t)h->sm_count) chunk /= 2;
    std::vector<SymItem> items;
    int64_t B = 0, P1 = 0, S1 = 0;
    for (int s = 0; s < n_sys; ++s) {
        SymSys d;
        d.n = off[s + 1] - off[s];
        d.g0 = off[s];
        d.n_pad = (d.n + HT2 - 1) / HT2 * HT2;
        d.B = B;
        d.T = (int)(d.n_pad / HT2);
        d.chunk = chunk;
        d.P1 = P1;
        d.S1 = S1;
        const int slots = d.T > 0 ? 1 + (int)((d.n_pad - HT2 + chunk - 1) / chunk) : 0;
        const int nseg = (d.T + SEG - 1) / SEG;
        for (int H = 0; H < d.T; ++H) {
            const int home = (int)(B / HT2) + H;
            items.push_back(SymItem{home, (int)(B + (int64_t)H * HT2), HT2 / VT, 0, s});
            int c = 1;
            for (int64_t v0 = (int64_t)(H + 1) * HT2; v0 < d.n_pad; v0 += chunk, ++c) {
                const int64_t v1 = std::min<int64_t>(d.n_pad, v0 + chunk);
                items.push_back(SymItem{home, (int)(B + v0), (int)((v1 - v0) / VT), c, s});
            }
        }
        p->max_nseg = std::max(p->max_nseg, nseg);
        B += d.n_pad;
        P1 += (int64_t)(d.T + slots) * d.n_pad;
        S1 += (int64_t)nseg * d.n_pad;
        p->sys.push_back(d);
    }
    // longest items first so the hardware scheduler fills the tail with short ones
    std::stable_sort(items.begin(), items.end(), [](const SymItem& a, const SymItem& b) { return a.ntile > b.ntile; });
    p->n_items = (int)items.size();
    p->rec_end = B;
    p->part_rows = P1;
    p->seg_rows = S1;
    if (B > ((int64_t)1 << 31) - HT2 || cudaMalloc(&p->d_items, sizeof(SymItem) * std::max<size_t>(1, items.size())) !=
                                            cudaSuccess ||
        cudaMalloc(&p->d_sys, sizeof(SymSys) * n_sys) != cudaSuccess ||
        (!items.empty() &&
         cudaMemcpy(p->d_items, items.data(), sizeof(SymItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(p->d_sys, p->sys.data(), sizeof(SymSys) * n_sys, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p->d_items);
        cudaFree(p->d_sys);
        delete p;
        return set_error(h, RPBD_NO_MEM, "packed symmetric kernel: work list upload failed");
    }
    h->sym2_plans.push_back(p);
    *out = p;
    return RPBD_OK;
}

// the packed symmetric matvec of one system (n_sys = 1) or a batch; PER: the
// pseudo-periodic cell (single systems only)
template <int K, bool PER, class In, class Out>
static int run2(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const In* F, Out* U, int k,
                const int* active, Buf b_rec, Buf b_scale, Buf b_part, Buf b_seg, cudaStream_t st)
{
    constexpr int LEN = Rec2<K>::LEN;
    const int64_t n_tot = off[n_sys];
    if (n_tot <= 0) return RPBD_OK;
    Sym2Plan* pl = nullptr;
    RPBD_TRY(get_plan2(h, n_sys, off, &pl));
    float* rec;
    double* scale;
    float* partial;
    double* segsum = nullptr;
    // fixed-point accumulation, one integer per record and component (memory
    // O(n), deterministic); per-home-tile partials with the fixed-order
    // reduction on request (RPBD_OPT_SYM_PARTIALS; a single system only while
    // they stay under SYM_PARTIAL_LIMIT bytes and the far field is off)
    const bool atom = !h->sym_partials ||
                      (n_sys == 1 && (h->far_field ||
                                      (double)pl->part_rows * 3 * K * sizeof(float) > SYM_PARTIAL_LIMIT));
    const int64_t acc_stride = pl->rec_end;
    unsigned* fmax_bits = nullptr;
    RPBD_TRY(ensure_t(h, b_rec, (size_t)pl->rec_end * LEN, &rec));
    RPBD_TRY(ensure_t(h, b_scale, (size_t)n_tot, &scale));
    if (atom) {
        // [3K][records] accumulators, then two words per system (largest |force|, non-finite flag)
        unsigned long long* acc;
        const size_t words = (size_t)3 * K * acc_stride + (size_t)n_sys;
        RPBD_TRY(ensure_t(h, b_part, words, &acc));
        RPBD_CU(h, cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * words, st));
        partial = reinterpret_cast<float*>(acc);
        fmax_bits = reinterpret_cast<unsigned*>(acc + 3 * K * acc_stride);
    } else {
        RPBD_TRY(ensure_t(h, b_part, (size_t)pl->part_rows * 3 * K, &partial));
        RPBD_TRY(ensure_t(h, b_seg, (size_t)std::max<int64_t>(1, pl->seg_rows) * 3 * K, &segsum));
    }
    pack2_kernel<K, In><<<(unsigned)((pl->rec_end + 255) / 256), 256, 0, st>>>(
        n_sys, pl->d_sys, pl->rec_end, n_tot, k, r, F, h->p.a, h->p.wall, h->p.s_min, active, rec, scale, fmax_bits);
    count_launch();
    const float Lxa = (float)(h->p.Lx / h->p.a), Lya = (float)(h->p.Ly / h->p.a);  // periodic cell in units of a
    if (h->profile) prof_begin(h, st);
    const int sv = h->sym_variant[sym_class(K)];
    const SymItem* items = pl->d_items;
    const SymSys* sys = pl->d_sys;
    const int ni = pl->n_items;
    const int64_t n1 = pl->sys[0].n, np1 = pl->sys[0].n_pad;
    const int T1 = pl->sys[0].T;
    const RingTest rt = ring_test(h);
    // tuning variants, see Sym2Var; -1: the autotuner's usual pick at 65,535 blobs (k = 1: variant 3,
    // k = 2: variant 5, k = 3..4: variant 4)
    const int var = sv >= 0 ? sv : (K == 1 ? 3 : (K == 2 ? 5 : 4));
#define RPBD_SYM2_LAUNCH(V, FARV, ATOMV)                                                                          \
    sym2_kernel<K, PER, Sym2Var<K, V, PER>::UNR, Sym2Var<K, V, PER>::MINB, false, Sym2Var<K, V, PER>::HP, FARV, ATOMV> \
        <<<ni, Sym2Var<K, V, PER>::NT, Sym2Var<K, V, PER>::smem(LEN), st>>>(rec, items, n1, np1, T1, sys, nullptr,     \
                                                                            Lxa, Lya, partial, h->dev_flag, rt,        \
                                                                            fmax_bits, acc_stride)
    if (n_sys > 1) {  // batches: four home blobs per thread (variant 5's shape; 3-5% faster than two
                      // on 64 uneven suspensions of 480-22,500 blobs)
        if constexpr (!PER) {
            using V5 = Sym2Var<K, 5>;
            if (atom)
                sym2_kernel<K, false, V5::UNR, V5::MINB, true, V5::HP, false, true><<<ni, V5::NT, V5::smem(LEN), st>>>(
                    rec, items, 0, 0, 0, sys, active, Lxa, Lya, partial, h->dev_flag, rt, fmax_bits, acc_stride);
            else
                sym2_kernel<K, false, V5::UNR, V5::MINB, true, V5::HP><<<ni, V5::NT, V5::smem(LEN), st>>>(
                    rec, items, 0, 0, 0, sys, active, Lxa, Lya, partial, h->dev_flag, rt);
        } else
            return set_error(h, RPBD_BAD_ARG, "packed symmetric kernel: batches are open in x, y");
    } else if (h->far_field) {  // the cancellation-free block: one compiled variant per k
        RPBD_SYM2_LAUNCH(K == 1 ? 3 : (K == 2 || !PER ? 5 : 3), true, true);  // (k > 2 periodic: no spill)
    } else if (!atom) {  // per-home-tile partials and the fixed-order reduction: the default variant
        RPBD_SYM2_LAUNCH(K == 1 ? 3 : (K == 2 ? 5 : 4), false, false);
    } else {
        switch (var) {
        case 1: RPBD_SYM2_LAUNCH(1, false, true); break;
        case 2: RPBD_SYM2_LAUNCH(2, false, true); break;
        case 3: RPBD_SYM2_LAUNCH(3, false, true); break;
        case 4: RPBD_SYM2_LAUNCH(4, false, true); break;
        case 5: RPBD_SYM2_LAUNCH(5, false, true); break;
        default: RPBD_SYM2_LAUNCH(0, false, true); break;
        }
    }
#undef RPBD_SYM2_LAUNCH
    count_launch();
    if (h->profile) {
        double pairs = 0.0;
        for (int s = 0; s < n_sys; ++s) pairs += (double)(off[s + 1] - off[s]) * (double)(off[s + 1] - off[s]);
        prof_end(h, st, n_sys > 1 ? 2 /* batched */ : (PER ? 3 : 4) /* symmetric (images) or factored */, K, pairs);
    }
    // blocks were formed in units of a: M = M(a = 1) / a
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta * h->p.a);
    if (atom) {
        const dim3 fgrid((unsigned)((n_tot + 255) / 256), (unsigned)(3 * k));
        const auto* acc = reinterpret_cast<const unsigned long long*>(partial);
        if (n_sys == 1)
            finish_fixed_kernel<Out><<<fgrid, 256, 0, st>>>(n_tot, acc_stride, k, sym::fixed_cap(PER), acc, fmax_bits,
                                                            scale, inv8pieta, U);
        else
            finish_fixed_batch_kernel<Out><<<fgrid, 256, 0, st>>>(n_sys, sys, n_tot, k, acc_stride, active, acc,
                                                                  fmax_bits, scale, inv8pieta, U);
        count_launch();
        RPBD_LAUNCH_CHECK(h);
        return RPBD_OK;
    }
    reduce2_visitors_kernel<K><<<dim3((unsigned)((n_tot + 255) / 256), (unsigned)pl->max_nseg), 256, 0, st>>>(
        n_sys, sys, n_tot, k, active, partial, segsum);
    count_launch();
    reduce2_kernel<Out><<<dim3((unsigned)((n_tot + 255) / 256), (unsigned)(3 * k)), 256, 0, st>>>(
        n_sys, sys, n_tot, k, K, active, partial, segsum, scale, inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

template <int K, bool PER, class In, class Out>
static int run2(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    const int64_t off[2] = {0, n};
    return run2<K, PER>(h, 1, off, r, F, U, k, nullptr, BUF_PACK, BUF_SCALE, BUF_PARTIAL, BUF_SYM_SEG, st);
}

}  // namespace sym

template <int K, class In, class Out>
static int sym_k(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    if (h->use_packed && h->p.wall)
        return h->p.Lx > 0.0 ? sym::run2<K, true>(h, n, r, F, U, k, st) : sym::run2<K, false>(h, n, r, F, U, k, st);
    if (h->p.Lx > 0.0) return sym::run<K, true, true>(h, n, r, F, U, k, st);
    return h->p.wall ? sym::run<K, true, false>(h, n, r, F, U, k, st) : sym::run<K, false, false>(h, n, r, F, U, k, st);
}

template <class In, class Out>
static int sym_dispatch(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    if (k <= 1) return sym_k<1>(h, n, r, F, U, k, st);
    if (k <= 2) return sym_k<2>(h, n, r, F, U, k, st);
    return sym_k<4>(h, n, r, F, U, k, st);
}

int sym_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k, bool io_double,
                   cudaStream_t st)
{
    if (io_double) return sym_dispatch(h, n, r, (const double*)F, (double*)U, k, st);
    return sym_dispatch(h, n, r, (const float*)F, (float*)U, k, st);
}

template <class In, class Out>
static int sym_batched_dispatch(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const In* F, Out* U,
                                int k, const int* active, cudaStream_t st)
{
    if (k <= 1) return sym::run2<1, false>(h, n_sys, off, r, F, U, k, active, BUF_BPACK, BUF_BSCALE, BUF_BPARTIAL, BUF_BSEG, st);
    if (k <= 2) return sym::run2<2, false>(h, n_sys, off, r, F, U, k, active, BUF_BPACK, BUF_BSCALE, BUF_BPARTIAL, BUF_BSEG, st);
    return sym::run2<4, false>(h, n_sys, off, r, F, U, k, active, BUF_BPACK, BUF_BSCALE, BUF_BPARTIAL, BUF_BSEG, st);
}

int sym_batched_apply_impl(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const void* F, void* U,
                           int k, bool io_double, const int* active, cudaStream_t st)
{
    if (!h->p.wall || h->p.Lx > 0.0 || k < 1 || k > 4)
        return set_error(h, RPBD_BAD_ARG, "batched symmetric variant: wall, open cell, 1 <= k <= 4");
    if (io_double) return sym_batched_dispatch(h, n_sys, off, r, (const double*)F, (double*)U, k, active, st);
    return sym_batched_dispatch(h, n_sys, off, r, (const float*)F, (float*)U, k, active, st);
}

}  // namespace rpbd
