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
// A reduce kernel adds, for blob i, the visitor partials of every home tile
// before i's tile and the home partials of i's own tile in a fixed order
// (FP64, deterministic), then applies s_i / (8 pi eta).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "rpbd_internal.cuh"
#include "wall_rpy.cuh"

namespace rpbd {
namespace sym {

constexpr int HT = 128;    // home tile (threads per CTA)
constexpr int VT = 32;     // visitor tile (records per stage)
constexpr int NST = 4;     // TMA ring depth
constexpr int CHUNK = 2048;  // visitors per off-diagonal item

template <int K>
struct Rec {
    static constexpr int TAIL = ((1 + 3 * K) + 3) / 4 * 4;
    static constexpr int LEN = 4 + TAIL;
};

// tuning variants per K: visitor-loop unroll and minimum resident CTAs per SM
// (the latter caps registers: 65536 / (MINB * 128)); chosen so no variant spills
template <int K, int V>
struct SymVar {
    static constexpr int UNR = V == 1 ? 1 : (V == 3 ? 4 : 2);
    static constexpr int MINB = K == 1 ? (V == 2 ? 9 : 8) : (K == 2 ? (V == 2 ? 8 : 7) : (V == 2 ? 5 : 4));
};

struct SymItem {
    int home;   // home tile index
    int v0;     // first visitor blob (multiple of VT)
    int ntile;  // visitor tiles
    int slot;   // home-partial slot (0: diagonal item)
};

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
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 4000000000LL) return false;
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
                                                 float* __restrict__ partial, int* __restrict__ err_flag)
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
    if (tid == 0)
        for (int s = 0; s < NST && s < it.ntile; ++s) {
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
        const bool ok = mbar_wait_bounded(&bar[s], (t / NST) & 1);
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
#pragma unroll
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
// Both passes use a fixed order (deterministic).
constexpr int SEG = 64;  // home tiles per segment

template <int KT, class P>
__global__ void reduce_visitors_kernel(int64_t n, int64_t n_pad, int k, const P* __restrict__ partial,
                                       double* __restrict__ segsum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int h = (int)(i / HT);
    const int H0 = blockIdx.y * SEG;
    const int H1 = (H0 + SEG) < h ? (H0 + SEG) : h;
    if (H0 >= H1) return;
    double acc[3 * KT];
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q) acc[q] = 0.0;
    for (int H = H0; H < H1; ++H)
#pragma unroll
        for (int q = 0; q < 3 * KT; ++q)
            if (q < 3 * k) acc[q] += (double)partial[((int64_t)H * 3 * KT + q) * n_pad + i];
#pragma unroll
    for (int q = 0; q < 3 * KT; ++q)
        if (q < 3 * k) segsum[((int64_t)blockIdx.y * 3 * KT + q) * n_pad + i] = acc[q];
}

// U_i = s_i/(8 pi eta) [sum_{segments before tile(i)} + sum_c home partial(c)]
template <class P, class Out>
__global__ void reduce_kernel(int64_t n, int64_t n_pad, int k, int kt, int n_home_tiles, int chunk,
                              const P* __restrict__ partial, const double* __restrict__ segsum,
                              const double* __restrict__ scale, double inv8pieta, Out* __restrict__ U)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int h = (int)(i / HT);
    const int nseg = (h + SEG - 1) / SEG;
    const int64_t vis = n_pad - (int64_t)(h + 1) * HT;  // visitors of tile h
    const int home_slots = 1 + (int)((vis + chunk - 1) / chunk);
    const double sc = scale[i] * inv8pieta;
    for (int q = 0; q < 3 * k; ++q) {
        double sum = 0.0;
        for (int sg = 0; sg < nseg; ++sg) sum += segsum[((int64_t)sg * 3 * kt + q) * n_pad + i];
        for (int c = 0; c < home_slots; ++c)
            sum += (double)partial[((int64_t)(n_home_tiles + c) * 3 * kt + q) * n_pad + i];
        U[(int64_t)q * n + i] = (Out)(sc * sum);
    }
}

static int get_items(rpbd_handle* h, int64_t n, int64_t n_pad, SymItem** d_items, int* n_items, int* n_home,
                     int* max_slots)
{
    if (h->sym_plan_n != n) {
        std::vector<SymItem> items;
        const int T = (int)(n_pad / HT);
        int ms = 1;
        for (int H = 0; H < T; ++H) {
            items.push_back(SymItem{H, H * HT, HT / VT, 0});
            int c = 1;
            for (int64_t v0 = (int64_t)(H + 1) * HT; v0 < n_pad; v0 += CHUNK, ++c) {
                const int64_t v1 = std::min<int64_t>(n_pad, v0 + CHUNK);
                items.push_back(SymItem{H, (int)v0, (int)((v1 - v0) / VT), c});
            }
            ms = std::max(ms, c);
        }
        // longest items first so the hardware scheduler fills the tail with short ones
        std::stable_sort(items.begin(), items.end(), [](const SymItem& a, const SymItem& b) { return a.ntile > b.ntile; });
        void* d = nullptr;
        RPBD_TRY(ensure(h, BUF_SYM_ITEMS, items.size() * sizeof(SymItem), &d));
        RPBD_CU(h, cudaMemcpy(d, items.data(), items.size() * sizeof(SymItem), cudaMemcpyHostToDevice));
        h->sym_plan_n = n;
        h->sym_n_items = (int)items.size();
        h->sym_n_home = T;
        h->sym_max_slots = ms;
    }
    *d_items = reinterpret_cast<SymItem*>(h->buf[BUF_SYM_ITEMS]);
    *n_items = h->sym_n_items;
    *n_home = h->sym_n_home;
    *max_slots = h->sym_max_slots;
    return RPBD_OK;
}

template <int K, bool WALL, bool PER, class In, class Out>
static int run(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
    constexpr int LEN = Rec<K>::LEN;
    const int64_t n_pad = (n + HT - 1) / HT * HT;
    SymItem* items;
    int n_items, n_home, max_slots;
    RPBD_TRY(get_items(h, n, n_pad, &items, &n_items, &n_home, &max_slots));
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
    // variant -1: the measured default per K (k = 1: unroll 4; otherwise unroll 2)
    const int sv = h->sym_variant[sym_class(K)];
    const int var = sv >= 0 ? sv : (K == 1 ? 3 : 0);
    switch (var) {  // tuning variants: (visitor-loop unroll, min CTAs per SM), see SymVar
    case 1: sym_kernel<K, WALL, PER, SymVar<K, 1>::UNR, SymVar<K, 1>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag); break;
    case 2: sym_kernel<K, WALL, PER, SymVar<K, 2>::UNR, SymVar<K, 2>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag); break;
    case 3: sym_kernel<K, WALL, PER, SymVar<K, 3>::UNR, SymVar<K, 3>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag); break;
    default: sym_kernel<K, WALL, PER, SymVar<K, 0>::UNR, SymVar<K, 0>::MINB><<<n_items, HT, smem, st>>>(rec, n, n_pad, items, n_home, pc, partial, h->dev_flag); break;
    }
    count_launch();
    if (h->profile) prof_end(h, st, (K <= 2 && !PER) ? 4 /* symmetric, factored */ : 3 /* symmetric */, K,
                             (double)n * (double)n);
    const double inv8pieta = 1.0 / (8.0 * 3.14159265358979323846 * h->p.eta);
    const int nseg = (n_home + SEG - 1) / SEG;
    double* segsum;
    RPBD_TRY(ensure_t(h, BUF_SYM_SEG, (size_t)nseg * 3 * K * n_pad, &segsum));
    reduce_visitors_kernel<K, float><<<dim3((unsigned)((n + 255) / 256), (unsigned)nseg), 256, 0, st>>>(
        n, n_pad, k, partial, segsum);
    count_launch();
    reduce_kernel<float, Out><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, n_pad, k, K, n_home, CHUNK, partial,
                                                                           segsum, scale, inv8pieta, U);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

}  // namespace sym

template <int K, class In, class Out>
static int sym_k(rpbd_handle* h, int64_t n, const double* r, const In* F, Out* U, int k, cudaStream_t st)
{
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

}  // namespace rpbd
