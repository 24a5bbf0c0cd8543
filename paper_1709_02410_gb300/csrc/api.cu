// C ABI entry points: argument checks, workspace, dispatch.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <set>
#include <utility>

#include "rpbd_internal.cuh"

namespace rpbd {

static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t pool_event(rpbd_handle* h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(rpbd_handle* h, cudaStream_t st)
{
    ProfRec r{pool_event(h), pool_event(h), 0, 0, 0.0};
    cudaEventRecord(r.a, st);
    h->prof.push_back(r);
}

void prof_end(rpbd_handle* h, cudaStream_t st, int dtype, int k, double pairs)
{
    ProfRec& r = h->prof.back();
    cudaEventRecord(r.b, st);
    r.dtype = dtype;
    r.k = k;
    r.pairs = pairs;
}

int set_error(rpbd_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    return code;
}

bool once_per_device(rpbd_handle* h, const void* key)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> seen;
    std::lock_guard<std::mutex> lock(mu);
    return seen.insert(std::make_pair(h->device, key)).second;
}

int ensure(rpbd_handle* h, Buf b, size_t bytes, void** out)
{
    if (bytes == 0) bytes = 16;
    if (h->cap[b] < bytes) {
        if (h->buf[b]) {
            cudaError_t e = cudaFree(h->buf[b]);
            h->buf[b] = nullptr;
            h->cap[b] = 0;
            if (e != cudaSuccess) return set_error(h, RPBD_CUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
        }
        size_t want = bytes + bytes / 8;  // headroom for slowly growing sizes
        cudaError_t e = cudaMalloc(&h->buf[b], want);
        if (e != cudaSuccess) {
            h->buf[b] = nullptr;
            return set_error(h, RPBD_NO_MEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        h->cap[b] = want;
    }
    *out = h->buf[b];
    return RPBD_OK;
}

}  // namespace rpbd

using namespace rpbd;

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char* rpbd_status_string(int status)
{
    switch (status) {
    case RPBD_OK: return "ok";
    case RPBD_BAD_ARG: return "bad argument";
    case RPBD_BAD_INPUT: return "bad input (non-finite values)";
    case RPBD_CUDA: return "CUDA error";
    case RPBD_NOT_CONVERGED: return "iteration did not converge";
    case RPBD_TIMEOUT: return "device wait timed out";
    case RPBD_NO_MEM: return "out of device memory";
    case RPBD_TOO_LARGE: return "size beyond the allocation-free matvec's fixed scratch (n <= 16384, k <= 16)";
    default: return "unknown status";
    }
}

const char* rpbd_last_error(const rpbd_handle* h) { return h ? h->err.c_str() : "null handle"; }

int rpbd_create(rpbd_handle** out, const rpbd_params* p)
{
    if (!out || !p) return RPBD_BAD_ARG;
    *out = nullptr;
    if (!(p->eta > 0) || !(p->a > 0) || !(p->kT >= 0) || !(p->s_min > 0) || p->s_min > 1) return RPBD_BAD_ARG;
    if (!(p->Lx >= 0) || !(p->Ly >= 0) || ((p->Lx > 0) != (p->Ly > 0)) || (p->Lx > 0 && !p->wall)) return RPBD_BAD_ARG;
    rpbd_handle* h = new (std::nothrow) rpbd_handle();
    if (!h) return RPBD_NO_MEM;
    h->p = *p;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return RPBD_CUDA;
    }
    if (cudaMalloc(&h->dev_flag, sizeof(int)) != cudaSuccess || cudaMemset(h->dev_flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->host_small, 4096 * sizeof(double)) != cudaSuccess) {
        if (h->dev_flag) cudaFree(h->dev_flag);
        delete h;
        return RPBD_CUDA;
    }
    *out = h;
    return RPBD_OK;
}

int rpbd_destroy(rpbd_handle* h)
{
    if (!h) return RPBD_OK;
    for (auto& r : h->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    batched_free_graphs(h);
    batched_free_plans(h);
    for (int b = 0; b < BUF_COUNT; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    if (h->dev_flag) cudaFree(h->dev_flag);
    if (h->host_small) cudaFreeHost(h->host_small);
    delete h;
    return RPBD_OK;
}

int rpbd_reserve(rpbd_handle* h, int64_t n, int64_t nb, int nper, int k, int basis)
{
    if (!h || n < 0 || nb < 0 || k < 0 || basis < 0) return RPBD_BAD_ARG;
    void* p;
    const int64_t n_pad = (n + 255) / 256 * 256;
    const int kk = k < 1 ? 1 : k;
    RPBD_TRY(ensure(h, BUF_PACK, (size_t)n_pad * (8 + 3 * kk + 4) * sizeof(double), &p));
    RPBD_TRY(ensure(h, BUF_SCALE, (size_t)n_pad * sizeof(double), &p));
    if (basis > 0) {
        const int64_t len = 3 * n + 6 * nb;
        RPBD_TRY(ensure(h, BUF_KRYLOV, (size_t)(basis + 1) * len * sizeof(double), &p));
    }
    (void)nper;
    return RPBD_OK;
}

long long rpbd_launch_count(void) { return g_launches.load(); }

}  // extern "C"

namespace rpbd {
// FMA-throughput probe: every thread runs 8 independent FMA chains of
// 16 * iters links each; the result is stored only under a condition the
// chains never meet, so the work cannot be dropped.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T a, T b, T* __restrict__ sink)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == T(-1)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the same chains with packed two-wide FP32 FMAs (one instruction, two FMAs)
__global__ void __launch_bounds__(256) fma2_peak_kernel(int iters, float a, float b, float* __restrict__ sink)
{
    float2 x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] = make_float2((threadIdx.x + 2 * c) * 1e-3f, (threadIdx.x + 2 * c + 1) * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += x[c].x + x[c].y;
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed FMAs whose three operands are all distinct, varying registers (no
// immediate, no loop-invariant or repeated operand): a twelve-value tangle
// where every step reads three different pairs, 8 packed FMAs (16 FMAs) per
// unrolled step.  The register file supplies such an instruction more
// slowly than one with a constant operand, which bounds kernels made of them.
__global__ void __launch_bounds__(256) fma2_varying_kernel(int iters, float a, float b, float* __restrict__ sink)
{
    float2 v[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = make_float2((threadIdx.x + c) * 1e-3f * a, c * b + 1.0f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = __ffma2_rn(v[c + 4], v[(c + 3) % 12], v[c]);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 12; ++c) s += v[c].x + v[c].y;
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, bool PACKED = false, bool VARYING = false>
static int measure_peak(rpbd_handle* h, int iters, double* tflops, cudaStream_t st)
{
    int dev = 0, sms = 0;
    RPBD_CU(h, cudaGetDevice(&dev));
    RPBD_CU(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)sms * 8;
    T* sink;
    RPBD_TRY(ensure_t(h, BUF_AUX, (size_t)grid * 256, &sink));
    cudaEvent_t e0, e1;
    RPBD_CU(h, cudaEventCreate(&e0));
    RPBD_CU(h, cudaEventCreate(&e1));
    for (int rep = 0; rep < 2; ++rep) {  // warm-up, then the timed launch
        if (rep == 1) RPBD_CU(h, cudaEventRecord(e0, st));
        const int it = rep == 0 ? iters / 8 + 1 : iters;
        if (VARYING) fma2_varying_kernel<<<grid, 256, 0, st>>>(it, 0.9999999f, 1e-7f, reinterpret_cast<float*>(sink));
        else if (PACKED) fma2_peak_kernel<<<grid, 256, 0, st>>>(it, 0.9999999f, 1e-7f, reinterpret_cast<float*>(sink));
        else fma_peak_kernel<T><<<grid, 256, 0, st>>>(it, T(0.9999999), T(1e-7), sink);
        count_launch();
    }
    RPBD_CU(h, cudaEventRecord(e1, st));
    RPBD_CU(h, cudaEventSynchronize(e1));
    float ms = 0.0f;
    RPBD_CU(h, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // FMAs per unrolled step of one thread: 8 chains (scalar), 4 packed pairs, or 8 packed
    // pairs in the varying-operand form
    const double fmas = VARYING ? 16.0 : 8.0;
    const double flops = 2.0 * fmas * 16 * (double)iters * grid * 256;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return RPBD_OK;
}
}  // namespace rpbd

extern "C" {

int rpbd_measure_fma_peak(rpbd_handle* h, int dtype, double* tflops, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (!tflops) return set_error(h, RPBD_BAD_ARG, "measure_fma_peak: null output");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (dtype == RPBD_F32) return measure_peak<float>(h, 4096, tflops, st);
    if (dtype == 2) return measure_peak<float, true>(h, 4096, tflops, st);  // packed two-wide FP32
    if (dtype == 3) return measure_peak<float, true, true>(h, 4096, tflops, st);  // packed, three varying operands
    if (dtype == RPBD_F64) return measure_peak<double>(h, 64, tflops, st);
    return set_error(h, RPBD_BAD_ARG, "measure_fma_peak: bad dtype");
}

int rpbd_set_option(rpbd_handle* h, int option, int value)
{
    if (!h) return RPBD_BAD_ARG;
    switch (option) {
    case RPBD_OPT_SYMMETRIC:
        for (int c = 0; c < 3; ++c) h->use_sym[c] = value != 0;
        return RPBD_OK;
    case RPBD_OPT_PACKED: h->use_packed = value != 0; return RPBD_OK;
    case RPBD_OPT_BATCH_VARIANT:
        if (value < -1 || value > 4) return set_error(h, RPBD_BAD_ARG, "batched variant must be -1..4");
        if (value >= 3 && !h->p.wall) return set_error(h, RPBD_BAD_ARG, "the packed batched variants need the wall");
        h->batch_variant = value;
        return RPBD_OK;
    case RPBD_OPT_SYM_VARIANT:
        if (value < -1 || value > 5) return set_error(h, RPBD_BAD_ARG, "symmetric variant must be -1..5");
        for (int c = 0; c < 3; ++c) h->sym_variant[c] = value;
        return RPBD_OK;
    case RPBD_OPT_TEST_STALL: h->test_stall = value != 0; return RPBD_OK;
    case RPBD_OPT_FARFIELD: h->far_field = value != 0; return RPBD_OK;
    case RPBD_OPT_SYM_PARTIALS: h->sym_partials = value != 0; return RPBD_OK;
    default: return set_error(h, RPBD_BAD_ARG, "unknown option");
    }
}

int rpbd_profile_enable(rpbd_handle* h, int on)
{
    if (!h) return RPBD_BAD_ARG;
    h->profile = on != 0;
    return RPBD_OK;
}

int rpbd_profile_read(rpbd_handle* h, int dtype, int k, double* ms, long long* launches, double* pairs, int reset)
{
    if (!h || !ms || !launches || !pairs) return RPBD_BAD_ARG;
    *ms = 0.0;
    *launches = 0;
    *pairs = 0.0;
    RPBD_CU(h, cudaDeviceSynchronize());
    std::vector<ProfRec> keep;
    for (auto& r : h->prof) {
        if (r.dtype == dtype && r.k == k) {
            float t = 0.0f;
            RPBD_CU(h, cudaEventElapsedTime(&t, r.a, r.b));
            *ms += t;
            *launches += 1;
            *pairs += r.pairs;
        }
        if (reset) {
            h->ev_pool.push_back(r.a);
            h->ev_pool.push_back(r.b);
        } else {
            keep.push_back(r);
        }
    }
    h->prof.swap(keep);
    return RPBD_OK;
}

int rpbd_autotune(rpbd_handle* h, int64_t n, const double* r, int k, double* best_ms, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n <= 0 || !r || k < 1 || k > 16) return set_error(h, RPBD_BAD_ARG, "autotune: bad arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float* F;
    RPBD_TRY(ensure_t(h, BUF_AUX, (size_t)2 * k * 3 * n, &F));
    float* U = F + (size_t)k * 3 * n;
    RPBD_CU(h, cudaMemsetAsync(F, 0, sizeof(float) * k * 3 * n, st));
    cudaEvent_t e0, e1;
    RPBD_CU(h, cudaEventCreate(&e0));
    RPBD_CU(h, cudaEventCreate(&e1));
    // candidates: one-direction kernel (-1) and, for k <= 4, the symmetric variants (0..5 of the
    // packed kernel with the wall, 0..3 of the one-home kernel otherwise)
    const int nsym = (h->use_packed && h->p.wall) ? 6 : 4;
    const int ncand = k <= 4 ? 1 + nsym : 1;
    double best = 1e300;
    int best_c = -1;
    const bool prof = h->profile;
    h->profile = false;
    const int cls = sym_class(k);
    for (int c = -1; c < ncand - 1; ++c) {
        h->use_sym[cls] = c >= 0;
        if (c >= 0) h->sym_variant[cls] = c;
        int s = mobility_apply_impl(h, n, r, F, U, k, RPBD_F32, false, st);
        if (s != RPBD_OK) { h->profile = prof; return s; }
        RPBD_CU(h, cudaEventRecord(e0, st));
        for (int rep = 0; rep < 2; ++rep) RPBD_TRY(mobility_apply_impl(h, n, r, F, U, k, RPBD_F32, false, st));
        RPBD_CU(h, cudaEventRecord(e1, st));
        RPBD_CU(h, cudaEventSynchronize(e1));
        float ms = 0.0f;
        RPBD_CU(h, cudaEventElapsedTime(&ms, e0, e1));
        if (ms / 2.0 < best) {
            best = ms / 2.0;
            best_c = c;
        }
    }
    h->profile = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->use_sym[cls] = best_c >= 0;
    h->sym_variant[cls] = best_c >= 0 ? best_c : -1;
    if (best_ms) *best_ms = best;
    return best_c + 1;
}

int rpbd_blobs_from_bodies(rpbd_handle* h, int64_t nb, int nper, const double* shape, const double* q,
                           const double* theta, double* r, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (nb < 0 || nper <= 0 || !shape || !q || !theta || !r)
        return set_error(h, RPBD_BAD_ARG, "blobs_from_bodies: bad arguments");
    launch_blobs(nb, nper, shape, q, theta, r, S(stream));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_mobility_apply(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k, int dtype,
                        void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0) return set_error(h, RPBD_BAD_ARG, "n < 0");
    return mobility_apply_impl(h, n, r, F, U, k, dtype, false, S(stream));
}

int rpbd_mobility_apply_mixed(rpbd_handle* h, int64_t n, const double* r, const double* F, double* U, int k,
                              int dtype, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0) return set_error(h, RPBD_BAD_ARG, "n < 0");
    return mobility_apply_impl(h, n, r, F, U, k, dtype, true, S(stream));
}

int rpbd_K_apply(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* U,
                 double* out, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (nb < 0 || nper <= 0 || !r || !q || !U || !out) return set_error(h, RPBD_BAD_ARG, "K_apply: bad arguments");
    launch_K(nb, nper, r, q, U, out, S(stream));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_KT_apply(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* lam,
                  double* out, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (nb < 0 || nper <= 0 || !r || !q || !lam || !out)
        return set_error(h, RPBD_BAD_ARG, "KT_apply: bad arguments");
    launch_KT(nb, nper, r, q, lam, out, S(stream));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_philox_normals(rpbd_handle* h, uint64_t seed, uint32_t step, uint32_t sid, int64_t n, double* out,
                        void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || (n > 0 && !out)) return set_error(h, RPBD_BAD_ARG, "philox_normals: bad arguments");
    if (n / 4 >= (int64_t)0xffffffffLL) return set_error(h, RPBD_BAD_ARG, "philox_normals: n too large");
    launch_normals(seed, step, sid, n, out, S(stream));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

int rpbd_blob_forces(rpbd_handle* h, int64_t n, int nper, const double* r, const rpbd_forces* f, int dtype,
                     double* out, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || !r || !f || !out) return set_error(h, RPBD_BAD_ARG, "blob_forces: bad arguments");
    if (f->steric_gamma != 0.0 && (nper <= 0 || n % nper != 0 || !(f->steric_b > 0) || !(f->r_floor > 0)))
        return set_error(h, RPBD_BAD_ARG, "blob_forces: steric forces need nper | n, steric_b > 0, r_floor > 0");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "blob_forces: bad dtype");
    RPBD_TRY(launch_blob_forces(h, n, nper, r, *f, dtype, out, S(stream)));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

}  // extern "C"
