// Batched preconditioned Lanczos M^{1/2} W (Sec. 2.2) for many independent
// suspensions, plus an optional matvec per system, as one CUDA graph.
//
// All systems advance in lockstep, one Lanczos iteration per step: the matvec
// is the persistent batched pair kernel (batched.cu); dot products, the
// classical Gram-Schmidt reorthogonalisation (applied twice), the
// normalisation and the FP64 tridiagonal square root (one warp per system,
// cyclic Jacobi) all use per-system coefficients.  A system whose relative
// change |y_m - y_{m-1}|/|y_m| drops below tol is switched off by a device flag;
// later iterations skip its work, so max_iter iterations can be captured once
// and replayed without any host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rpbd_internal.cuh"
#include "tridiag_sqrt.cuh"

namespace rpbd {

constexpr int BLZ_MAX = 64;

__device__ __forceinline__ int bl_find_sys(const int64_t* off, int n_sys, int64_t i)
{
    int lo = 0, hi = n_sys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// out[s * ldo + i] = <V_i, w> restricted to system s (3 components)
__global__ void seg_dot_kernel(int64_t n, const int64_t* __restrict__ off, const double* __restrict__ V, int64_t ld,
                               const double* __restrict__ w, double* __restrict__ out, int ldo,
                               const int* __restrict__ active)
{
    const int s = blockIdx.x, i = blockIdx.y;
    if (active && !active[s]) return;
    const int64_t a = off[s], b = off[s + 1];
    const double* v = V + (int64_t)i * ld;
    double acc = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) acc += v[c * n + e] * w[c * n + e];
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[s * ldo + i] = acc;
    }
}

// w -= sum_i h[s][i] V_i   (s = system of the element)
__global__ void seg_axpy_kernel(int64_t n, int n_sys, const int64_t* __restrict__ off, const double* __restrict__ V,
                                int64_t ld, int nv, const double* __restrict__ h, int ldh, double* __restrict__ w,
                                const int* __restrict__ active)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = bl_find_sys(off, n_sys, e % n);
        if (!active[s]) continue;
        double acc = w[e];
        for (int i = 0; i < nv; ++i) acc -= h[s * ldh + i] * V[(int64_t)i * ld + e];
        w[e] = acc;
    }
}

__global__ void seg_add_kernel(int n_sys, int nv, int ldh, const double* __restrict__ a, double* __restrict__ b,
                               const int* __restrict__ active)
{
    const int s = blockIdx.x;
    if (!active[s]) return;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) b[s * ldh + i] += a[s * ldh + i];
}

// V_out = x / sqrt(nrm2[s]) for active systems
__global__ void seg_normalize_kernel(int64_t n, int n_sys, const int64_t* __restrict__ off, const double* __restrict__ x,
                                     const double* __restrict__ nrm2, double* __restrict__ out,
                                     const int* __restrict__ active)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = bl_find_sys(off, n_sys, e % n);
        if (active && !active[s]) continue;
        const double nv = sqrt(nrm2[s]);
        out[e] = nv > 0.0 ? x[e] / nv : 0.0;
    }
}

__global__ void blz_init_kernel(int n_sys, const double* __restrict__ W2, int* __restrict__ active,
                                int* __restrict__ iters, double* __restrict__ change, double* __restrict__ c,
                                double* __restrict__ cprev, int mdim)
{
    const int s = blockIdx.x;
    if (threadIdx.x == 0) {
        active[s] = W2[s] > 0.0 ? 1 : 0;
        iters[s] = 0;
        change[s] = 0.0;
    }
    for (int i = threadIdx.x; i < mdim; i += blockDim.x) {
        c[s * mdim + i] = 0.0;
        cprev[s * mdim + i] = 0.0;
    }
}

// one warp per system: alpha_m, beta_m; T^{1/2} e_1 (tridiag_sqrt.cuh); stop test
__global__ void blz_sqrt_kernel(int m, int max_iter, double tol, int mdim, const double* __restrict__ H,
                                const double* __restrict__ nrm2, const double* __restrict__ W2,
                                double* __restrict__ alpha, double* __restrict__ beta, double* __restrict__ c,
                                double* __restrict__ cprev, double* __restrict__ change, int* __restrict__ active,
                                int* __restrict__ iters)
{
    extern __shared__ double sm[];
    const int s = blockIdx.x;
    const int lane = threadIdx.x;
    if (!active[s]) return;
    const int m1 = m + 1;
    double* al = alpha + s * mdim;
    double* be = beta + s * mdim;
    if (lane == 0) {
        al[m] = H[s * (mdim + 1) + m];
        be[m] = sqrt(nrm2[s]);
    }
    __syncwarp();
    double* cs = c + s * mdim;
    tridiag_sqrt_e1(m1, al, be, sm, cs);
    double nc = 0.0, nd = 0.0;
    double* cp = cprev + s * mdim;
    for (int i = lane; i < m1; i += 32) {
        const double v = cs[i];
        const double prev = i < m1 - 1 ? cp[i] : 0.0;
        nc += v * v;
        nd += (v - prev) * (v - prev);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    __syncwarp();
    for (int i = lane; i < m1; i += 32) cp[i] = cs[i];
    if (lane == 0) {
        const double ch = nc > 0.0 ? sqrt(nd / nc) : 0.0;
        bool stop = false;
        if (m >= 1) {
            change[s] = ch;
            if (ch < tol) stop = true;
        }
        if (!(nrm2[s] > 1e-300 * W2[s])) stop = true;  // invariant subspace
        if (m1 >= max_iter) stop = true;
        if (stop) {
            active[s] = 0;
            iters[s] = m1;
        }
    }
}

// y[e] = sqrt(W2[s]) sum_{i < iters[s]} c[s][i] V_i[e]
__global__ void blz_combine_kernel(int64_t n, int n_sys, const int64_t* __restrict__ off, const double* __restrict__ V,
                                   int64_t ld, const double* __restrict__ c, int mdim, const int* __restrict__ iters,
                                   const double* __restrict__ W2, double* __restrict__ y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int s = bl_find_sys(off, n_sys, e % n);
        double acc = 0.0;
        for (int i = 0; i < iters[s]; ++i) acc += c[s * mdim + i] * V[(int64_t)i * ld + e];
        y[e] = sqrt(W2[s]) * acc;
    }
}

struct BatchGraph {
    std::vector<int64_t> off;
    int max_iter = 0;
    double tol = 0.0;
    int use_precond = 0;
    bool with_apply = false;
    int variant = -1;
    int test_stall = 0;  // the failure-path test option the kernels were captured with
    // every workspace buffer the captured kernels address: a buffer that has
    // grown (moved) since the capture invalidates the graph
    static constexpr int NSIG = 8;
    void* sig[NSIG] = {};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
};

void batched_free_graphs(rpbd_handle* h)
{
    for (BatchGraph* g : h->bgraphs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->cap) cudaStreamDestroy(g->cap);
        delete g;
    }
    h->bgraphs.clear();
}

struct BlzBufs {
    double *V, *z, *y, *w, *Win, *rin, *out, *Fin, *Uout;
    double *H1, *H2, *alpha, *beta, *c, *cprev, *nrm2, *W2, *change;
    int *active, *iters;
    int64_t* doff;
};

static unsigned sgrid(int64_t n)
{
    int64_t g = (3 * n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

// every kernel of one batched Lanczos (+ optional matvec), no host sync
static int blz_body(rpbd_handle* h, int n_sys, const int64_t* off, int64_t n, const BlzBufs& B, double tol,
                    int max_iter, int use_precond, bool with_apply, cudaStream_t st)
{
    const int mdim = BLZ_MAX + 1;
    const int64_t len = 3 * n;
    const unsigned g = sgrid(n);
    seg_dot_kernel<<<dim3(n_sys, 1), 256, 0, st>>>(n, B.doff, B.Win, 0, B.Win, B.W2, 1, nullptr);
    count_launch();
    blz_init_kernel<<<n_sys, 64, 0, st>>>(n_sys, B.W2, B.active, B.iters, B.change, B.c, B.cprev, mdim);
    count_launch();
    seg_normalize_kernel<<<g, 256, 0, st>>>(n, n_sys, B.doff, B.Win, B.W2, B.V, nullptr);
    count_launch();
    for (int m = 0; m < max_iter; ++m) {
        const double* vm = B.V + (int64_t)m * len;
        if (use_precond) {
            RPBD_TRY(precond_apply_impl(h, 2, vm, B.z, st, B.active, B.doff, n_sys));
            RPBD_TRY(batched_apply_impl(h, n_sys, off, B.rin, B.z, B.y, 1, true, B.active, st));
            RPBD_TRY(precond_apply_impl(h, 1, B.y, B.w, st, B.active, B.doff, n_sys));
        } else {
            RPBD_TRY(batched_apply_impl(h, n_sys, off, B.rin, vm, B.w, 1, true, B.active, st));
        }
        const int nv = m + 1;
        seg_dot_kernel<<<dim3(n_sys, nv), 256, 0, st>>>(n, B.doff, B.V, len, B.w, B.H1, mdim + 1, B.active);
        count_launch();
        seg_axpy_kernel<<<g, 256, 0, st>>>(n, n_sys, B.doff, B.V, len, nv, B.H1, mdim + 1, B.w, B.active);
        count_launch();
        seg_dot_kernel<<<dim3(n_sys, nv), 256, 0, st>>>(n, B.doff, B.V, len, B.w, B.H2, mdim + 1, B.active);
        count_launch();
        seg_axpy_kernel<<<g, 256, 0, st>>>(n, n_sys, B.doff, B.V, len, nv, B.H2, mdim + 1, B.w, B.active);
        count_launch();
        seg_add_kernel<<<n_sys, 64, 0, st>>>(n_sys, nv, mdim + 1, B.H2, B.H1, B.active);
        count_launch();
        seg_dot_kernel<<<dim3(n_sys, 1), 256, 0, st>>>(n, B.doff, B.w, 0, B.w, B.nrm2, 1, B.active);
        count_launch();
        const int m1 = m + 1;
        blz_sqrt_kernel<<<n_sys, 32, tridiag_sqrt_smem_doubles(m1) * sizeof(double), st>>>(m, max_iter, tol, mdim, B.H1, B.nrm2, B.W2,
                                                                         B.alpha, B.beta, B.c, B.cprev, B.change,
                                                                         B.active, B.iters);
        count_launch();
        seg_normalize_kernel<<<g, 256, 0, st>>>(n, n_sys, B.doff, B.w, B.nrm2, B.V + (int64_t)(m + 1) * len,
                                                B.active);
        count_launch();
    }
    blz_combine_kernel<<<g, 256, 0, st>>>(n, n_sys, B.doff, B.V, len, B.c, mdim, B.iters, B.W2,
                                          use_precond ? B.y : B.out);
    count_launch();
    if (use_precond) RPBD_TRY(precond_apply_impl(h, 0, B.y, B.out, st));
    if (with_apply) RPBD_TRY(batched_apply_impl(h, n_sys, off, B.rin, B.Fin, B.Uout, 1, true, nullptr, st));
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

static int blz_bufs(rpbd_handle* h, int n_sys, const int64_t* off, int64_t n, int max_iter, BlzBufs* B)
{
    const int64_t len = 3 * n;
    const int mdim = BLZ_MAX + 1;
    double* big;
    RPBD_TRY(ensure_t(h, BUF_BLZ, (size_t)(max_iter + 1) * len + 8 * len, &big));
    B->V = big;
    double* p = big + (size_t)(max_iter + 1) * len;
    B->z = p; p += len;
    B->y = p; p += len;
    B->w = p; p += len;
    B->Win = p; p += len;
    B->rin = p; p += len;
    B->out = p; p += len;
    B->Fin = p; p += len;
    B->Uout = p; p += len;
    double* sm;
    const size_t nsm = (size_t)n_sys * (2 * (mdim + 1) + 4 * mdim + 3) + (size_t)2 * n_sys + (n_sys + 1);
    RPBD_TRY(ensure_t(h, BUF_BLZ_SMALL, nsm, &sm));
    B->H1 = sm; sm += (size_t)n_sys * (mdim + 1);
    B->H2 = sm; sm += (size_t)n_sys * (mdim + 1);
    B->alpha = sm; sm += (size_t)n_sys * mdim;
    B->beta = sm; sm += (size_t)n_sys * mdim;
    B->c = sm; sm += (size_t)n_sys * mdim;
    B->cprev = sm; sm += (size_t)n_sys * mdim;
    B->nrm2 = sm; sm += n_sys;
    B->W2 = sm; sm += n_sys;
    B->change = sm; sm += n_sys;
    B->active = reinterpret_cast<int*>(sm); sm += n_sys;
    B->iters = reinterpret_cast<int*>(sm); sm += n_sys;
    B->doff = reinterpret_cast<int64_t*>(sm);
    RPBD_CU(h, cudaMemcpy(B->doff, off, sizeof(int64_t) * (n_sys + 1), cudaMemcpyHostToDevice));
    return RPBD_OK;
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

int rpbd_lanczos_sqrt_apply_batched(rpbd_handle* h, int n_sys, const int64_t* offsets, const double* r, const double* W,
                                    double* out, const double* F, double* U, double tol, int max_iter,
                                    int use_precond, int use_graph, int* iters, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n_sys <= 0 || !offsets || !r || !W || !out || (F && !U) || (!F && U))
        return set_error(h, RPBD_BAD_ARG, "batched lanczos: bad arguments");
    if (!(tol > 0) || max_iter < 1 || max_iter > BLZ_MAX)
        return set_error(h, RPBD_BAD_ARG, "batched lanczos: need tol > 0 and 1 <= max_iter <= 64");
    if (offsets[0] != 0) return set_error(h, RPBD_BAD_ARG, "batched lanczos: offsets must start at 0");
    const int64_t n = offsets[n_sys];
    if (use_precond && (!h->prec_valid || h->prec_nb * h->prec_nper != n))
        return set_error(h, RPBD_BAD_ARG, "batched lanczos: preconditioner not built for these blobs");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (once_per_device(h, reinterpret_cast<const void*>(blz_sqrt_kernel)))
        RPBD_CU(h, cudaFuncSetAttribute(blz_sqrt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        tridiag_sqrt_smem_doubles(BLZ_MAX) * (int)sizeof(double)));
    BlzBufs B;
    RPBD_TRY(blz_bufs(h, n_sys, offsets, n, max_iter, &B));
    const bool with_apply = F != nullptr;
    RPBD_CU(h, cudaMemcpyAsync(B.Win, W, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    RPBD_CU(h, cudaMemcpyAsync(B.rin, r, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    if (with_apply) RPBD_CU(h, cudaMemcpyAsync(B.Fin, F, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    RPBD_CU(h, cudaMemsetAsync(h->dev_flag, 0, sizeof(int), st));
    if (!use_graph) {
        RPBD_TRY(blz_body(h, n_sys, offsets, n, B, tol, max_iter, use_precond, with_apply, st));
    } else {
        BatchGraph* G = nullptr;
        auto signature = [&](void** sg) {
            const Buf bs[BatchGraph::NSIG] = {BUF_BLZ,     BUF_BLZ_SMALL, BUF_BPACK,  BUF_BPARTIAL,
                                              BUF_BSCALE,  BUF_BSEG,      BUF_PREC_L, BUF_PREC_LINV};
            for (int i = 0; i < BatchGraph::NSIG; ++i) sg[i] = h->buf[bs[i]];
        };
        void* sig[BatchGraph::NSIG];
        signature(sig);
        for (BatchGraph* c : h->bgraphs)
            if (c->max_iter == max_iter && c->tol == tol && c->use_precond == use_precond &&
                c->with_apply == with_apply && c->variant == h->batch_variant && c->test_stall == h->test_stall &&
                (int)c->off.size() == n_sys + 1 &&
                std::equal(c->off.begin(), c->off.end(), offsets) && std::equal(sig, sig + BatchGraph::NSIG, c->sig))
                G = c;
        if (!G) {
            // run once eagerly so every workspace buffer and work list exists,
            // then capture the same sequence of kernels
            RPBD_TRY(blz_body(h, n_sys, offsets, n, B, tol, max_iter, use_precond, with_apply, st));
            RPBD_CU(h, cudaStreamSynchronize(st));
            void* sig2[BatchGraph::NSIG];
            signature(sig2);
            G = new BatchGraph();
            G->off.assign(offsets, offsets + n_sys + 1);
            G->max_iter = max_iter;
            G->tol = tol;
            G->use_precond = use_precond;
            G->with_apply = with_apply;
            G->variant = h->batch_variant;
            G->test_stall = h->test_stall;
            std::copy(sig2, sig2 + BatchGraph::NSIG, G->sig);
            h->bgraphs.push_back(G);
            RPBD_CU(h, cudaStreamCreateWithFlags(&G->cap, cudaStreamNonBlocking));
            const bool prof = h->profile;
            h->profile = false;
            RPBD_CU(h, cudaStreamBeginCapture(G->cap, cudaStreamCaptureModeThreadLocal));
            const int s_body = blz_body(h, n_sys, offsets, n, B, tol, max_iter, use_precond, with_apply, G->cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t e_end = cudaStreamEndCapture(G->cap, &graph);
            h->profile = prof;
            if (s_body != RPBD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s_body;
            }
            if (e_end != cudaSuccess) return set_error(h, RPBD_CUDA, "batched lanczos: graph capture failed");
            const cudaError_t e_inst = cudaGraphInstantiate(&G->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e_inst != cudaSuccess) return set_error(h, RPBD_CUDA, "batched lanczos: graph instantiate failed");
        }
        RPBD_CU(h, cudaGraphLaunch(G->exec, st));
        count_launch();
    }
    RPBD_CU(h, cudaMemcpyAsync(out, B.out, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    if (with_apply) RPBD_CU(h, cudaMemcpyAsync(U, B.Uout, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st));
    if (iters) {
        RPBD_CU(h, cudaMemcpyAsync(iters, B.iters, sizeof(int) * n_sys, cudaMemcpyDeviceToHost, st));
        RPBD_CU(h, cudaStreamSynchronize(st));
        int flag = 0;
        RPBD_CU(h, cudaMemcpy(&flag, h->dev_flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag == 1) return set_error(h, RPBD_TIMEOUT, "batched lanczos: a pair kernel's bounded wait expired");
    }
    return RPBD_OK;
}

}  // extern "C"
