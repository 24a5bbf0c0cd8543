// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rpbd.h"

namespace rpbd {

// ---------------------------------------------------------------------------
// Error handling

struct Status {
    int code = RPBD_OK;
};

#define RPBD_CU(h, call)                                                          \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return rpbd::set_error((h), RPBD_CUDA,             \
                                                      std::string(#call) + ": " + \
                                                          cudaGetErrorString(e_)); \
    } while (0)

#define RPBD_LAUNCH_CHECK(h)                                                  \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess)                                                \
            return rpbd::set_error((h), RPBD_CUDA,                            \
                                   std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define RPBD_TRY(expr)          \
    do {                        \
        int s_ = (expr);        \
        if (s_ != RPBD_OK) return s_; \
    } while (0)

// ---------------------------------------------------------------------------
// Device workspace: named growable buffers owned by the handle.

enum Buf {
    BUF_PACK = 0,    // packed source records of the pair kernels
    BUF_SCALE,       // per-blob overlap scale s_i
    BUF_PARTIAL,     // per-chunk partial sums of the pair kernels
    BUF_PREC_L,      // block Cholesky factors
    BUF_PREC_LINV,   // their inverses
    BUF_PREC_MINV,   // M(pp)^-1
    BUF_PREC_MINVK,  // M(pp)^-1 K_p
    BUF_PREC_N,      // N_p
    BUF_PREC_Q,      // tracking points of the preconditioner's bodies
    BUF_KRYLOV,      // Krylov basis
    BUF_VEC,         // solver vectors
    BUF_SMALL,       // small device scalars (Hessenberg, tridiagonal, flags)
    BUF_STEP,        // time-step vectors
    BUF_R2,          // displaced positions (RFD, predictor)
    BUF_AUX,         // misc
    BUF_BPACK,       // batched: packed records of all systems
    BUF_BSCALE,      // batched: overlap scales
    BUF_BPARTIAL,    // batched: chunk partials
    BUF_BAUX,        // batched: autotune vectors
    BUF_BLZ,         // batched Lanczos: basis and vectors
    BUF_BLZ_SMALL,   // batched Lanczos: per-system scalars
    BUF_SYM_ITEMS,   // symmetric kernel: work items
    BUF_GMRES_MV,    // lockstep GMRES: gathered multi-RHS matvec operands
    BUF_SYM_SEG,     // symmetric kernel: segment sums of the visitor partials
    BUF_BSEG,        // batched symmetric kernel: segment sums of the visitor partials
    BUF_COUNT
};

struct BatchPlan;
struct BatchGraph;
struct Sym2Plan;

struct ProfRec {
    cudaEvent_t a, b;
    int dtype, k;
    double pairs;
};

// cached work list of a symmetric kernel (per n)
struct SymPlan {
    int64_t n = -1;
    int n_items = 0, n_home = 0, max_slots = 0, chunk = 0;
};

}  // namespace rpbd

#include <vector>

inline int sym_class(int k) { return k <= 1 ? 0 : (k == 2 ? 1 : 2); }

struct rpbd_handle {
    rpbd_params p;
    int device = 0;
    int sm_count = 0;
    std::string err;
    void* buf[rpbd::BUF_COUNT] = {};
    size_t cap[rpbd::BUF_COUNT] = {};
    // preconditioner state
    int64_t prec_nb = 0;
    int prec_nper = 0;
    bool prec_valid = false;
    // pinned host mirror for small read-backs
    double* host_small = nullptr;
    // device error flag (bounded waits in kernels)
    int* dev_flag = nullptr;
    // pair-kernel timing
    bool profile = false;
    std::vector<rpbd::ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    // batched launches: cached work lists, chosen tile variant, captured graphs
    std::vector<rpbd::BatchPlan*> bplans;
    int batch_variant = -1;
    std::vector<rpbd::BatchGraph*> bgraphs;
    rpbd::BatchPlan* mv_plan = nullptr;  // work list of the single-system packed matvec
    std::vector<rpbd::Sym2Plan*> sym2_plans;  // work lists of the packed symmetric kernel, per offsets
    // symmetric FP32 kernel (k <= 4): on by default, work list cached per n
    // symmetric-kernel choice per right-hand-side class (k = 1, k = 2, 3 <= k <= 4):
    // use it (1) or the one-direction kernel (0); variant -1: default, 0..3:
    // loop unroll / occupancy variants
    int use_sym[3] = {1, 1, 1};
    int sym_variant[3] = {-1, -1, -1};
    rpbd::SymPlan sym_plan;     // work list of the one-home symmetric kernel (128-blob home tiles)
    int use_packed = 1;         // k <= 4 with the wall: the packed two-homes-per-thread symmetric kernel
    // failure-path test (RPBD_OPT_TEST_STALL): the pair kernels leave their
    // first source stage's barrier without a copy, so its bounded wait runs
    // out after a short limit and the kernel reports RPBD_TIMEOUT
    int test_stall = 0;
    // RPBD_OPT_FARFIELD: single-system FP32 matvecs with the wall form every
    // block with the cancellation-free direct-minus-image differences
    int far_field = 0;
    // RPBD_OPT_SYM_PARTIALS: the packed symmetric kernel of one system writes
    // per-home-tile partials reduced in a fixed order (memory O(n^2)) instead of
    // its fixed-point accumulation (memory O(n))
    int sym_partials = 0;
};

namespace rpbd {

int set_error(rpbd_handle* h, int code, const std::string& msg);
// true the first time it is called for (h's device, key), false afterwards;
// guards per-device one-time settings such as a kernel's shared-memory limit
bool once_per_device(rpbd_handle* h, const void* key);
// wait limit (SM clock cycles) and first-stage skip of the pair kernels'
// source ring: ~2 s normally; a short limit with the skip under the
// failure-path test option
struct RingTest {
    long long limit;
    int skip_first;
};
inline RingTest ring_test(const rpbd_handle* h)
{
    return h->test_stall ? RingTest{200000LL, 1} : RingTest{4000000000LL, 0};
}
// library-wide count of kernel launches (read by rpbd_launch_count)
void count_launch();
// pair-kernel timing records (rpbd_profile_*)
void prof_begin(rpbd_handle* h, cudaStream_t st);
void prof_end(rpbd_handle* h, cudaStream_t st, int dtype, int k, double pairs);
// Ensure buffer b holds at least `bytes`; contents are not preserved.
int ensure(rpbd_handle* h, Buf b, size_t bytes, void** out);
template <class T>
inline int ensure_t(rpbd_handle* h, Buf b, size_t count, T** out)
{
    void* p = nullptr;
    int s = ensure(h, b, count * sizeof(T), &p);
    *out = static_cast<T*>(p);
    return s;
}

// mobility apply on FP64 blob vectors; dtype chooses the pair arithmetic
int mobility_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U,
                        int k, int dtype, bool io_double, cudaStream_t st);

// rigid kernels (FP64)
void launch_K(int64_t nb, int nper, const double* r, const double* q, const double* U,
              double* out, cudaStream_t st);
void launch_KT(int64_t nb, int nper, const double* r, const double* q, const double* lam,
               double* out, cudaStream_t st);
void launch_blobs(int64_t nb, int nper, const double* shape, const double* q,
                  const double* theta, double* r, cudaStream_t st);
void launch_normals(uint64_t seed, uint32_t step, uint32_t sid, int64_t n, double* out,
                    cudaStream_t st);
int launch_blob_forces(rpbd_handle* h, int64_t n, int nper, const double* r, const rpbd_forces& f, int dtype,
                       double* out, cudaStream_t st);
// q += s * U[:, :3]; theta = Rotate(theta, s * U[:, 3:])
void launch_advance(int64_t nb, const double* q0, const double* th0, const double* U, double s,
                    double* q1, double* th1, cudaStream_t st);

// FP64 vector helpers
void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t st);
void launch_scale_copy(int64_t n, double a, const double* x, double* out, cudaStream_t st);
int check_finite(rpbd_handle* h, int64_t n, const double* x, cudaStream_t st);

// active != nullptr (batches): bodies of systems with active[s] == 0 skipped,
// systems at device blob offsets off[0..n_sys]
int precond_apply_impl(rpbd_handle* h, int mode, const double* x, double* out, cudaStream_t st,
                       const int* active = nullptr, const int64_t* off = nullptr, int n_sys = 0);
// saddle block solve: (lam, U) = P^-1 (a, b)
int precond_saddle_impl(rpbd_handle* h, const double* a, const double* b, double* lam,
                        double* U, cudaStream_t st);

int lanczos_impl(rpbd_handle* h, int64_t n, const double* r, const double* W, double* out,
                 double tol, int max_iter, int dtype, int use_precond, rpbd_stats* stats,
                 cudaStream_t st);
// One saddle problem for gmres_multi_impl: b = [-slip; -FT] (either may be
// null: zero), outputs lambda [3][n], U [nb][6]; warm != 0: they hold x0.
struct GmresProblem {
    const double* slip;
    const double* FT;
    double* lambda;
    double* U;
    double tol;
    int max_iter;
    int warm;
};
// 1..4 GMRES processes on the same positions, advanced in lockstep so their
// matvecs share one multi-RHS launch.
int gmres_multi_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, int nsys,
                     const GmresProblem* probs, int restart, int dtype, int build_precond, rpbd_stats* stats,
                     cudaStream_t st);
int gmres_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
               const double* slip, const double* FT, double* lambda, double* U, double tol,
               int max_iter, int restart, int dtype, int build_precond, int warm, rpbd_stats* stats,
               cudaStream_t st);
int precond_build_impl(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
                       cudaStream_t st);

// symmetric FP32 matvec, k <= 4
int sym_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k, bool io_double,
                   cudaStream_t st);

// batched systems (concatenated SoA; host offsets)
int batched_apply_impl(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const void* F, void* U,
                       int k, bool io_double, const int* active, cudaStream_t st);
// one system through the packed batched tile (two targets per thread): the
// one-direction FP32 matvec with the wall in the open cell, k in {1, 3, 4}
int single_packed_apply_impl(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U, int k,
                             bool io_double, cudaStream_t st);
// the packed symmetric kernel over a batch of systems (wall, open cell, k <= 4)
int sym_batched_apply_impl(rpbd_handle* h, int n_sys, const int64_t* off, const double* r, const void* F, void* U,
                           int k, bool io_double, const int* active, cudaStream_t st);
void free_sym2_plans(rpbd_handle* h);
void batched_free_plans(rpbd_handle* h);
void batched_free_graphs(rpbd_handle* h);

}  // namespace rpbd
