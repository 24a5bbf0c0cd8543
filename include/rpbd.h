/*
 * rpbd.h -- C ABI of the GB300 library for rigid-multiblob Brownian dynamics
 * above a no-slip wall (Sprinkle, Balboa Usabiaga, Patankar, Donev, "Large
 * Scale Brownian Dynamics of Confined Suspensions of Rigid Particles").
 *
 * Conventions (all entry points):
 *  - Every array argument is a DEVICE pointer owned by the caller, unless
 *    the comment says "host".  The library never frees caller memory.
 *  - Blob positions are SoA: r[0..n) = x, r[n..2n) = y, r[2n..3n) = z (FP64).
 *  - Blob vectors (forces, velocities) are [k][3][n]: RHS-major, then
 *    component, then blob.
 *  - Bodies: nb bodies of one shape with nper blobs each; blob i of body p is
 *    index p * nper + i.  Body vectors are [nb][6] rows (u, omega) or
 *    (f, tau); tracking points q [nb][3]; unit quaternions theta [nb][4] as
 *    (s, p_x, p_y, p_z).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    Kernel-only calls are asynchronous on that stream.  Calls that run a
 *    Krylov iteration (Lanczos, GMRES, steps) read a residual back to the
 *    host once per iteration and return only when done.
 *  - Return value: RPBD_OK (0) or a negative status; rpbd_last_error(h)
 *    gives a message.  The calls that synchronise (Lanczos, GMRES, time
 *    steps) check the blob positions first and return RPBD_BAD_INPUT for
 *    NaN/Inf; the asynchronous kernel-only calls do not read anything back,
 *    so non-finite inputs there give non-finite outputs.
 *  - The handle owns a device workspace that grows on demand
 *    (cudaMalloc); rpbd_reserve() sizes it ahead of time.  A handle is used
 *    by one host thread at a time.
 *  - Units are the caller's; the paper's workloads use um, s, mg.
 */
#ifndef RPBD_H
#define RPBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RPBD_OK 0
#define RPBD_BAD_ARG (-1)
#define RPBD_BAD_INPUT (-2)
#define RPBD_CUDA (-3)
#define RPBD_NOT_CONVERGED (-4)
#define RPBD_TIMEOUT (-5)
#define RPBD_NO_MEM (-6)
#define RPBD_TOO_LARGE (-7) /* beyond the fixed scratch of rpbd_mobility_apply_f32_noalloc */

/* arithmetic of the pair kernels */
#define RPBD_F64 0 /* FP64 pair math, FP64 accumulation */
#define RPBD_F32 1 /* FP32 pair math; FP32 tile partials summed as compensated float pairs (two-sum, ~48 bits), then FP64 */

typedef struct rpbd_handle rpbd_handle;

/* Physical parameters (Sec. 2.1, Sec. 4). */
typedef struct rpbd_params {
    double eta;   /* fluid viscosity */
    double a;     /* blob hydrodynamic radius */
    double kT;    /* thermal energy k_B T */
    int wall;     /* 1: no-slip wall at z = 0 (Rotne-Prager-Blake); 0: unbounded RPY */
    double s_min; /* floor of the wall-overlap scale s_i = clamp(z_i/a, s_min, 1) */
    double Lx, Ly; /* > 0 (both): pseudo-periodic cell of Sec. 4.2 -- every pair sums the
                      source's minimum image in x, y and its 8 nearest periodic images;
                      needs wall = 1.  0, 0: open in x, y.  The batched and
                      allocation-free calls take open systems only. */
} rpbd_params;

/* Per-call solver statistics (host struct, filled before return). */
typedef struct rpbd_stats {
    int iterations;  /* Krylov iterations */
    int matvecs;     /* applications of M */
    double residual; /* GMRES: relative residual; Lanczos: last relative change */
    int status;      /* RPBD_OK or RPBD_NOT_CONVERGED */
} rpbd_stats;

/* Deterministic forces for the time steps (Sec. 4): per-blob gravity -weight z^,
 * blob-wall Yukawa repulsion gamma exp(-h/b)/h evaluated at h = max(z, h_floor),
 * a constant torque on every body, and (steric_gamma != 0) the blob-blob
 * Yukawa repulsion steric_gamma exp(-r/steric_b)/r between blobs of different
 * bodies, evaluated at max(r, r_floor) and skipped beyond r_cut (0: no cut). */
typedef struct rpbd_forces {
    double weight;
    double wall_gamma;
    double wall_b;
    double h_floor;
    double torque[3];
    double steric_gamma;
    double steric_b;
    double r_floor;
    double r_cut;
} rpbd_forces;

/* Time-step controls (Algorithms 1 and 2). */
typedef struct rpbd_step_params {
    double dt;          /* time step */
    double delta;       /* RFD displacement parameter */
    double Lp;          /* body length scale L_p of the RFD (same for all bodies) */
    double tol_gmres;   /* relative residual of every saddle solve */
    double tol_lanczos; /* relative change stop test of Lanczos */
    int max_iter_gmres;
    int restart;        /* GMRES(m) restart length */
    int max_iter_lanczos;
    int dtype;          /* RPBD_F32 or RPBD_F64 pair arithmetic */
    uint64_t seed;      /* Philox key */
    uint32_t step;      /* step counter (Philox counter word 1) */
    int cold_start;     /* 0 (default): a solve that follows one with a nearby operator and
                           right-hand side (T-S / T-T corrector after the predictor, EM-RFD
                           solve at Q- after Q+) starts GMRES from that solution; 1: every
                           solve starts from zero */
} rpbd_step_params;

/* ---- handle ------------------------------------------------------------ */

/* Create a handle bound to the current CUDA device.  *h receives it. */
int rpbd_create(rpbd_handle** h, const rpbd_params* p);
int rpbd_destroy(rpbd_handle* h);
/* Pre-size the workspace for n blobs, nb bodies of nper blobs, k right-hand
 * sides and a Krylov basis of `basis` vectors (0 for none). */
int rpbd_reserve(rpbd_handle* h, int64_t n, int64_t nb, int nper, int k, int basis);
const char* rpbd_last_error(const rpbd_handle* h);
const char* rpbd_status_string(int status);

/* ---- a1: blob geometry (Sec. 2.1 multiblob model, App. B.1) ------------ */

/* r_i = q_p + R(theta_p) shape_i for every blob; shape [nper][3] (device). */
int rpbd_blobs_from_bodies(rpbd_handle* h, int64_t nb, int nper, const double* shape,
                           const double* q, const double* theta, double* r, void* stream);

/* ---- a2: wall-RPY matvec (Sec. 2.1; the dense GPU sum of Sec. 2.1/4.2) -- */

/* U = M(r) F for k right-hand sides (1 <= k <= 16; k in {1,2,4,8,16} hit
 * specialised kernels, other k run as the next larger one).  F and U are
 * [k][3][n] of type double (dtype RPBD_F64) or float (RPBD_F32).
 * M_ij = s_i s_j [M_RPY(r~_i - r~_j) + M_wall(r~_i, r~_j)], r~ = (x, y, max(z, a)). */
int rpbd_mobility_apply(rpbd_handle* h, int64_t n, const double* r, const void* F, void* U,
                        int k, int dtype, void* stream);

/* Same, FP64 blob vectors in and out with the pair arithmetic chosen by
 * dtype (the mixed mode the Krylov solvers use). */
int rpbd_mobility_apply_mixed(rpbd_handle* h, int64_t n, const double* r, const double* F,
                              double* U, int k, int dtype, void* stream);

/* Allocation-free FP32 matvec, for callers that must not call the CUDA
 * allocator at all: for example a plug-in running inside a host framework
 * whose caching allocator owns the device memory, or a real-time loop where
 * an allocation's latency or failure is not acceptable.  The paper has no
 * counterpart; it computes exactly what rpbd_mobility_apply computes with
 * dtype RPBD_F32 (F and U float [k][3][n], r double SoA).
 *  - No handle: the physical parameters come in *p.  Allocates nothing and
 *    calls no allocating routine; its scratch is one 27.6 MiB array in device
 *    memory that the library declares statically, which every GPU that loads
 *    the library holds until the process exits.
 *  - Limits set by that array: n <= 16384 blobs and k <= 16; larger sizes
 *    return RPBD_TOO_LARGE and do nothing.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call uses the same array, whatever the stream: calls that can
 *    overlap on the GPU (different streams, or different host threads) race
 *    on it and corrupt each other's results; order them.
 *  - Asynchronous on `stream`; returns RPBD_OK, RPBD_TOO_LARGE, RPBD_BAD_ARG
 *    or RPBD_CUDA (no handle, so no message beyond rpbd_status_string).
 *  - The pair kernel's waits for its source copies are bounded (~2 s); if
 *    one runs out, every value of U is set to NaN, since the status has
 *    already been returned when the kernel runs. */
int rpbd_mobility_apply_f32_noalloc(const rpbd_params* p, int64_t n, const double* r, const float* F,
                                    float* U, int k, void* stream);

/* ---- a7: adjoint and divergence ---------------------------------------- */

/* grad[3][n] = d(u^T M(r) F)/dr, FP64; u, F [3][n].  The derivative of the
 * matvec of Sec. 2.1 with respect to the blob positions. */
int rpbd_mobility_adjoint(rpbd_handle* h, int64_t n, const double* r, const double* u,
                          const double* F, double* grad, void* stream);

/* Same gradient with the pair block and its derivative evaluated in FP32
 * (position differences formed in FP64 first; sums in FP64). */
int rpbd_mobility_adjoint_f32(rpbd_handle* h, int64_t n, const double* r, const double* u,
                              const double* F, double* grad, void* stream);

/* grad[3][n] = d( sum_m u_m^T M(r) F_m )/dr for k right-hand-side pairs
 * (1 <= k <= 16; u, F [k][3][n] FP64): the gradient of a loss of the k-RHS
 * matvec of Sec. 2.1, summed over the pairs on the device.  Each pair block
 * and its derivative are formed once for all k (FP32: in passes of up to four
 * pairs).  dtype RPBD_F64 or RPBD_F32 selects the pair arithmetic as in the
 * two calls above; sums are FP64. */
int rpbd_mobility_adjoint_multi(rpbd_handle* h, int64_t n, const double* r, const double* u,
                                const double* F, int k, double* grad, int dtype, void* stream);

/* div[3][n] = sum_j d_{r_j} . M_ij (the quantity the RFD of Sec. 3 estimates
 * with B = M), FP64. */
int rpbd_mobility_divergence(rpbd_handle* h, int64_t n, const double* r, double* div,
                             void* stream);

/* ---- rigid operators (eq. K and force/torque balance, Sec. 2.1) -------- */

/* out[3][n] = K U: u_p + omega_p x (r_i - q_p). */
int rpbd_K_apply(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
                 const double* U, double* out, void* stream);
/* out[nb][6] = K^T lam: (sum_i lam_i, sum_i (r_i - q_p) x lam_i). */
int rpbd_KT_apply(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
                  const double* lam, double* out, void* stream);

/* ---- a3: body-block-diagonal preconditioner (Sec. 2.2) ----------------- */

/* Build, for every body p, the dense M(pp) of its blobs alone (wall
 * included), its Cholesky factor L_p, L_p^-1, M(pp)^-1 and
 * N_p = (K_p^T M(pp)^-1 K_p)^-1 in FP64.  Kept in the handle until the next
 * build. */
int rpbd_precond_build(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
                       void* stream);
/* Apply a stored factor to a blob vector [3][n]: mode 0: out = L x;
 * 1: out = L^-1 x; 2: out = L^-T x; 3: out = M~^-1 x. */
int rpbd_precond_apply(rpbd_handle* h, int mode, const double* x, double* out, void* stream);

/* ---- a4: preconditioned Lanczos M^{1/2} W (Sec. 2.2) ------------------- */

/* out[3][n] ~ L f(L^-1 M L^-T) W with f = sqrt, by Lanczos with full
 * reorthogonalisation from v_1 = W/|W|; stops when |y_m - y_{m-1}|/|y_m| < tol.
 * use_precond = 0 runs on M itself (L = I).  W, out: [3][n] FP64.
 * 1 <= max_iter <= 80 (the basis and the tridiagonal square root are sized
 * for 80); RPBD_NOT_CONVERGED when it stops at max_iter (out then holds the
 * last iterate). */
int rpbd_lanczos_sqrt_apply(rpbd_handle* h, int64_t n, const double* r, const double* W,
                            double* out, double tol, int max_iter, int dtype, int use_precond,
                            rpbd_stats* stats, void* stream);

/* nsys (1..4) Lanczos square roots M^{1/2} W_s at the same r (same M and
 * preconditioner), each as in rpbd_lanczos_sqrt_apply.  The processes are
 * advanced in lockstep, so each iteration's matvecs go out as one multi-RHS
 * launch and their scalars come back with one synchronisation; every process
 * keeps its own basis, tridiagonal matrix and stopping test (the answers are
 * those of nsys separate calls; this is not a block-Krylov method).  W and out
 * are HOST arrays of nsys DEVICE pointers ([3][n] each); stats (host, may be
 * NULL) receives nsys records.  Returns RPBD_NOT_CONVERGED when any process
 * stopped at max_iter. */
int rpbd_lanczos_sqrt_apply_multi(rpbd_handle* h, int64_t n, const double* r, int nsys,
                                  const double* const* W, double* const* out, double tol, int max_iter,
                                  int dtype, int use_precond, rpbd_stats* stats, void* stream);

/* ---- a5: GMRES saddle-point mobility solve (eq. saddle, Sec. 2.1) ------ */

/* Solve [M -K; -K^T 0][lambda; U] = [-slip; -FT] by right-preconditioned
 * restarted GMRES with the body-block preconditioner built on the same r, q
 * (built here when build_precond != 0).  slip [3][n] or NULL (zero); FT
 * [nb][6] or NULL (zero); lambda [3][n] and U [nb][6] outputs.  Stops on
 * the relative residual |b - A x|/|b| <= tol.  warm_start != 0: lambda and U
 * hold the initial guess x0 on entry (the stopping test is still relative to
 * |b|); otherwise x0 = 0 and their contents are ignored. */
int rpbd_gmres_rigid_solve(rpbd_handle* h, int64_t nb, int nper, const double* r,
                           const double* q, const double* slip, const double* FT,
                           double* lambda, double* U, double tol, int max_iter, int restart,
                           int dtype, int build_precond, int warm_start, rpbd_stats* stats,
                           void* stream);

/* nsys (1..4) saddle problems at the same r, q (same M, K and preconditioner),
 * each as in rpbd_gmres_rigid_solve with x0 = 0.  Their GMRES processes are
 * advanced in lockstep, so each iteration's matvecs go out as one multi-RHS
 * launch and the residuals come back with one synchronisation.  slip, FT,
 * lambda and U are HOST arrays of nsys DEVICE pointers (slip[s], FT[s] may be
 * NULL: zero); stats (host, may be NULL) receives nsys records.  Returns
 * RPBD_NOT_CONVERGED when any process stopped at max_iter. */
int rpbd_gmres_rigid_solve_multi(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q,
                                 int nsys, const double* const* slip, const double* const* FT,
                                 double* const* lambda, double* const* U, double tol, int max_iter,
                                 int restart, int dtype, int build_precond, rpbd_stats* stats,
                                 void* stream);

/* ---- a6: random finite difference drift (Sec. 3, eq. RFDcenter) -------- */

/* drift[3][n] = (1/delta) [M(r + delta/2 W) - M(r - delta/2 W)] W; its mean
 * over W ~ N(0, I) is div M + O(delta^2). */
int rpbd_rfd_drift(rpbd_handle* h, int64_t n, const double* r, const double* W, double delta,
                   double* drift, int dtype, void* stream);

/* ---- many independent suspensions (batched; the paper's per-suspension
 *      matvec and Lanczos of Sec. 2.1-2.2 applied to a batch) --------------- */

/* System s owns blobs [offsets[s], offsets[s+1]) of the concatenated SoA
 * arrays r [3][N], F, U [k][3][N] (N = offsets[n_sys]); blobs interact only
 * inside their system.  offsets is a HOST array of n_sys + 1 int64 starting
 * at 0.  FP32 pair arithmetic, FP32 F and U, 1 <= k <= 16 (k in {1, 4, 16}
 * hit specialised kernels, other k run as the next larger one).  One
 * persistent launch over a work list of (system, target tile, source chunk)
 * items with the tile shape chosen by rpbd_autotune_batched (default: the
 * packed 256-target tile with the wall, else 128 targets x 64 sources).  The
 * work list is cached per offsets. */
int rpbd_mobility_apply_batched(rpbd_handle* h, int n_sys, const int64_t* offsets, const double* r,
                                const float* F, float* U, int k, void* stream);

/* Times every compiled tile variant of the batched kernel on this batch (k
 * right-hand sides, zero forces), keeps the fastest in the handle and
 * returns its index (>= 0) or a negative status.  *best_ms (host, may be
 * NULL) receives its time per launch.  Synchronises the stream. */
int rpbd_autotune_batched(rpbd_handle* h, int n_sys, const int64_t* offsets, const double* r, int k,
                          double* best_ms, void* stream);

/* Preconditioned (use_precond != 0: the block preconditioner built on all N
 * blobs) Lanczos M^{1/2} W of every system at once, FP32 pairs, FP64 vectors
 * and tridiagonal square root, per-system stop test as in
 * rpbd_lanczos_sqrt_apply; optionally also U = M F per system (F, U FP64
 * [3][N], both NULL to skip).  use_graph != 0 captures the whole sequence
 * (max_iter iterations, converged systems masked off on the device) into a
 * CUDA graph on first use and replays it: one launch per call.  iters (host,
 * n_sys ints, may be NULL) receives each system's Lanczos iterations; then
 * the call synchronises the stream.  1 <= max_iter <= 64. */
int rpbd_lanczos_sqrt_apply_batched(rpbd_handle* h, int n_sys, const int64_t* offsets,
                                    const double* r, const double* W, double* out, const double* F,
                                    double* U, double tol, int max_iter, int use_precond,
                                    int use_graph, int* iters, void* stream);

/* ---- random numbers ---------------------------------------------------- */

/* out[e] for e < n: standard normals from Philox4x32-10 (Salmon et al.,
 * SC'11) keyed by seed, counter (e/4, step, sid, 0), Box-Muller on word pairs. */
int rpbd_philox_normals(rpbd_handle* h, uint64_t seed, uint32_t step, uint32_t sid, int64_t n,
                        double* out, void* stream);

/* ---- a8: time steps ----------------------------------------------------- */

/* One Trapezoidal-Slip step (Algorithm 2) or Euler-Maruyama-Traction step
 * (Algorithm 1) of nb bodies: q [nb][3] and theta [nb][4] are updated in
 * place; shape [nper][3].  Random vectors are drawn with
 * rpbd_philox_normals(seed, step, sid): T-S uses sid 0 for W^s [3][n] and
 * sid 1 for W [3][n]; EM-T uses sid 2 for (W^f, W^tau) as [nb][6] rows and
 * sid 1 for W.  stats (host) receives, in order: T-S: RFD solve, Lanczos,
 * predictor solve, corrector solve; EM-T: RFD solve, Lanczos, solve. */
int rpbd_step_ts(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q,
                 double* theta, const rpbd_forces* forces, const rpbd_step_params* sp,
                 rpbd_stats* stats /* host, 4 entries */, void* stream);
int rpbd_step_emt(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q,
                  double* theta, const rpbd_forces* forces, const rpbd_step_params* sp,
                  rpbd_stats* stats /* host, 3 entries */, void* stream);

/* One Euler-Maruyama RFD step (Algorithm 3, App. A): mobility problems with
 * random force W^FT at Q+- = Q +- delta/2 [L_p W^f; W^tau], Lanczos, one solve
 * at Q^n, Q^{n+1} = Q^n + dt (U^n + (U+ - U-)/delta).  Random draws as EM-T
 * (sid 2 for (W^f, W^tau), sid 1 for W).  stats (host, 4 entries): solve at
 * Q+, solve at Q-, Lanczos, solve at Q^n. */
int rpbd_step_emrfd(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q,
                    double* theta, const rpbd_forces* forces, const rpbd_step_params* sp,
                    rpbd_stats* stats /* host, 4 entries */, void* stream);
/* One Trapezoidal Traction step (Sec. 3.2): D^F and D^S as in step 1 of
 * Algorithm 1 without the U^RFD term, then the predictor-corrector of
 * Algorithm 2 (corrector slip 2 D^S + ..., force F~ - 2 D^F).  Random draws as
 * EM-T.  stats (host, 4 entries): RFD solve, Lanczos, predictor, corrector. */
int rpbd_step_tt(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q,
                 double* theta, const rpbd_forces* forces, const rpbd_step_params* sp,
                 rpbd_stats* stats /* host, 4 entries */, void* stream);

/* Blob forces [3][n] of the force model at r (gravity, wall repulsion and,
 * with nper > 0 bodies of nper consecutive blobs, the blob-blob repulsion,
 * an all-pairs O(n^2) sum computed in `dtype` arithmetic from FP64
 * separations).  BAD_ARG when steric_gamma != 0 and nper does not divide n,
 * steric_b <= 0 or r_floor <= 0. */
int rpbd_blob_forces(rpbd_handle* h, int64_t n, int nper, const double* r, const rpbd_forces* forces,
                     int dtype, double* f, void* stream);

/* ---- options -------------------------------------------------------------- */

/* value != 0 (default): FP32 matvecs with k <= 4 use the symmetric kernel,
 * which forms each unordered pair's block once and applies it both ways
 * (M_ji = M_ij^T, Sec. 2.1); 0: the one-direction kernel for every k.  Sets
 * every right-hand-side class (see rpbd_autotune). */
#define RPBD_OPT_SYMMETRIC 1
/* -1 (default): per-k default; 0..5: loop-unroll / occupancy variant of the
 * symmetric kernel, for every right-hand-side class (4, 5: the packed kernel
 * with four home blobs per thread; the one-home kernel has 0..3 and runs 4, 5
 * as 0). */
#define RPBD_OPT_SYM_VARIANT 2
/* value != 0 (default): with the wall (open or periodic cell), symmetric
 * matvecs (k <= 4) use the packed kernel (two home blobs per thread, both
 * pair blocks formed by two-wide FP32 instructions); 0: the one-home kernel. */
#define RPBD_OPT_PACKED 3
/* tile variant of the batched kernel (what rpbd_autotune_batched picks):
 * -1: the default (4 with the wall, else 0); 0: 128 targets x 64-source
 * tiles, 1: 64 x 64, 2: 256 x 32, 3 (wall only): 256 targets, two per thread
 * in packed two-wide FP32 x 64-source tiles; 4 (wall only, k <= 4): the
 * packed symmetric kernel over the batch (each system's unordered pairs
 * formed once, applied both ways; k > 4 then runs on variant 3). */
#define RPBD_OPT_BATCH_VARIANT 4
/* Failure-path test of the bounded waits (value != 0; default 0): the
 * pair kernels of the handle (one-direction, symmetric, packed symmetric --
 * the last also as batched variant 4; not the persistent batched tiles of
 * variants 0-3) leave the barrier of their first source stage without a
 * copy and wait on it for about 0.1 ms instead of ~2 s, so the wait runs out:
 * the kernel records the timeout, lets its other copies land and exits, and
 * the synchronising calls (Lanczos, GMRES, steps, batched Lanczos with iters)
 * return RPBD_TIMEOUT.  The kernel-only calls then return garbage without a
 * status.  For tests of the error path only; set it back to 0 afterwards. */
#define RPBD_OPT_TEST_STALL 5
/* value != 0 (default 0): FP32 matvecs of one system with the wall form each
 * pair block with the direct-minus-image differences written without
 * cancellation (1/r - 1/|R| = 4 zi zj / (r |R| (r + |R|)) and the matching
 * cubic), so every block keeps FP32 relative accuracy (~1e-7) at any
 * separation; the default form loses digits in proportion to
 * |R|^2 / (zi zj) (~1e-3 relative for a block 700 a away), which the matvec's
 * rows do not show because such blocks are tiny.  Runs the packed symmetric
 * kernel for every k (groups of up to four right-hand sides), 5-12%
 * slower per launch; RPBD_BAD_ARG when packing is off.  Batched and adjoint
 * calls keep the default form. */
#define RPBD_OPT_FARFIELD 6
/* value != 0 (default 0): the FP32 matvec of a single system keeps partial
 * sums reduced in a fixed order: the packed symmetric kernel one FP32 visitor
 * partial per (256-blob home tile, blob) (memory about n^2 / 256 * 3k floats;
 * past 16 GiB the option is ignored), the one-direction kernel one per
 * (2048-source chunk, blob) (n^2 / 2048 * 3k floats).  By default both
 * accumulate in fixed point instead: every contribution to a blob's velocity
 * (a tile's or a chunk's FP32 sum) is scaled by 2^S, rounded to a 64-bit
 * integer and added atomically, one accumulator per blob and component
 * (memory 3k n integers; S from the largest |force|, so that no sum can
 * overflow; the rounding step is at most 2^-60 of the largest possible sum,
 * 4 n max|F| in units of 1 / (8 pi eta a), x 9 in the periodic cell; any
 * finite FP32 forces).  Integer addition does not depend on its order, so
 * both are deterministic; they differ by FP32 output rounding.  Batches on
 * the packed symmetric kernel follow the same option (one maximum force per
 * system); the FP64 kernels and the batched one-direction tiles always keep
 * their partials. */
#define RPBD_OPT_SYM_PARTIALS 7
int rpbd_set_option(rpbd_handle* h, int option, int value);

/* Times the FP32 matvec kernels on n blobs at r (k right-hand sides, zero
 * forces): the one-direction kernel and, for k <= 4, every symmetric variant;
 * keeps the fastest in the handle for k's class (k = 1, k = 2, 3..4; other
 * classes keep their setting) and returns its index (0: one-direction,
 * 1 + v: symmetric variant v) or a negative status.  *best_ms (host, may be
 * NULL) receives its time per launch.  Synchronises the stream. */
int rpbd_autotune(rpbd_handle* h, int64_t n, const double* r, int k, double* best_ms, void* stream);

/* ---- instrumentation ----------------------------------------------------- */

/* Number of kernels this library has launched since it was loaded. */
long long rpbd_launch_count(void);
/* Measures the FMA throughput of this GPU in dtype (RPBD_F32, RPBD_F64, 2:
 * FP32 with packed two-wide FMA instructions, or 3: packed FMAs whose three
 * operands are distinct varying registers -- the form the pair kernels'
 * accumulations take, which the register file feeds more slowly):
 * one launch of independent FMA chains filling every SM, timed with CUDA
 * events on the stream; *tflops (host) receives FLOP/s / 1e12 (FMA = 2).
 * The denominator for roofline fractions of ALU-bound kernels.  Synchronises
 * the stream. */
int rpbd_measure_fma_peak(rpbd_handle* h, int dtype, double* tflops, void* stream);
/* on != 0: bracket every pair-kernel launch of h with CUDA events on its
 * stream (used to time the kernel inside a larger step). */
int rpbd_profile_enable(rpbd_handle* h, int on);
/* Sum of the recorded pair-kernel durations for (kind, k-variant), their
 * launch count and pairs (n^2 per launch); kind: RPBD_F64, RPBD_F32 (one-direction
 * kernel), 2 (batched FP32), 3 (symmetric FP32 with the assembled block, or
 * the packed kernel in a periodic cell), 4 (symmetric FP32 applying the block
 * in factored form: the packed kernel in an open cell, or the one-home kernel
 * with k <= 2).  Synchronises the device.  reset != 0 drops every record
 * afterwards. */
int rpbd_profile_read(rpbd_handle* h, int dtype, int k, double* ms, long long* launches, double* pairs,
                      int reset);

#ifdef __cplusplus
}
#endif

#endif /* RPBD_H */
