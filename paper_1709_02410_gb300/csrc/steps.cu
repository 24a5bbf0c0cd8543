// Random finite difference drift (Sec. 3) and the time integrators:
// Euler-Maruyama Traction (Algorithm 1, Sec. 3.1), Trapezoidal Slip
// (Algorithm 2, Sec. 3.2), Euler-Maruyama RFD (Algorithm 3, App. A) and the
// Trapezoidal Traction variant (Sec. 3.2).  Every saddle solve is the GMRES of krylov.cu with
// the body-block preconditioner built at the configuration it solves at; the
// Brownian slip M^{1/2} W is the preconditioned Lanczos of krylov.cu.
#include <cuda_runtime.h>

#include <cmath>

#include "rpbd_internal.cuh"

namespace rpbd {

// out = (a - b) * s, elementwise
__global__ void diff_scale_kernel(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double s,
                                  double* __restrict__ out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (a[e] - b[e]) * s;
}

// FT[p] += (0, 0, 0, torque)
__global__ void add_torque_kernel(int64_t nb, double t0, double t1, double t2, double* __restrict__ FT)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nb) return;
    FT[6 * p + 3] += t0;
    FT[6 * p + 4] += t1;
    FT[6 * p + 5] += t2;
}

// EM-T random body vectors from rows (W^f, W^tau): W^FT = kT [W^f/L; W^tau],
// dQ = [L W^f; W^tau]
__global__ void emt_random_kernel(int64_t nb, const double* __restrict__ Wb, double kT, double L,
                                  double* __restrict__ WFT, double* __restrict__ dQ)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nb) return;
    for (int c = 0; c < 3; ++c) {
        WFT[6 * p + c] = kT * Wb[6 * p + c] / L;
        WFT[6 * p + 3 + c] = kT * Wb[6 * p + 3 + c];
        dQ[6 * p + c] = L * Wb[6 * p + c];
        dQ[6 * p + 3 + c] = Wb[6 * p + 3 + c];
    }
}

static unsigned g1(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

static int rfd_impl(rpbd_handle* h, int64_t n, const double* r, const double* W, double delta, double* drift,
                    int dtype, cudaStream_t st)
{
    double* buf;
    RPBD_TRY(ensure_t(h, BUF_R2, (size_t)12 * n, &buf));
    double* rp = buf;
    double* rm = buf + 3 * n;
    double* Up = buf + 6 * n;
    double* Um = buf + 9 * n;
    launch_axpby(3 * n, 1.0, r, 0.5 * delta, W, rp, st);
    launch_axpby(3 * n, 1.0, r, -0.5 * delta, W, rm, st);
    RPBD_TRY(mobility_apply_impl(h, n, rp, W, Up, 1, dtype, true, st));
    RPBD_TRY(mobility_apply_impl(h, n, rm, W, Um, 1, dtype, true, st));
    diff_scale_kernel<<<g1(3 * n), 256, 0, st>>>(3 * n, Up, Um, 1.0 / delta, drift); count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

// step workspace
struct StepBufs {
    double *r, *Ws, *W, *WD, *WF, *lam, *dQ, *qp, *tp, *qm, *tm, *rp, *rm, *DF, *DS, *t1, *t2, *MhW, *fb, *FT, *Un,
        *qt, *tt, *rt, *slip, *Ut, *b6a, *b6b, *Wb;
    static size_t count(int64_t n, int64_t nb) { return (size_t)(17 * 3 * n + 16 * 6 * nb + 6 * 4 * nb); }
    void carve(double* base, int64_t n, int64_t nb)
    {
        double* p = base;
        auto take = [&](int64_t c) { double* o = p; p += c; return o; };
        r = take(3 * n); Ws = take(3 * n); W = take(3 * n); WD = take(3 * n); WF = take(3 * n);
        lam = take(3 * n); rp = take(3 * n); rm = take(3 * n); DS = take(3 * n); t1 = take(3 * n);
        t2 = take(3 * n); MhW = take(3 * n); fb = take(3 * n); rt = take(3 * n); slip = take(3 * n);
        dQ = take(6 * nb); DF = take(6 * nb); FT = take(6 * nb); Un = take(6 * nb); Ut = take(6 * nb);
        b6a = take(6 * nb); b6b = take(6 * nb); Wb = take(6 * nb);
        qp = take(6 * nb); tp = take(6 * nb); qm = take(6 * nb); tm = take(6 * nb); qt = take(6 * nb);
        tt = take(6 * nb);
    }
};

static int body_forces(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const rpbd_forces& f,
                       int dtype, double* fb, double* FT, cudaStream_t st)
{
    RPBD_TRY(launch_blob_forces(h, nb * nper, nper, r, f, dtype, fb, st));
    launch_KT(nb, nper, r, q, fb, FT, st);
    add_torque_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, f.torque[0], f.torque[1], f.torque[2], FT); count_launch();
    RPBD_LAUNCH_CHECK(h);
    return RPBD_OK;
}

static int check_step_args(rpbd_handle* h, int64_t nb, int nper, const double* shape, const double* q,
                           const double* theta, const rpbd_forces* f, const rpbd_step_params* sp)
{
    if (nb <= 0 || nper <= 0 || !shape || !q || !theta || !f || !sp)
        return set_error(h, RPBD_BAD_ARG, "step: bad arguments");
    if (!(sp->dt > 0) || !(sp->delta > 0) || !(sp->Lp > 0) || !(sp->tol_gmres > 0) || !(sp->tol_lanczos > 0))
        return set_error(h, RPBD_BAD_ARG, "step: dt, delta, Lp and tolerances must be > 0");
    if (sp->dtype != RPBD_F32 && sp->dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "step: bad dtype");
    if (f->steric_gamma != 0.0 && (!(f->steric_b > 0) || !(f->r_floor > 0)))
        return set_error(h, RPBD_BAD_ARG, "step: steric forces need steric_b > 0 and r_floor > 0");
    return RPBD_OK;
}

// Saddle solve of a step.  warm_from (when not null and warm starts are on)
// holds the body velocities of an earlier solve whose blob tractions are
// still in lam; that solution is the initial guess.
static int solve(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* slip,
                 const double* FT, double* lam, double* U, const rpbd_step_params* sp, int build, rpbd_stats* stt,
                 cudaStream_t st, const double* warm_from = nullptr)
{
    const int warm = (warm_from && !sp->cold_start) ? 1 : 0;
    if (warm && warm_from != U)
        RPBD_CU(h, cudaMemcpyAsync(U, warm_from, sizeof(double) * 6 * nb, cudaMemcpyDeviceToDevice, st));
    int s = gmres_impl(h, nb, nper, r, q, slip, FT, lam, U, sp->tol_gmres, sp->max_iter_gmres, sp->restart, sp->dtype,
                       build, warm, stt, st);
    return (s == RPBD_NOT_CONVERGED) ? RPBD_OK : s;  // reported through stats
}

// Two saddle solves at the same positions, preconditioner already built;
// their GMRES iterations run in lockstep and share two-RHS matvecs.
static int solve_pair(rpbd_handle* h, int64_t nb, int nper, const double* r, const double* q, const double* slip0,
                      const double* FT0, double* lam0, double* U0, const double* slip1, const double* FT1,
                      double* lam1, double* U1, const rpbd_step_params* sp, rpbd_stats* st0, rpbd_stats* st1,
                      cudaStream_t st)
{
    const GmresProblem pb[2] = {{slip0, FT0, lam0, U0, sp->tol_gmres, sp->max_iter_gmres, 0},
                                {slip1, FT1, lam1, U1, sp->tol_gmres, sp->max_iter_gmres, 0}};
    rpbd_stats s2[2] = {};
    int s = gmres_multi_impl(h, nb, nper, r, q, 2, pb, sp->restart, sp->dtype, 0, s2, st);
    *st0 = s2[0];
    *st1 = s2[1];
    return (s == RPBD_NOT_CONVERGED) ? RPBD_OK : s;  // reported through stats
}

int step_ts_impl(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                 const rpbd_forces* f, const rpbd_step_params* sp, rpbd_stats* stats, cudaStream_t st)
{
    RPBD_TRY(check_step_args(h, nb, nper, shape, q, theta, f, sp));
    const int64_t n = nb * nper;
    double* base;
    RPBD_TRY(ensure_t(h, BUF_STEP, StepBufs::count(n, nb), &base));
    StepBufs B;
    B.carve(base, n, nb);
    const double kT = h->p.kT, d = sp->delta, L = sp->Lp;
    const double c = std::sqrt(2.0 * kT / sp->dt);
    rpbd_stats dummy[4];
    rpbd_stats* S = stats ? stats : dummy;
    launch_blobs(nb, nper, shape, q, theta, B.r, st);
    RPBD_TRY(check_finite(h, 3 * n, B.r, st));
    // 1a: W^s, W^D = L W^s, W^F = kT/L W^s
    launch_normals(sp->seed, sp->step, 0, 3 * n, B.Ws, st);
    launch_normals(sp->seed, sp->step, 1, 3 * n, B.W, st);
    launch_scale_copy(3 * n, L, B.Ws, B.WD, st);
    launch_scale_copy(3 * n, kT / L, B.Ws, B.WF, st);
    // the preconditioner at Q^n serves the RFD solve, Lanczos and the predictor
    RPBD_TRY(precond_build_impl(h, nb, nper, B.r, q, st));
    // 2: M^{1/2} W
    {
        int s = lanczos_impl(h, n, B.r, B.W, B.MhW, sp->tol_lanczos, sp->max_iter_lanczos, sp->dtype, 1, &S[1], st);
        if (s != RPBD_OK && s != RPBD_NOT_CONVERGED) return s;
    }
    // 3 (right-hand side): slip c M^{1/2} W, force F^n
    RPBD_TRY(body_forces(h, nb, nper, B.r, q, *f, sp->dtype, B.fb, B.FT, st));
    launch_scale_copy(3 * n, c, B.MhW, B.slip, st);
    // 1b and 3: the RFD displacement problem (slip W^D, no force) and the
    // predictor share M^n, so they are solved together (two-RHS matvecs)
    RPBD_TRY(solve_pair(h, nb, nper, B.r, q, B.WD, nullptr, B.t2, B.dQ, B.slip, B.FT, B.lam, B.Un, sp, &S[0],
                        &S[2], st));
    // 1c: Q+- = Q +- delta/2 dQ
    launch_advance(nb, q, theta, B.dQ, 0.5 * d, B.qp, B.tp, st);
    launch_advance(nb, q, theta, B.dQ, -0.5 * d, B.qm, B.tm, st);
    launch_blobs(nb, nper, shape, B.qp, B.tp, B.rp, st);
    launch_blobs(nb, nper, shape, B.qm, B.tm, B.rm, st);
    // 1d: D^F = (K^T(Q+) - K^T(Q-)) W^F / delta ; D^S = (M(Q+) - M(Q-)) W^F / delta
    launch_KT(nb, nper, B.rp, B.qp, B.WF, B.b6a, st);
    launch_KT(nb, nper, B.rm, B.qm, B.WF, B.b6b, st);
    diff_scale_kernel<<<g1(6 * nb), 256, 0, st>>>(6 * nb, B.b6a, B.b6b, 1.0 / d, B.DF); count_launch();
    RPBD_TRY(mobility_apply_impl(h, n, B.rp, B.WF, B.t1, 1, sp->dtype, true, st));
    RPBD_TRY(mobility_apply_impl(h, n, B.rm, B.WF, B.t2, 1, sp->dtype, true, st));
    diff_scale_kernel<<<g1(3 * n), 256, 0, st>>>(3 * n, B.t1, B.t2, 1.0 / d, B.DS); count_launch();
    RPBD_LAUNCH_CHECK(h);
    // 4: Q~ = Q^n + dt U^n
    launch_advance(nb, q, theta, B.Un, sp->dt, B.qt, B.tt, st);
    launch_blobs(nb, nper, shape, B.qt, B.tt, B.rt, st);
    // 5: corrector at Q~: slip 2 D^S + c M^{1/2} W, force F~ - 2 D^F
    RPBD_TRY(body_forces(h, nb, nper, B.rt, B.qt, *f, sp->dtype, B.fb, B.FT, st));
    launch_axpby(6 * nb, 1.0, B.FT, -2.0, B.DF, B.FT, st);
    launch_axpby(3 * n, 2.0, B.DS, c, B.MhW, B.slip, st);
    RPBD_TRY(solve(h, nb, nper, B.rt, B.qt, B.slip, B.FT, B.lam, B.Ut, sp, 1, &S[3], st, B.Un));
    // 6: Q^{n+1} = Q^n + dt/2 (U^n + U~)
    launch_axpby(6 * nb, 0.5, B.Un, 0.5, B.Ut, B.b6a, st);
    launch_advance(nb, q, theta, B.b6a, sp->dt, q, theta, st);
    RPBD_LAUNCH_CHECK(h);
    for (int i = 0; i < 4; ++i)
        if (S[i].status != RPBD_OK) return RPBD_NOT_CONVERGED;
    return RPBD_OK;
}

int step_emt_impl(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                  const rpbd_forces* f, const rpbd_step_params* sp, rpbd_stats* stats, cudaStream_t st)
{
    RPBD_TRY(check_step_args(h, nb, nper, shape, q, theta, f, sp));
    const int64_t n = nb * nper;
    double* base;
    RPBD_TRY(ensure_t(h, BUF_STEP, StepBufs::count(n, nb), &base));
    StepBufs B;
    B.carve(base, n, nb);
    const double kT = h->p.kT, d = sp->delta, L = sp->Lp;
    const double c = std::sqrt(2.0 * kT / sp->dt);
    rpbd_stats dummy[3];
    rpbd_stats* S = stats ? stats : dummy;
    launch_blobs(nb, nper, shape, q, theta, B.r, st);
    RPBD_TRY(check_finite(h, 3 * n, B.r, st));
    // 1a: W^FT = kT [W^f / L; W^tau], dQ = [L W^f; W^tau]
    launch_normals(sp->seed, sp->step, 2, 6 * nb, B.Wb, st);
    launch_normals(sp->seed, sp->step, 1, 3 * n, B.W, st);
    emt_random_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, B.Wb, kT, L, B.b6a, B.dQ); count_launch();
    RPBD_LAUNCH_CHECK(h);
    // 1b: RFD mobility problem, force W^FT, no slip
    RPBD_TRY(solve(h, nb, nper, B.r, q, nullptr, B.b6a, B.lam, B.Un, sp, 1, &S[0], st));
    // 1c: Q+- = Q +- delta/2 dQ
    launch_advance(nb, q, theta, B.dQ, 0.5 * d, B.qp, B.tp, st);
    launch_advance(nb, q, theta, B.dQ, -0.5 * d, B.qm, B.tm, st);
    launch_blobs(nb, nper, shape, B.qp, B.tp, B.rp, st);
    launch_blobs(nb, nper, shape, B.qm, B.tm, B.rm, st);
    // 1d: D^F = (K^T(Q+) - K^T(Q-)) lam^RFD / delta
    launch_KT(nb, nper, B.rp, B.qp, B.lam, B.b6a, st);
    launch_KT(nb, nper, B.rm, B.qm, B.lam, B.b6b, st);
    diff_scale_kernel<<<g1(6 * nb), 256, 0, st>>>(6 * nb, B.b6a, B.b6b, 1.0 / d, B.DF); count_launch();
    //     D^S = [(M(Q+) - M(Q-)) lam^RFD - (K(Q+) - K(Q-)) U^RFD] / delta
    RPBD_TRY(mobility_apply_impl(h, n, B.rp, B.lam, B.t1, 1, sp->dtype, true, st));
    RPBD_TRY(mobility_apply_impl(h, n, B.rm, B.lam, B.t2, 1, sp->dtype, true, st));
    diff_scale_kernel<<<g1(3 * n), 256, 0, st>>>(3 * n, B.t1, B.t2, 1.0 / d, B.DS); count_launch();
    launch_K(nb, nper, B.rp, B.qp, B.Un, B.t1, st);
    launch_K(nb, nper, B.rm, B.qm, B.Un, B.t2, st);
    diff_scale_kernel<<<g1(3 * n), 256, 0, st>>>(3 * n, B.t1, B.t2, 1.0 / d, B.fb); count_launch();
    launch_axpby(3 * n, 1.0, B.DS, -1.0, B.fb, B.DS, st);
    RPBD_LAUNCH_CHECK(h);
    // 2: M^{1/2} W
    {
        int s = lanczos_impl(h, n, B.r, B.W, B.MhW, sp->tol_lanczos, sp->max_iter_lanczos, sp->dtype, 1, &S[1], st);
        if (s != RPBD_OK && s != RPBD_NOT_CONVERGED) return s;
    }
    // 3: slip D^S + c M^{1/2} W, force F^n - D^F
    RPBD_TRY(body_forces(h, nb, nper, B.r, q, *f, sp->dtype, B.fb, B.FT, st));
    launch_axpby(6 * nb, 1.0, B.FT, -1.0, B.DF, B.FT, st);
    launch_axpby(3 * n, 1.0, B.DS, c, B.MhW, B.slip, st);
    RPBD_TRY(solve(h, nb, nper, B.r, q, B.slip, B.FT, B.lam, B.Un, sp, 0, &S[2], st));
    // 4: Q^{n+1} = Q^n + dt U^n
    launch_advance(nb, q, theta, B.Un, sp->dt, q, theta, st);
    RPBD_LAUNCH_CHECK(h);
    for (int i = 0; i < 3; ++i)
        if (S[i].status != RPBD_OK) return RPBD_NOT_CONVERGED;
    return RPBD_OK;
}

int step_emrfd_impl(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                    const rpbd_forces* f, const rpbd_step_params* sp, rpbd_stats* stats, cudaStream_t st)
{
    RPBD_TRY(check_step_args(h, nb, nper, shape, q, theta, f, sp));
    const int64_t n = nb * nper;
    double* base;
    RPBD_TRY(ensure_t(h, BUF_STEP, StepBufs::count(n, nb), &base));
    StepBufs B;
    B.carve(base, n, nb);
    const double kT = h->p.kT, d = sp->delta, L = sp->Lp;
    const double c = std::sqrt(2.0 * kT / sp->dt);
    rpbd_stats dummy[4];
    rpbd_stats* S = stats ? stats : dummy;
    launch_blobs(nb, nper, shape, q, theta, B.r, st);
    RPBD_TRY(check_finite(h, 3 * n, B.r, st));
    // 1a: W^FT = kT [W^f / L; W^tau], dQ = [L W^f; W^tau]
    launch_normals(sp->seed, sp->step, 2, 6 * nb, B.Wb, st);
    launch_normals(sp->seed, sp->step, 1, 3 * n, B.W, st);
    emt_random_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, B.Wb, kT, L, B.b6a, B.dQ);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    // 1b: Q+- = Q +- delta/2 dQ
    launch_advance(nb, q, theta, B.dQ, 0.5 * d, B.qp, B.tp, st);
    launch_advance(nb, q, theta, B.dQ, -0.5 * d, B.qm, B.tm, st);
    launch_blobs(nb, nper, shape, B.qp, B.tp, B.rp, st);
    launch_blobs(nb, nper, shape, B.qm, B.tm, B.rm, st);
    // 1c: mobility problems with force W^FT at Q+ and Q- (preconditioner built at each)
    RPBD_TRY(solve(h, nb, nper, B.rp, B.qp, nullptr, B.b6a, B.lam, B.Ut, sp, 1, &S[0], st));
    RPBD_TRY(solve(h, nb, nper, B.rm, B.qm, nullptr, B.b6a, B.lam, B.b6b, sp, 1, &S[1], st, B.Ut));
    // (U+ - U-) / delta
    diff_scale_kernel<<<g1(6 * nb), 256, 0, st>>>(6 * nb, B.Ut, B.b6b, 1.0 / d, B.DF);
    count_launch();
    // 2: M^{1/2} W at Q^n
    RPBD_TRY(precond_build_impl(h, nb, nper, B.r, q, st));
    {
        int s = lanczos_impl(h, n, B.r, B.W, B.MhW, sp->tol_lanczos, sp->max_iter_lanczos, sp->dtype, 1, &S[2], st);
        if (s != RPBD_OK && s != RPBD_NOT_CONVERGED) return s;
    }
    // 3: slip c M^{1/2} W, force F^n
    RPBD_TRY(body_forces(h, nb, nper, B.r, q, *f, sp->dtype, B.fb, B.FT, st));
    launch_scale_copy(3 * n, c, B.MhW, B.slip, st);
    RPBD_TRY(solve(h, nb, nper, B.r, q, B.slip, B.FT, B.lam, B.Un, sp, 0, &S[3], st));
    // 4: Q^{n+1} = Q^n + dt (U^n + (U+ - U-) / delta)
    launch_axpby(6 * nb, 1.0, B.Un, 1.0, B.DF, B.b6a, st);
    launch_advance(nb, q, theta, B.b6a, sp->dt, q, theta, st);
    RPBD_LAUNCH_CHECK(h);
    for (int i = 0; i < 4; ++i)
        if (S[i].status != RPBD_OK) return RPBD_NOT_CONVERGED;
    return RPBD_OK;
}

int step_tt_impl(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                 const rpbd_forces* f, const rpbd_step_params* sp, rpbd_stats* stats, cudaStream_t st)
{
    RPBD_TRY(check_step_args(h, nb, nper, shape, q, theta, f, sp));
    const int64_t n = nb * nper;
    double* base;
    RPBD_TRY(ensure_t(h, BUF_STEP, StepBufs::count(n, nb), &base));
    StepBufs B;
    B.carve(base, n, nb);
    const double kT = h->p.kT, d = sp->delta, L = sp->Lp;
    const double c = std::sqrt(2.0 * kT / sp->dt);
    rpbd_stats dummy[4];
    rpbd_stats* S = stats ? stats : dummy;
    launch_blobs(nb, nper, shape, q, theta, B.r, st);
    RPBD_TRY(check_finite(h, 3 * n, B.r, st));
    // traction RFD as in step 1 of Algorithm 1
    launch_normals(sp->seed, sp->step, 2, 6 * nb, B.Wb, st);
    launch_normals(sp->seed, sp->step, 1, 3 * n, B.W, st);
    emt_random_kernel<<<(unsigned)((nb + 127) / 128), 128, 0, st>>>(nb, B.Wb, kT, L, B.b6a, B.dQ);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    // the preconditioner at Q^n serves the RFD solve, Lanczos and the predictor
    RPBD_TRY(precond_build_impl(h, nb, nper, B.r, q, st));
    {
        int s = lanczos_impl(h, n, B.r, B.W, B.MhW, sp->tol_lanczos, sp->max_iter_lanczos, sp->dtype, 1, &S[1], st);
        if (s != RPBD_OK && s != RPBD_NOT_CONVERGED) return s;
    }
    // predictor right-hand side, as step 3 of Algorithm 2
    RPBD_TRY(body_forces(h, nb, nper, B.r, q, *f, sp->dtype, B.fb, B.FT, st));
    launch_scale_copy(3 * n, c, B.MhW, B.slip, st);
    // the traction RFD problem (force W^FT, no slip; lambda^RFD -> WD, U^RFD
    // unused) and the predictor share M^n: solved together
    RPBD_TRY(solve_pair(h, nb, nper, B.r, q, nullptr, B.b6a, B.WD, B.Ut, B.slip, B.FT, B.lam, B.Un, sp, &S[0],
                        &S[2], st));
    launch_advance(nb, q, theta, B.dQ, 0.5 * d, B.qp, B.tp, st);
    launch_advance(nb, q, theta, B.dQ, -0.5 * d, B.qm, B.tm, st);
    launch_blobs(nb, nper, shape, B.qp, B.tp, B.rp, st);
    launch_blobs(nb, nper, shape, B.qm, B.tm, B.rm, st);
    // D^F and D^S without the U^RFD term (the trapezoidal corrector supplies it)
    launch_KT(nb, nper, B.rp, B.qp, B.WD, B.b6a, st);
    launch_KT(nb, nper, B.rm, B.qm, B.WD, B.b6b, st);
    diff_scale_kernel<<<g1(6 * nb), 256, 0, st>>>(6 * nb, B.b6a, B.b6b, 1.0 / d, B.DF);
    count_launch();
    RPBD_TRY(mobility_apply_impl(h, n, B.rp, B.WD, B.t1, 1, sp->dtype, true, st));
    RPBD_TRY(mobility_apply_impl(h, n, B.rm, B.WD, B.t2, 1, sp->dtype, true, st));
    diff_scale_kernel<<<g1(3 * n), 256, 0, st>>>(3 * n, B.t1, B.t2, 1.0 / d, B.DS);
    count_launch();
    RPBD_LAUNCH_CHECK(h);
    launch_advance(nb, q, theta, B.Un, sp->dt, B.qt, B.tt, st);
    launch_blobs(nb, nper, shape, B.qt, B.tt, B.rt, st);
    // corrector at Q~ with 2 D^S and 2 D^F
    RPBD_TRY(body_forces(h, nb, nper, B.rt, B.qt, *f, sp->dtype, B.fb, B.FT, st));
    launch_axpby(6 * nb, 1.0, B.FT, -2.0, B.DF, B.FT, st);
    launch_axpby(3 * n, 2.0, B.DS, c, B.MhW, B.slip, st);
    RPBD_TRY(solve(h, nb, nper, B.rt, B.qt, B.slip, B.FT, B.lam, B.Ut, sp, 1, &S[3], st, B.Un));
    launch_axpby(6 * nb, 0.5, B.Un, 0.5, B.Ut, B.b6a, st);
    launch_advance(nb, q, theta, B.b6a, sp->dt, q, theta, st);
    RPBD_LAUNCH_CHECK(h);
    for (int i = 0; i < 4; ++i)
        if (S[i].status != RPBD_OK) return RPBD_NOT_CONVERGED;
    return RPBD_OK;
}

}  // namespace rpbd

using namespace rpbd;

extern "C" {

int rpbd_rfd_drift(rpbd_handle* h, int64_t n, const double* r, const double* W, double delta, double* drift, int dtype,
                   void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    if (n < 0 || (n > 0 && (!r || !W || !drift)) || !(delta > 0))
        return set_error(h, RPBD_BAD_ARG, "rfd_drift: bad arguments");
    if (dtype != RPBD_F32 && dtype != RPBD_F64) return set_error(h, RPBD_BAD_ARG, "rfd_drift: bad dtype");
    if (n == 0) return RPBD_OK;
    return rfd_impl(h, n, r, W, delta, drift, dtype, reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_step_ts(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                 const rpbd_forces* forces, const rpbd_step_params* sp, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    return step_ts_impl(h, nb, nper, shape, q, theta, forces, sp, stats, reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_step_emt(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                  const rpbd_forces* forces, const rpbd_step_params* sp, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    return step_emt_impl(h, nb, nper, shape, q, theta, forces, sp, stats, reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_step_emrfd(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                    const rpbd_forces* forces, const rpbd_step_params* sp, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    return step_emrfd_impl(h, nb, nper, shape, q, theta, forces, sp, stats, reinterpret_cast<cudaStream_t>(stream));
}

int rpbd_step_tt(rpbd_handle* h, int64_t nb, int nper, const double* shape, double* q, double* theta,
                 const rpbd_forces* forces, const rpbd_step_params* sp, rpbd_stats* stats, void* stream)
{
    if (!h) return RPBD_BAD_ARG;
    return step_tt_impl(h, nb, nper, shape, q, theta, forces, sp, stats, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
