"""GPU parity of the block preconditioner, Lanczos M^{1/2} W, GMRES saddle
solve, RFD drift, adjoint and divergence against the oracle."""
import numpy as np
import pytest
import scipy.linalg
import torch

from oracle import krylov, mobility as om, precond, rfd, saddle
from paper_1709_02410_gb300 import RpbdError, F32, F64, synth

from gpu_util import handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def small(nb=8, seed=3, box=8.0, lift=True):
    return synth.boomerang_suspension(nb, box, seed, lift=lift)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_precond_apply_modes(mode):
    s = small(12, 4)
    r = positions(s)
    pc = precond.BlockPrecond(r, s.q, s.nper, oracle_params(s))
    x = np.random.default_rng(mode).standard_normal((3, s.n))
    ref = [pc.L_apply, pc.Linv_apply, pc.LinvT_apply,
           lambda v: om.blob_to_soa(np.concatenate([pc.Minv[p] @ om.soa_to_blob(v).reshape(s.nb, -1)[p]
                                                    for p in range(s.nb)]))][mode](x)
    h = handle_for(s)
    h.precond_build(s.nper, to_dev(r), to_dev(s.q))
    out = h.precond_apply(mode, to_dev(x)).cpu().numpy()
    assert rel2(out, ref) <= 1e-11


def test_lanczos_preconditioned_matches_dense():
    s = small(8, 5)
    r = positions(s)
    prm = oracle_params(s)
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    M = om.dense(r, prm)
    Lb = scipy.linalg.block_diag(*pc.L)
    G = np.linalg.solve(Lb, np.linalg.solve(Lb, M).T).T
    W = synth.gaussian(6, (3, s.n))
    ref = Lb @ (scipy.linalg.sqrtm(0.5 * (G + G.T)).real @ om.soa_to_blob(W))
    h = handle_for(s)
    h.precond_build(s.nper, to_dev(r), to_dev(s.q))
    out, st = h.lanczos_sqrt_apply(to_dev(r), to_dev(W), tol=1e-12, max_iter=80)
    assert st["status"] == 0
    assert rel2(om.soa_to_blob(out.cpu().numpy()), ref) <= 1e-9


def test_lanczos_matches_oracle_iterates():
    """same tolerance, same stop rule: same iteration count and answer"""
    s = small(10, 7)
    r = positions(s)
    prm = oracle_params(s)
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    W = synth.gaussian(8, (3, s.n))
    G = lambda v: pc.Linv_apply(om.apply(r, pc.LinvT_apply(v), prm))
    y, it, ch = krylov.lanczos_sqrt(G, W, 1e-4, 80)
    ref = pc.L_apply(y)
    h = handle_for(s)
    h.precond_build(s.nper, to_dev(r), to_dev(s.q))
    out, st = h.lanczos_sqrt_apply(to_dev(r), to_dev(W), tol=1e-4, max_iter=80)
    assert abs(st["iterations"] - it) <= 1
    assert rel2(out.cpu().numpy(), ref) <= 1e-4


def test_lanczos_1920_fixed_iterations_matches_oracle():
    """1,920 boomerang blobs: with the iteration count pinned on both sides
    (20 iterations, a tolerance neither side reaches) the FP64 Lanczos of the
    library and of the oracle build the same Krylov space and differ only by
    rounding: <= 1e-12."""
    s = synth.boomerangs_1920()
    r = positions(s)
    prm = oracle_params(s)
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    W = synth.gaussian(9, (3, s.n))
    G = lambda v: pc.Linv_apply(om.apply(r, pc.LinvT_apply(v), prm))
    y, it, ch = krylov.lanczos_sqrt(G, W, 0.0, 20)
    assert it == 20
    h = handle_for(s)
    h.precond_build(s.nper, to_dev(r), to_dev(s.q))
    out, st = h.lanczos_sqrt_apply(to_dev(r), to_dev(W), tol=1e-300, max_iter=20)
    assert st["status"] == -4 and st["iterations"] == 20
    assert rel2(out.cpu().numpy(), pc.L_apply(y)) <= 1e-12


@pytest.mark.parametrize("dtype,tol,bound", [(F64, 1e-10, 1e-9), (F32, 1e-5, 1e-4)])
@pytest.mark.parametrize("nw", [2, 3, 4])
def test_lanczos_multi_matches_single(dtype, tol, bound, nw):
    """Lockstep Lanczos (shared multi-RHS matvecs): each W gets the answer
    and iteration count of its own run; one W = 0 gives zero."""
    s = small(8, 41)
    r = positions(s)
    h = handle_for(s)
    rd = to_dev(r)
    h.precond_build(s.nper, rd, to_dev(s.q))
    rng = np.random.default_rng(42)
    Ws = [rng.standard_normal((3, s.n)) for _ in range(nw)]
    Ws[-1] = np.zeros((3, s.n)) if nw == 3 else Ws[-1]
    out = h.lanczos_sqrt_apply_multi(rd, [to_dev(w) for w in Ws], tol=tol, max_iter=60, dtype=dtype)
    for w, (y, st) in zip(Ws, out):
        y1, st1 = h.lanczos_sqrt_apply(rd, to_dev(w), tol=tol, max_iter=60, dtype=dtype)
        if not np.any(w):
            assert float(y.abs().max()) == 0.0 and st["iterations"] == 0
            continue
        assert st["status"] == 0
        assert abs(st["iterations"] - st1["iterations"]) <= (0 if dtype == F64 else 1)
        assert rel2(y.cpu().numpy(), y1.cpu().numpy()) <= bound


def test_lanczos_unpreconditioned():
    s = small(4, 9)
    r = positions(s)
    M = om.dense(r, oracle_params(s))
    W = synth.gaussian(10, (3, s.n))
    ref = scipy.linalg.sqrtm(M).real @ om.soa_to_blob(W)
    h = handle_for(s)
    out, st = h.lanczos_sqrt_apply(to_dev(r), to_dev(W), tol=1e-11, max_iter=80, use_precond=False)
    assert rel2(om.soa_to_blob(out.cpu().numpy()), ref) <= 1e-8


@pytest.mark.parametrize("dtype,tol,bound", [(F64, 1e-12, 1e-9), (F32, 1e-6, 1e-4)])
def test_gmres_matches_dense_schur(dtype, tol, bound):
    s = small(8, 11)
    r = positions(s)
    rng = np.random.default_rng(12)
    slip = rng.standard_normal((3, s.n))
    FT = rng.standard_normal((s.nb, 6)) * 1e-2
    lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), slip, FT)
    h = handle_for(s)
    lam, U, st = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), to_dev(slip), to_dev(FT), tol=tol,
                                     max_iter=200, restart=30, dtype=dtype)
    assert st["status"] == 0
    assert rel2(U.cpu().numpy(), U_d) <= bound
    assert rel2(lam.cpu().numpy(), lam_d) <= 10 * bound


def test_gmres_restarts_and_null_inputs():
    s = small(6, 13)
    r = positions(s)
    FT = np.random.default_rng(14).standard_normal((s.nb, 6)) * 1e-2
    lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), None, FT)
    h = handle_for(s)
    lam, U, st = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), None, to_dev(FT), tol=1e-12, restart=4,
                                     max_iter=400)
    assert st["status"] == 0
    assert rel2(U.cpu().numpy(), U_d) <= 1e-9
    # zero right-hand side gives zero
    lam0, U0, st0 = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), None, None, tol=1e-8)
    assert float(U0.abs().max()) == 0.0 and st0["iterations"] == 0


def test_gmres_warm_start():
    """Initial guess x0: the stopping test stays relative to |b|, so a start at
    the converged answer takes no iteration, a start near it takes fewer than
    a cold start, and the answers agree with the dense Schur solution."""
    s = small(8, 21)
    r = positions(s)
    rng = np.random.default_rng(22)
    slip = rng.standard_normal((3, s.n))
    FT = rng.standard_normal((s.nb, 6)) * 1e-2
    lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), slip, FT)
    h = handle_for(s)
    args = (s.nper, to_dev(r), to_dev(s.q), to_dev(slip), to_dev(FT))
    lam, U, st = h.gmres_rigid_solve(*args, tol=1e-10, max_iter=200, restart=30)
    assert st["status"] == 0 and rel2(U.cpu().numpy(), U_d) <= 1e-8
    # start at the answer: converged before the first iteration, x0 unchanged
    lam1, U1, st1 = h.gmres_rigid_solve(*args, tol=1e-8, max_iter=200, restart=30, x0=(lam, U))
    assert st1["status"] == 0 and st1["iterations"] == 0
    assert float((U1 - U).abs().max()) == 0.0
    # start near the answer (1e-4 perturbation): fewer iterations, same answer
    p_lam = lam * (1 + 1e-4 * to_dev(rng.standard_normal(lam.shape)))
    p_U = U * (1 + 1e-4 * to_dev(rng.standard_normal(U.shape)))
    lam2, U2, st2 = h.gmres_rigid_solve(*args, tol=1e-10, max_iter=200, restart=30, x0=(p_lam, p_U))
    assert st2["status"] == 0 and st2["iterations"] < st["iterations"]
    assert rel2(U2.cpu().numpy(), U_d) <= 1e-8
    assert rel2(lam2.cpu().numpy(), lam_d) <= 1e-7
    # a zero right-hand side still gives zero, whatever x0
    lam3, U3, st3 = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), None, None, tol=1e-8, x0=(lam, U))
    assert float(U3.abs().max()) == 0.0 and float(lam3.abs().max()) == 0.0


@pytest.mark.parametrize("dtype,tol,bound", [(F64, 1e-12, 1e-9), (F32, 1e-6, 1e-4)])
@pytest.mark.parametrize("restart", [6, 60])
def test_gmres_multi_matches_single_solves(dtype, tol, bound, restart):
    """Lockstep GMRES (shared multi-RHS matvecs) gives each problem the
    answer of its own solve: three problems (slip + force, force only, slip
    only), also with restarts every 6 iterations (GMRES(4) stalls on the
    force-only problem, in the oracle as well)."""
    s = small(8, 31)
    r = positions(s)
    rng = np.random.default_rng(32)
    slip = rng.standard_normal((3, s.n))
    slip2 = rng.standard_normal((3, s.n))
    FT = rng.standard_normal((s.nb, 6)) * 1e-2
    FT2 = rng.standard_normal((s.nb, 6)) * 1e-2
    probs = [(slip, FT), (None, FT2), (slip2, None)]
    h = handle_for(s)
    dev = lambda x: None if x is None else to_dev(x)
    out = h.gmres_rigid_solve_multi(s.nper, to_dev(r), to_dev(s.q), [(dev(a), dev(b)) for a, b in probs], tol=tol,
                                    max_iter=400, restart=restart, dtype=dtype)
    for (a, b), (lam, U, st) in zip(probs, out):
        assert st["status"] == 0, st
        lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), a, b)
        assert rel2(U.cpu().numpy(), U_d) <= bound
        assert rel2(lam.cpu().numpy(), lam_d) <= 10 * bound
        lam1, U1, st1 = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), dev(a), dev(b), tol=tol, max_iter=400,
                                            restart=restart, dtype=dtype)
        # same Krylov process: same iteration count up to rounding of the shared launch
        assert abs(st1["iterations"] - st["iterations"]) <= (1 if dtype == F64 else 2)


def test_gmres_multi_zero_problem_and_limits():
    s = small(6, 33)
    r = positions(s)
    FT = np.random.default_rng(34).standard_normal((s.nb, 6)) * 1e-2
    h = handle_for(s)
    out = h.gmres_rigid_solve_multi(s.nper, to_dev(r), to_dev(s.q), [(None, None), (None, to_dev(FT))], tol=1e-10,
                                    max_iter=300, restart=40)
    (lam0, U0, st0), (lam1, U1, st1) = out
    assert st0["status"] == 0 and st0["iterations"] == 0 and float(U0.abs().max()) == 0.0
    assert st1["status"] == 0 and st1["iterations"] > 0
    with pytest.raises(RpbdError):
        h.gmres_rigid_solve_multi(s.nper, to_dev(r), to_dev(s.q), [(None, to_dev(FT))] * 5)


def test_gmres_not_converged_reports_status():
    s = small(8, 15)
    r = positions(s)
    slip = np.random.default_rng(16).standard_normal((3, s.n))
    h = handle_for(s)
    lam, U, st = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), to_dev(slip), None, tol=1e-14, max_iter=2)
    assert st["status"] == -4 and st["iterations"] == 2


@pytest.mark.parametrize("dtype,delta,bound", [(F64, 1e-6, 1e-9), (F32, 1e-3, 2e-3)])
def test_rfd_drift_matches_oracle(dtype, delta, bound):
    s = synth.boomerangs_1920()
    r = positions(s)
    W = synth.gaussian(17, (3, s.n))
    ref = rfd.rfd_drift(r, W, delta, oracle_params(s))
    h = handle_for(s)
    out = h.rfd_drift(to_dev(r), to_dev(W), delta, dtype=dtype).cpu().numpy()
    assert rel2(out, ref) <= bound


@pytest.mark.parametrize("lift", [True, False])
def test_adjoint_matches_oracle_gradient(lift):
    s = synth.boomerang_suspension(40, 10.0, 18, lift=lift)
    r = positions(s)
    rng = np.random.default_rng(19)
    u, F = rng.standard_normal((2, 3, s.n))
    h = handle_for(s)
    g = h.mobility_adjoint(to_dev(r), to_dev(u), to_dev(F)).cpu().numpy()
    go = om.grad(r, u, F, oracle_params(s))
    assert rel2(g, go) <= 1e-11


def test_divergence_matches_oracle():
    s = synth.boomerang_suspension(30, 8.0, 20, lift=False)
    r = positions(s)
    h = handle_for(s)
    d = h.mobility_divergence(to_dev(r)).cpu().numpy()
    assert rel2(d, om.divergence(r, oracle_params(s))) <= 1e-11


def test_adjoint_16380_sampled_and_fd():
    """16,380 blobs: oracle gradient on sampled blobs, plus central
    differences of the GPU matvec itself (h = 1e-6 a) on 64 coordinates."""
    s = synth.blobs_16384()
    r = positions(s)
    rng = np.random.default_rng(21)
    u, F = rng.standard_normal((2, 3, s.n))
    h = handle_for(s)
    rd, ud, Fd = to_dev(r), to_dev(u), to_dev(F)
    g = h.mobility_adjoint(rd, ud, Fd).cpu().numpy()
    rows = rng.choice(s.n, 24, replace=False)
    go = om.grad(r, u, F, oracle_params(s), rows=rows)
    assert rel2(g[:, rows], go) <= 1e-11
    hstep = 1e-6 * s.a
    coords = rng.choice(3 * s.n, 64, replace=False)
    for cidx in coords:
        c, k = divmod(int(cidx), s.n)
        rp, rm = r.copy(), r.copy()
        rp[c, k] += hstep
        rm[c, k] -= hstep
        fp = float((ud * h.mobility_apply(to_dev(rp), Fd)).sum())
        fm = float((ud * h.mobility_apply(to_dev(rm), Fd)).sum())
        fd = (fp - fm) / (2 * hstep)
        assert abs(fd - g[c, k]) <= 1e-5 * np.abs(g).max() + 1e-6 * abs(g[c, k])


def test_rfd_mean_matches_exact_divergence():
    """Sec. 3 (eq. RFDB): the mean of the blob RFD over random W is div M.
    GPU RFD samples (FP64, delta = 1e-5) against the GPU divergence kernel,
    which is itself checked against the oracle; 4,000 seeds on 60 blobs."""
    s = synth.boomerang_suspension(4, 4.0, 22, lift=False)
    r = positions(s)
    h = handle_for(s)
    rd = to_dev(r)
    div = h.mobility_divergence(rd).cpu().numpy()
    np.testing.assert_allclose(div, om.divergence(r, oracle_params(s)), rtol=1e-10, atol=1e-10 * np.abs(div).max())
    ns = 4000
    Ws = torch.randn((ns, 3, s.n), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    acc = torch.zeros((3, s.n), dtype=torch.float64, device="cuda")
    acc2 = torch.zeros_like(acc)
    for i in range(ns):
        d = h.rfd_drift(rd, Ws[i].contiguous(), 1e-5, dtype=F64)
        acc += d
        acc2 += d * d
    mean = (acc / ns).cpu().numpy()
    se = np.sqrt(np.maximum((acc2 / ns).cpu().numpy() - mean**2, 0) / ns)
    z = np.abs(mean - div) / (se + 1e-30)
    assert np.mean(z < 3) > 0.97 and z.max() < 6


@pytest.mark.parametrize("nb,box,lift", [(1, 4.0, True), (60, 12.0, False), (301, 30.0, True)])
def test_adjoint_f32_variant(nb, box, lift):
    """FP32 adjoint (hi/lo separations, FP32 sums per 2048-source chunk): one
    body, overlapping wall blobs, and 4,515 blobs (three chunks, the last
    ragged) against the FP64 oracle gradient."""
    s = synth.boomerang_suspension(nb, box, 23, lift=lift)
    r = positions(s)
    rng = np.random.default_rng(24)
    u, F = rng.standard_normal((2, 3, s.n))
    h = handle_for(s)
    g = h.mobility_adjoint(to_dev(r), to_dev(u), to_dev(F), dtype=F32).cpu().numpy()
    go = om.grad(r, u, F, oracle_params(s))
    assert rel2(g, go) <= 1e-5
    # per-blob: no blob's gradient is off by more than 1e-4 of the largest
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
