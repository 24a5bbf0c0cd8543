"""Pins of the oracle's preconditioner, Lanczos M^{1/2} W (Sec. 2.2) and
GMRES saddle solve (eq. saddle) against dense linear algebra."""
import numpy as np
import scipy.linalg
import pytest

from oracle import krylov, mobility as om, precond, rigid, saddle
from paper_1709_02410_gb300 import synth

KT = synth.KT


def small(nb=6, seed=0, box=6.0):
    s = synth.boomerang_suspension(nb, box, seed)
    prm = om.Params(synth.ETA, s.a)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    return s, prm, r


def test_block_precond_saddle_solve_is_exact_per_body():
    s, prm, r = small(3, 1)
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3, s.n))
    b = rng.standard_normal((s.nb, 6))
    lam, U = pc.saddle_solve(a, b)
    for p in range(s.nb):
        sl = slice(p * s.nper, (p + 1) * s.nper)
        Mpp = om.dense(r[:, sl], prm)
        Kp = rigid.K_matrix_body(r[:, sl], s.q[p])
        A = np.block([[Mpp, -Kp], [-Kp.T, np.zeros((6, 6))]])
        x = np.linalg.solve(A, np.concatenate([om.soa_to_blob(a[:, sl]), b[p]]))
        np.testing.assert_allclose(om.soa_to_blob(lam[:, sl]), x[:3 * s.nper], rtol=1e-8, atol=1e-10 * np.abs(x).max())
        np.testing.assert_allclose(U[p], x[3 * s.nper:], rtol=1e-8, atol=1e-10 * np.abs(x).max())
    # Cholesky factor reproduces the diagonal blocks
    Mpp = om.dense(r[:, :s.nper], prm)
    np.testing.assert_allclose(pc.L[0] @ pc.L[0].T, Mpp, rtol=1e-12, atol=1e-12 * np.abs(Mpp).max())


def test_gmres_matches_dense_schur():
    s, prm, r = small(6, 3)
    rng = np.random.default_rng(4)
    slip = rng.standard_normal((3, s.n))
    F = rng.standard_normal((s.nb, 6)) * 1e-2
    S = saddle.Saddle(r, s.q, s.nper, prm)
    lam, U, it, rel = S.solve(slip, F, tol=1e-12)
    lam_d, U_d, N = saddle.dense_solution(r, s.q, s.nper, prm, slip, F)
    assert rel <= 1e-12
    np.testing.assert_allclose(U, U_d, rtol=1e-9, atol=1e-9 * np.abs(U_d).max())
    np.testing.assert_allclose(lam, lam_d, rtol=1e-8, atol=1e-8 * np.abs(lam_d).max())
    # restarts give the same answer
    lam2, U2, it2, rel2 = S.solve(slip, F, tol=1e-12, restart=5)
    np.testing.assert_allclose(U2, U_d, rtol=1e-8, atol=1e-8 * np.abs(U_d).max())


def test_one_body_is_N_F():
    s, prm, r = small(1, 5)
    F = np.array([[0.3, -0.2, 0.1, 0.05, 0.02, -0.04]])
    S = saddle.Saddle(r, s.q, s.nper, prm)
    lam, U, it, rel = S.solve(None, F, tol=1e-13)
    Mpp = om.dense(r, prm)
    Kp = rigid.K_matrix_body(r, s.q[0])
    N = np.linalg.inv(Kp.T @ np.linalg.solve(Mpp, Kp))
    np.testing.assert_allclose(U[0], N @ F[0], rtol=1e-10)
    assert it <= 2          # the preconditioner is exact for one body


def test_N_half_identity():
    """N^{1/2} = N K^T M^{-1/2} satisfies N^{1/2} N^{1/2 T} = N (eq. sqrtN_def)."""
    s, prm, r = small(3, 6)
    M = om.dense(r, prm)
    Kd = scipy.linalg.block_diag(*[rigid.K_matrix_body(r[:, p * 15:(p + 1) * 15], s.q[p]) for p in range(3)])
    Minv = np.linalg.inv(M)
    N = np.linalg.inv(Kd.T @ Minv @ Kd)
    Mh = scipy.linalg.sqrtm(M).real
    Nh = N @ Kd.T @ np.linalg.inv(Mh)
    np.testing.assert_allclose(Nh @ Nh.T, N, rtol=1e-7, atol=1e-9 * np.abs(N).max())


def _G_dense(r, s, prm):
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    M = om.dense(r, prm)
    Lb = scipy.linalg.block_diag(*pc.L)
    G = np.linalg.solve(Lb, np.linalg.solve(Lb, M).T).T
    return pc, M, Lb, 0.5 * (G + G.T)


def test_lanczos_preconditioned_matches_dense_sqrt():
    s, prm, r = small(8, 7)
    pc, M, Lb, G = _G_dense(r, s, prm)
    W = np.random.default_rng(8).standard_normal((3, s.n))
    apply_G = lambda v: pc.Linv_apply(om.apply(r, pc.LinvT_apply(v), prm))
    y, it, ch = krylov.lanczos_sqrt(apply_G, W, 1e-12, 300)
    ref = scipy.linalg.sqrtm(G).real @ om.soa_to_blob(W)
    np.testing.assert_allclose(om.soa_to_blob(y), ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    # the preconditioned product L y is a valid square root: L G L^T = M
    np.testing.assert_allclose(Lb @ G @ Lb.T, M, rtol=1e-9, atol=1e-10 * np.abs(M).max())


def test_lanczos_unpreconditioned_matches_sqrtm():
    s, prm, r = small(4, 9)
    M = om.dense(r, prm)
    W = np.random.default_rng(10).standard_normal((3, s.n))
    y, it, ch = krylov.lanczos_sqrt(lambda v: om.apply(r, v, prm), W, 1e-12, 400)
    ref = scipy.linalg.sqrtm(M).real @ om.soa_to_blob(W)
    np.testing.assert_allclose(om.soa_to_blob(y), ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_lanczos_tolerance_tracks_error():
    s, prm, r = small(8, 11)
    pc, M, Lb, G = _G_dense(r, s, prm)
    W = np.random.default_rng(12).standard_normal((3, s.n))
    ref = scipy.linalg.sqrtm(G).real @ om.soa_to_blob(W)
    apply_G = lambda v: G @ v.reshape(-1)
    its = []
    for tol in (1e-2, 1e-4, 1e-6):
        y, it, ch = krylov.lanczos_sqrt(apply_G, om.soa_to_blob(W), tol, 300)
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 20 * tol
        its.append(it)
    assert its[0] <= its[1] <= its[2]


def test_lanczos_covariance_is_M():
    """Over many W, cov(L y) -> M: the result is a valid factor of M (Sec. 2.2)."""
    s, prm, r = small(2, 13, box=3.0)
    pc, M, Lb, G = _G_dense(r, s, prm)
    rng = np.random.default_rng(14)
    ns = 20000
    Ws = rng.standard_normal((ns, 3 * s.n))
    # dense G inside the same Lanczos routine (fast), tight tolerance
    Y = np.stack([krylov.lanczos_sqrt(lambda v: G @ v, w, 1e-10, 200)[0] for w in Ws[:ns]])
    X = Y @ Lb.T
    C = X.T @ X / ns
    err = np.linalg.norm(C - M)
    # Gaussian sample covariance: E|C - M|_F^2 = (|M|_F^2 + tr(M)^2) / ns
    expect = np.sqrt((np.linalg.norm(M) ** 2 + np.trace(M) ** 2) / ns)
    assert err < 1.5 * expect
    assert np.linalg.norm(G - M) > 10 * expect      # a missing L factor would fail
