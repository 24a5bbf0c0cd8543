"""GPU parity on the microroller geometry of the steps/s workload (12-blob
icosahedra, a = 0.416 um, packed at phi = 0.4 so neighbouring rollers'
blobs overlap): the 36 x 36 body blocks of the preconditioner in all four
apply modes, GMRES against the dense Schur solution (eq. sysDense),
preconditioned Lanczos against the dense L sqrtm(L^-1 M L^-T) W."""
import numpy as np
import pytest
import scipy.linalg

from oracle import mobility as om, precond, saddle
from paper_1709_02410_gb300 import F32, F64, synth

from gpu_util import handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def rollers(nb=8, seed=71):
    return synth.roller_suspension(nb, 0.4, seed)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_roller_precond_apply_modes(mode):
    s = rollers(10, 72)
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


@pytest.mark.parametrize("dtype,tol,bound", [(F64, 1e-12, 1e-9), (F32, 1e-6, 1e-4)])
def test_roller_gmres_matches_dense_schur(dtype, tol, bound):
    s = rollers(8, 73)
    r = positions(s)
    rng = np.random.default_rng(74)
    slip = rng.standard_normal((3, s.n))
    FT = rng.standard_normal((s.nb, 6)) * 1e-2
    lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), slip, FT)
    h = handle_for(s)
    lam, U, st = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), to_dev(slip), to_dev(FT), tol=tol,
                                     max_iter=300, restart=60, dtype=dtype)
    assert st["status"] == 0
    assert rel2(U.cpu().numpy(), U_d) <= bound
    assert rel2(lam.cpu().numpy(), lam_d) <= 10 * bound


def test_roller_lanczos_matches_dense_sqrt():
    s = rollers(8, 75)
    r = positions(s)
    prm = oracle_params(s)
    pc = precond.BlockPrecond(r, s.q, s.nper, prm)
    M = om.dense(r, prm)
    Lb = scipy.linalg.block_diag(*pc.L)
    G = np.linalg.solve(Lb, np.linalg.solve(Lb, M).T).T
    W = synth.gaussian(76, (3, s.n))
    ref = Lb @ (scipy.linalg.sqrtm(0.5 * (G + G.T)).real @ om.soa_to_blob(W))
    h = handle_for(s)
    h.precond_build(s.nper, to_dev(r), to_dev(s.q))
    out, st = h.lanczos_sqrt_apply(to_dev(r), to_dev(W), tol=1e-12, max_iter=80)
    assert st["status"] == 0
    assert rel2(om.soa_to_blob(out.cpu().numpy()), ref) <= 1e-9
