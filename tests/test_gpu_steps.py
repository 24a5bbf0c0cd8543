"""GPU parity of the T-S (Algorithm 2) and EM-T (Algorithm 1) steps: the
library draws its own Philox normals; the oracle takes the same normals and
solves densely."""
import numpy as np
import pytest

from oracle import philox, steps
from paper_1709_02410_gb300 import F64, synth
from paper_1709_02410_gb300._native import Forces, StepParams

from gpu_util import handle_for, oracle_params, to_dev

pytestmark = pytest.mark.gpu

FM = steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1, torque=(0.0, 0.2, 0.0))


def forces():
    return Forces(FM.weight, FM.wall_gamma, FM.wall_b, FM.h_floor, FM.torque)


def sp(seed=77, step=3, dt=0.01, delta=1e-4, L=1.0, cold_start=0):
    return StepParams(dt, delta, L, 1e-12, 1e-12, 300, 60, 80, F64, seed, step, cold_start)


@pytest.mark.parametrize("cold_start", [0, 1])
@pytest.mark.parametrize("kind", ["ts", "emt", "emrfd", "tt"])
def test_step_matches_oracle(kind, cold_start):
    s = synth.boomerang_suspension(4, 4.0, 31)
    p = sp(cold_start=cold_start)
    h = handle_for(s)
    q, th = to_dev(s.q), to_dev(s.theta)
    stats, status = getattr(h, "step_" + kind)(to_dev(s.shape), q, th, forces(), p)
    assert status == 0, stats
    n = s.n
    W = philox.normals(3 * n, p.seed, p.step, 1).reshape(3, n)
    sol = steps.Solver("dense")
    if kind == "ts":
        Ws = philox.normals(3 * n, p.seed, p.step, 0).reshape(3, n)
        qo, tho, _ = steps.step_ts(s.q, s.theta, s.shape, oracle_params(s), FM, p.dt, p.delta, p.Lp, Ws, W, sol,
                                   synth.KT)
    else:
        Wb = philox.normals(6 * s.nb, p.seed, p.step, 2).reshape(s.nb, 6)
        fn = {"emt": steps.step_emt, "emrfd": steps.step_emrfd, "tt": steps.step_tt}[kind]
        qo, tho, _ = fn(s.q, s.theta, s.shape, oracle_params(s), FM, p.dt, p.delta, p.Lp, Wb[:, :3], Wb[:, 3:], W,
                        sol, synth.KT)
    dq = q.cpu().numpy() - s.q
    np.testing.assert_allclose(q.cpu().numpy(), qo, rtol=0, atol=1e-7 * np.abs(qo - s.q).max() + 1e-12)
    np.testing.assert_allclose(th.cpu().numpy(), tho, rtol=0, atol=1e-7 * np.abs(tho - s.theta).max() + 1e-12)
    assert np.abs(dq).max() > 0


@pytest.mark.parametrize("kind", ["ts", "emt"])
def test_step_with_steric_forces_matches_oracle(kind):
    """Steps whose force model includes the blob-blob repulsion between
    bodies (four boomerangs packed closely enough for it to matter)."""
    fm = steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1, torque=(0.0, 0.2, 0.0),
                          steric_gamma=0.2, steric_b=0.5, r_floor=0.1, r_cut=3.0)
    f = Forces(fm.weight, fm.wall_gamma, fm.wall_b, fm.h_floor, fm.torque, fm.steric_gamma, fm.steric_b,
               fm.r_floor, fm.r_cut)
    s = synth.boomerang_suspension(4, 2.5, 37)
    p = sp(seed=5, step=1)
    h = handle_for(s)
    q, th = to_dev(s.q), to_dev(s.theta)
    stats, status = getattr(h, "step_" + kind)(to_dev(s.shape), q, th, f, p)
    assert status == 0, stats
    n = s.n
    W = philox.normals(3 * n, p.seed, p.step, 1).reshape(3, n)
    sol = steps.Solver("dense")
    if kind == "ts":
        Ws = philox.normals(3 * n, p.seed, p.step, 0).reshape(3, n)
        qo, tho, _ = steps.step_ts(s.q, s.theta, s.shape, oracle_params(s), fm, p.dt, p.delta, p.Lp, Ws, W, sol,
                                   synth.KT)
    else:
        Wb = philox.normals(6 * s.nb, p.seed, p.step, 2).reshape(s.nb, 6)
        qo, tho, _ = steps.step_emt(s.q, s.theta, s.shape, oracle_params(s), fm, p.dt, p.delta, p.Lp, Wb[:, :3],
                                    Wb[:, 3:], W, sol, synth.KT)
    np.testing.assert_allclose(q.cpu().numpy(), qo, rtol=0, atol=1e-7 * np.abs(qo - s.q).max() + 1e-12)
    np.testing.assert_allclose(th.cpu().numpy(), tho, rtol=0, atol=1e-7 * np.abs(tho - s.theta).max() + 1e-12)
    # the repulsion changes the result
    q0, th0, _ = (steps.step_ts(s.q, s.theta, s.shape, oracle_params(s), FM, p.dt, p.delta, p.Lp, Ws, W, sol,
                                synth.KT) if kind == "ts" else
                  steps.step_emt(s.q, s.theta, s.shape, oracle_params(s), FM, p.dt, p.delta, p.Lp, Wb[:, :3],
                                 Wb[:, 3:], W, sol, synth.KT))
    assert np.abs(tho - th0).max() > 1e-6 * np.abs(tho - s.theta).max()


def _oracle_step(kind, s, p, fm=FM, prm=None):
    n = s.n
    prm = oracle_params(s) if prm is None else prm
    W = philox.normals(3 * n, p.seed, p.step, 1).reshape(3, n)
    sol = steps.Solver("dense")
    if kind == "ts":
        Ws = philox.normals(3 * n, p.seed, p.step, 0).reshape(3, n)
        return steps.step_ts(s.q, s.theta, s.shape, prm, fm, p.dt, p.delta, p.Lp, Ws, W, sol, synth.KT)[:2]
    Wb = philox.normals(6 * s.nb, p.seed, p.step, 2).reshape(s.nb, 6)
    fn = {"emt": steps.step_emt, "emrfd": steps.step_emrfd, "tt": steps.step_tt}[kind]
    return fn(s.q, s.theta, s.shape, prm, fm, p.dt, p.delta, p.Lp, Wb[:, :3], Wb[:, 3:], W, sol, synth.KT)[:2]


@pytest.mark.parametrize("kind", ["ts", "tt"])
def test_fp32_step_matches_oracle(kind):
    """The arithmetic the bench times: FP32 pairs, GMRES to 1e-6, Lanczos to
    1e-4, delta = 1e-3, lockstep solves, warm-started corrector.  The oracle
    step is exact (dense solves, exact square root) on the same Philox draws,
    so the difference is the solvers' stopping error plus FP32 rounding:
    Lanczos' stop test leaves a relative error of about its tolerance in
    M^{1/2} W (the Brownian part, most of the displacement); GMRES to 1e-6 on
    FP32 matvecs leaves ~1e-6 times the preconditioned saddle system's
    condition number (1e-5..1e-4); the FP32 RFD differences carry ~1e-6 / delta
    = 1e-3 of D^S, a drift term ~10x smaller than the Brownian displacement at
    dt = 0.01.  Sum ~3e-4 of the largest displacement; bound 1e-3."""
    from paper_1709_02410_gb300 import F32
    s = synth.boomerang_suspension(6, 6.0, 61)
    p = StepParams(0.01, 1e-3, 14.7 * s.a, 1e-6, 1e-4, 300, 100, 60, F32, 13, 2, 0)
    h = handle_for(s)
    q, th = to_dev(s.q), to_dev(s.theta)
    stats, status = getattr(h, "step_" + kind)(to_dev(s.shape), q, th, forces(), p)
    assert status == 0, stats
    qo, tho = _oracle_step(kind, s, p)
    dq = np.abs(qo - s.q).max()
    dth = np.abs(tho - s.theta).max()
    assert np.abs(q.cpu().numpy() - qo).max() <= 1e-3 * dq
    assert np.abs(th.cpu().numpy() - tho).max() <= 1e-3 * dth


def test_fp64_ts_step_rollers_matches_oracle():
    """Microrollers (12-blob icosahedra, a = 0.416, L_p = R_h): the 36 x 36
    body blocks of the preconditioner, overlapping blobs of neighbouring
    rollers, and the constant torque about y of the roller workload."""
    s = synth.roller_suspension(6, 0.4, 62)
    fm = steps.ForceModel(weight=0.0124 / 12, wall_gamma=0.096, wall_b=0.162, h_floor=0.1, torque=(0.0, 1.0, 0.0))
    f = Forces(fm.weight, fm.wall_gamma, fm.wall_b, fm.h_floor, fm.torque)
    # overlapping rollers: Lanczos to 1e-9 (80 iterations do not reach 1e-12 here)
    p = StepParams(0.008, 1e-4, synth.RH_ROLLER, 1e-12, 1e-9, 300, 60, 80, F64, 17, 4, 0)
    h = handle_for(s)
    q, th = to_dev(s.q), to_dev(s.theta)
    stats, status = h.step_ts(to_dev(s.shape), q, th, f, p)
    assert status == 0, stats
    qo, tho = _oracle_step("ts", s, p, fm)
    np.testing.assert_allclose(q.cpu().numpy(), qo, rtol=0, atol=1e-7 * np.abs(qo - s.q).max() + 1e-12)
    np.testing.assert_allclose(th.cpu().numpy(), tho, rtol=0, atol=1e-7 * np.abs(tho - s.theta).max() + 1e-12)
