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
