"""Pins of the oracle time steps (Algorithms 1 and 2).

Deterministically (k_B T = 0) EM-T is the Euler rule and T-S the trapezoidal
rule (Sec. 3.2: T-S is second order deterministically): one-step errors
against a fine reference must fall like dt^2 and dt^3."""
import numpy as np

from oracle import mobility as om, rigid, steps
from paper_1709_02410_gb300 import synth


def two_bodies():
    s = synth.boomerang_suspension(2, 3.0, 21)
    prm = om.Params(synth.ETA, s.a)
    fm = steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1, torque=(0.0, 0.2, 0.0))
    return s, prm, fm


def one_step(kind, s, prm, fm, dt, kT=0.0):
    z3 = np.zeros((3, s.n))
    zb = np.zeros((s.nb, 3))
    sol = steps.Solver("dense")
    args = (s.q, s.theta, s.shape, prm, fm, dt, 1e-6, 14.7 * s.a)
    if kind == "ts":
        q, th, _ = steps.step_ts(*args, z3, z3, sol, kT)
    elif kind == "emt":
        q, th, _ = steps.step_emt(*args, zb, zb, z3, sol, kT)
    elif kind == "emrfd":
        q, th, _ = steps.step_emrfd(*args, zb, zb, z3, sol, kT)
    else:
        q, th, _ = steps.step_tt(*args, zb, zb, z3, sol, kT)
    return rigid.blob_positions(q, th, s.shape)


def reference(s, prm, fm, T, nsub):
    q, th = s.q.copy(), s.theta.copy()
    z3 = np.zeros((3, s.n))
    sol = steps.Solver("dense")
    for _ in range(nsub):
        q, th, _ = steps.step_ts(q, th, s.shape, prm, fm, T / nsub, 1e-6, 1.0, z3, z3, sol, 0.0)
    return rigid.blob_positions(q, th, s.shape)


def test_deterministic_orders():
    s, prm, fm = two_bodies()
    T = 0.01
    ref = {dt: reference(s, prm, fm, dt, 32) for dt in (T, T / 2)}
    e_ts = [np.abs(one_step("ts", s, prm, fm, dt) - ref[dt]).max() for dt in (T, T / 2)]
    e_em = [np.abs(one_step("emt", s, prm, fm, dt) - ref[dt]).max() for dt in (T, T / 2)]
    e_rfd = [np.abs(one_step("emrfd", s, prm, fm, dt) - ref[dt]).max() for dt in (T, T / 2)]
    e_tt = [np.abs(one_step("tt", s, prm, fm, dt) - ref[dt]).max() for dt in (T, T / 2)]
    assert 6.5 < e_ts[0] / e_ts[1] < 10.0      # local error O(dt^3)
    assert 6.5 < e_tt[0] / e_tt[1] < 10.0
    assert 3.4 < e_em[0] / e_em[1] < 4.6       # local error O(dt^2)
    assert 3.4 < e_rfd[0] / e_rfd[1] < 4.6
    # deterministically EM-T and EM-RFD are the same Euler rule
    np.testing.assert_allclose(e_rfd, e_em, rtol=1e-6)


def test_first_velocity_is_N_F():
    s, prm, fm = two_bodies()
    z3 = np.zeros((3, s.n))
    _, _, info = steps.step_ts(s.q, s.theta, s.shape, prm, fm, 1e-3, 1e-6, 1.0, z3, z3, steps.Solver("dense"), 0.0)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    from oracle import saddle
    _, _, N = saddle.dense_solution(r, s.q, s.nper, prm, None, None)
    F = steps.body_forces(r, s.q, s.nper, fm)
    np.testing.assert_allclose(info["Un"].reshape(-1), N @ F.reshape(-1), rtol=1e-9, atol=1e-12)


def test_iterative_matches_dense_step():
    s, prm, fm = two_bodies()
    rng = np.random.default_rng(5)
    Ws, W = rng.standard_normal((2, 3, s.n))
    args = (s.q, s.theta, s.shape, prm, fm, 0.01, 1e-4, 14.7 * s.a, Ws, W)
    qd, td, _ = steps.step_ts(*args, steps.Solver("dense"), synth.KT)
    qi, ti, _ = steps.step_ts(*args, steps.Solver("iterative", 1e-12, 1e-12), synth.KT)
    np.testing.assert_allclose(qi, qd, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ti, td, rtol=1e-9, atol=1e-9)


def test_steric_forces_are_a_gradient_and_balance():
    """Blob-blob Yukawa forces: minus the gradient of sum gamma e^{-r/b}/r over
    pairs of different bodies (central differences), and they sum to zero."""
    s = synth.boomerang_suspension(3, 2.0, 33)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    fm = steps.ForceModel(steric_gamma=0.096, steric_b=0.162, r_floor=1e-3)
    f = steps.blob_forces(r, fm, s.nper)
    body = np.arange(s.n) // s.nper

    def energy(rr):
        e = 0.0
        for i in range(s.n):
            for j in range(i + 1, s.n):
                if body[i] != body[j]:
                    d = np.linalg.norm(rr[:, i] - rr[:, j])
                    e += 0.096 * np.exp(-d / 0.162) / d
        return e
    h = 1e-6
    for i in (0, 7, 20, 44):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[c, i] += h
            rm[c, i] -= h
            assert abs(-(energy(rp) - energy(rm)) / (2 * h) - f[c, i]) < 1e-6 * max(1.0, np.abs(f).max())
    np.testing.assert_allclose(f.sum(axis=1), 0.0, atol=1e-10 * np.abs(f).max())
