"""Drift consistency of the oracle time steps (the stochastic terms of
Algorithms 1, 2, 3 and of T-T).

Every integrator exists to put the Ito drift of the overdamped Langevin
equation written with unit quaternions (App. B, eq. quatLangevin) into the
mean displacement: with no forces,

    E[Q^{n+1} - Q^n] / dt = kT d/dQ . (Psi N Psi^T) + O(dt),

where N = (K^T M^-1 K)^-1 is the body mobility (eq. N_def) and Psi maps body
velocities to dQ/dt.  The reference here shares nothing with the steps: N
comes from the dense Schur form, and the divergence is a central finite
difference of Psi N along the columns of Psi (tangent to the unit
quaternion sphere), summed as d_k (Psi N Psi^T)_lk with d_k Psi_kj = 0.

The mean of a step is taken two ways, at N_b = 2 boomerangs (30 blobs,
dense solves, the exact limit of Lanczos):
 * deterministically, by the symmetric sigma-point rule
   E f(W) = f(0) + 1/2 sum_i [f(e_i) + f(-e_i) - 2 f(0)], exact for
   polynomials of degree <= 3 in the normals W; the velocity's quartic part
   carries an extra factor dt, so the rule is exact to O(dt) -- the order
   of the schemes' own bias (the test sees the error fall 10x from
   dt = 1e-3 to 1e-4);
 * by Monte Carlo over normals drawn from the oracle's Philox generator
   (antithetic pairs), within the standard errors.
A variant of the T-S step with D^S negated, or with D^F negated, inside
this test must fail the same check: the check is sensitive to each term."""
import numpy as np
import pytest

import oracle.steps as steps_mod
from oracle import mobility as om, philox, rigid, saddle, steps
from paper_1709_02410_gb300 import synth

KT = synth.KT
DELTA = 1e-4


@pytest.fixture(scope="module")
def setup():
    # 30 blobs: threads (OpenMP in the oracle's matvec, BLAS in numpy) only add overhead
    prev = om.num_threads()
    om.set_num_threads(1)
    try:
        from threadpoolctl import threadpool_limits
        limits = threadpool_limits(1)
    except ImportError:
        limits = None
    s = synth.boomerang_suspension(2, 3.0, 21)   # lifted: every blob above a
    prm = om.Params(synth.ETA, s.a)
    yield s, prm, ito_drift(s, prm)
    om.set_num_threads(prev)
    if limits is not None:
        limits.restore_original_limits()


def psi_big(s, theta):
    """Psi of all bodies, [7 nb, 6 nb]: identity on q, Psi(theta) (App. B.1) on theta."""
    P = np.zeros((7 * s.nb, 6 * s.nb))
    ps = rigid.psi(theta)
    for p in range(s.nb):
        P[7 * p:7 * p + 3, 6 * p:6 * p + 3] = np.eye(3)
        P[7 * p + 3:7 * p + 7, 6 * p + 3:6 * p + 6] = ps[p]
    return P


def ito_drift(s, prm, eps=1e-5):
    """kT d_k (Psi N Psi^T)_lk at the suspension's configuration: for every body
    velocity j, the central difference of column j of Psi N along v_j = Psi e_j."""
    Q0 = np.concatenate([s.q, s.theta], axis=1).reshape(-1)
    P0 = psi_big(s, s.theta)
    d = np.zeros(7 * s.nb)
    for j in range(6 * s.nb):
        col = []
        for sg in (1.0, -1.0):
            Q = (Q0 + sg * eps * P0[:, j]).reshape(s.nb, 7)
            q, th = Q[:, :3], Q[:, 3:]
            r = rigid.blob_positions(q, th, s.shape)
            _, _, N = saddle.dense_solution(r, q, s.nper, prm, None, None)
            col.append((psi_big(s, th) @ N)[:, j])
        d += (col[0] - col[1]) / (2.0 * eps)
    return KT * d


def velocity(kind, s, prm, dt, z):
    """(Q^{n+1} - Q^n) / dt of one force-free oracle step; z holds its normals
    (T-S: W^s then W; the others: (W^f, W^tau) per body then W)."""
    n, nb = s.n, s.nb
    fm = steps.ForceModel()
    sol = steps.Solver("dense")
    Lp = 14.7 * s.a
    if kind == "ts":
        q, th, _ = steps.step_ts(s.q, s.theta, s.shape, prm, fm, dt, DELTA, Lp, z[:3 * n].reshape(3, n),
                                 z[3 * n:].reshape(3, n), sol, KT)
    else:
        Wb = z[:6 * nb].reshape(nb, 6)
        fn = {"emt": steps.step_emt, "emrfd": steps.step_emrfd, "tt": steps.step_tt}[kind]
        q, th, _ = fn(s.q, s.theta, s.shape, prm, fm, dt, DELTA, Lp, Wb[:, :3], Wb[:, 3:],
                      z[6 * nb:].reshape(3, n), sol, KT)
    return np.concatenate([q - s.q, th - s.theta], axis=1).reshape(-1) / dt


def dim(kind, s):
    return 6 * s.n if kind == "ts" else 6 * s.nb + 3 * s.n


def sigma_point_mean(kind, s, prm, dt):
    d = dim(kind, s)
    f0 = velocity(kind, s, prm, dt, np.zeros(d))
    acc = f0.copy()
    for i in range(d):
        e = np.zeros(d)
        e[i] = 1.0
        acc += 0.5 * (velocity(kind, s, prm, dt, e) + velocity(kind, s, prm, dt, -e) - 2.0 * f0)
    return acc


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_ito_drift_reference(setup):
    """Pins of the reference itself: it is not trivial, and its quaternion part
    has the radial component fixed by theta^T Psi = 0 (App. B.1).  Differentiating
    theta_l Psi_li = 0 gives theta_l d_k Psi_li = -Psi_ki, so
    theta . drift_theta = -kT tr(Psi^T Psi N_ww) = -(kT/4) tr N_ww per body
    (Psi^T Psi = I/4 for a unit quaternion): the mean step keeps |theta| = 1."""
    s, prm, ex = setup
    assert np.abs(ex).max() > 1e-2 and np.all(np.isfinite(ex))
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    _, _, N = saddle.dense_solution(r, s.q, s.nper, prm, None, None)
    d = ex.reshape(s.nb, 7)
    for p in range(s.nb):
        Nww = N[6 * p + 3:6 * p + 6, 6 * p + 3:6 * p + 6]
        radial = float(s.theta[p] @ d[p, 3:])
        assert abs(radial + 0.25 * KT * np.trace(Nww)) <= 1e-7 * KT * np.trace(Nww)


@pytest.mark.parametrize("kind", ["ts", "emt", "emrfd", "tt"])
def test_mean_step_is_ito_drift(setup, kind):
    s, prm, ex = setup
    e3 = rel(sigma_point_mean(kind, s, prm, 1e-3), ex)
    assert e3 <= 1e-4, (kind, e3)
    if kind in ("ts", "emt"):
        # the residual is the O(dt) bias of a weakly first-order scheme
        e4 = rel(sigma_point_mean(kind, s, prm, 1e-4), ex)
        assert e4 <= 0.2 * e3 + 1e-9, (kind, e3, e4)


class _Negated:
    """A module stand-in whose function `name` returns minus the original."""

    def __init__(self, mod, name):
        self._mod, self._name = mod, name

    def __getattr__(self, attr):
        f = getattr(self._mod, attr)
        if attr == self._name:
            return lambda *a, **k: -f(*a, **k)
        return f


@pytest.mark.parametrize("module,fn", [("mobility", "apply"), ("rigid", "KT_apply")])
def test_variant_with_a_drift_term_negated_is_rejected(setup, monkeypatch, module, fn):
    """In the force-free T-S step, steps.py calls mobility.apply only to form
    D^S and rigid.KT_apply only to form D^F (and the zero force), so negating
    one of them in the step's module negates exactly that drift term."""
    s, prm, ex = setup
    monkeypatch.setattr(steps_mod, module, _Negated(getattr(steps_mod, module), fn))
    err = rel(sigma_point_mean("ts", s, prm, 1e-3), ex)
    assert err > 5e-3, err      # D^S: ~0.44, D^F: ~0.011, against <= 1e-4 for the real step


def test_monte_carlo_mean_with_philox_normals(setup):
    """T-S over 300 antithetic pairs of Philox4x32-10 normals (seed, step = pair, sid
    0 for W^s, 1 for W): every component within 4.5 standard errors of the drift."""
    s, prm, ex = setup
    n = s.n
    P = 300
    xs = np.empty((P, ex.size))
    for i in range(P):
        z = np.concatenate([philox.normals(3 * n, 2024, i, 0), philox.normals(3 * n, 2024, i, 1)])
        xs[i] = 0.5 * (velocity("ts", s, prm, 1e-3, z) + velocity("ts", s, prm, 1e-3, -z))
    m = xs.mean(axis=0)
    se = xs.std(axis=0, ddof=1) / np.sqrt(P)
    z = (m - ex) / se
    assert np.abs(z).max() < 4.5, z
    # the sample is informative: the standard errors are well below the drift
    assert np.linalg.norm(se) < 0.25 * np.linalg.norm(ex)
