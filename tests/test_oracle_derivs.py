"""Pins of the oracle's exact derivatives (adjoint d(u^T M F)/dr and div M)
against central finite differences of the oracle mobility, translation
invariance and the divergence-free free-space RPY tensor."""
import numpy as np
import pytest

from oracle import mobility as om

ETA, A = 1e-3, 0.325
P = om.Params(ETA, A, wall=True)
P0 = om.Params(ETA, A, wall=False)


def cluster(n, seed, zlo=0.1, zhi=2.0, box=3.0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(zlo, zhi, n)])


@pytest.mark.parametrize("prm", [P, P0], ids=["wall", "free"])
def test_grad_matches_central_fd(prm):
    n = 12
    r = cluster(n, 3)
    rng = np.random.default_rng(4)
    u, F = rng.standard_normal((3, n)), rng.standard_normal((3, n))
    g = om.grad(r, u, F, prm)
    h = 1e-6 * A
    for k in range(n):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[c, k] += h
            rm[c, k] -= h
            fd = (np.sum(u * om.apply(rp, F, prm)) - np.sum(u * om.apply(rm, F, prm))) / (2 * h)
            assert abs(g[c, k] - fd) <= 1e-6 * np.abs(g).max()


def test_grad_translation_invariance():
    """M is invariant under horizontal translation: sum_k g_k,x = sum_k g_k,y = 0."""
    n = 30
    r = cluster(n, 5, zlo=-0.2)
    rng = np.random.default_rng(6)
    u, F = rng.standard_normal((3, n)), rng.standard_normal((3, n))
    g = om.grad(r, u, F, P)
    s = g.sum(axis=1)
    assert abs(s[0]) < 1e-10 * np.abs(g).sum() and abs(s[1]) < 1e-10 * np.abs(g).sum()
    assert abs(s[2]) > 1e-6 * np.abs(g).sum()      # z is not an invariance


def test_grad_rows_subset():
    n = 20
    r = cluster(n, 7)
    rng = np.random.default_rng(8)
    u, F = rng.standard_normal((3, n)), rng.standard_normal((3, n))
    rows = np.array([0, 5, 19])
    np.testing.assert_allclose(om.grad(r, u, F, P, rows=rows), om.grad(r, u, F, P)[:, rows], rtol=1e-14)


def test_divergence_free_space_is_zero():
    """Both RPY branches are divergence free (overlapping pairs included)."""
    r = cluster(20, 9, box=1.5)
    d = om.divergence(r, P0)
    assert np.abs(d).max() < 1e-9 * (1 / (6 * np.pi * ETA * A)) / A


@pytest.mark.parametrize("zlo", [0.5, -0.1], ids=["above", "penetrating"])
def test_divergence_matches_fd_of_dense(zlo):
    n = 8
    r = cluster(n, 10, zlo=zlo)
    d = om.divergence(r, P)
    h = 1e-6 * A
    ref = np.zeros((3, n))
    for j in range(n):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[c, j] += h
            rm[c, j] -= h
            dM = (om.dense(rp, P) - om.dense(rm, P)) / (2 * h)
            # (div M)_i = sum_j d (M_ij)_{:,c} / d r_j,c
            ref += dM[:, 3 * j + c].reshape(n, 3).T
    np.testing.assert_allclose(d, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_divergence_single_blob_is_dmu_perp_dh():
    """One blob: div M = d mu_perp / dh along z (only the wall term survives)."""
    h = 1.7 * A
    d = om.divergence(np.array([[0.0], [0.0], [h]]), P)[:, 0]
    x = A / h
    mu0 = 1 / (6 * np.pi * ETA * A)
    dmu = mu0 * (9 / 8 * A / h**2 - 1.5 * A**3 / h**4 + 5 / 8 * A**5 / h**6)
    np.testing.assert_allclose(d, [0, 0, dmu], rtol=1e-12, atol=1e-12 * mu0)
