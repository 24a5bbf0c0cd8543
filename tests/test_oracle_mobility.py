"""Pins of the oracle blob mobility against what the mathematics fixes.

The paper (Sec. 2.1, Sec. 4) uses the Rotne-Prager-Blake tensor without
printing it; these tests tie the oracle's definition to independent facts:
near-wall self mobility in closed form, the double surface average of the
Green's function (which the RPY/Faxen form must equal for separated spheres),
no-slip, reciprocity, symmetry, positive definiteness, continuity, decay.
"""
import numpy as np
import pytest

from oracle import mobility as om

ETA, A = 1e-3, 0.325
P = om.Params(ETA, A, wall=True)
P0 = om.Params(ETA, A, wall=False)
MU0 = 1.0 / (6 * np.pi * ETA * A)


def blake_numpy(x, y):
    """Blake's image system (point force at y above a no-slip plane z = 0),
    times 8 pi eta, vectorised over leading axes of x and y.  Written
    independently of the oracle's symbolic derivation:
    G = S(x - y) - S(R) + 2h D_jk d/dR_k [h R_i/|R|^3 - S_i3(R)], R = x - y*."""
    d = x - y
    R = x - y * np.array([1.0, 1.0, -1.0])
    h = y[..., 2]
    def S(v):
        n = np.linalg.norm(v, axis=-1)
        return (np.eye(3) / n[..., None, None]
                + v[..., :, None] * v[..., None, :] / n[..., None, None] ** 3)
    Rn = np.linalg.norm(R, axis=-1)[..., None, None]
    Ri = R[..., :, None]
    Rk = R[..., None, :]
    I = np.eye(3)
    e3 = np.array([0.0, 0.0, 1.0])
    hh = h[..., None, None]
    # d/dR_k of phi_i = h R_i/R^3 - delta_i3/R - R_i R_3/R^3, indexed [i, k]
    R3 = R[..., 2][..., None, None]
    dphi = (hh * (I / Rn**3 - 3 * Ri * Rk / Rn**5)
            + e3[:, None] * Rk / Rn**3
            - (I * R3 + Ri * e3[None, :]) / Rn**3
            + 3 * Ri * R3 * Rk / Rn**5)
    D = np.diag([1.0, 1.0, -1.0])
    img = 2 * hh * np.einsum('...ik,jk->...ij', dphi, D)
    return S(d) - S(R) + img


def sphere_rule(n_t=24, n_p=48):
    """Product Gauss-Legendre (cos theta) x trapezoid (phi) rule on the unit
    sphere, weights summing to 1."""
    ct, wt = np.polynomial.legendre.leggauss(n_t)
    ph = 2 * np.pi * np.arange(n_p) / n_p
    st = np.sqrt(1 - ct**2)
    pts = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(n_p))], -1)
    w = np.outer(wt, np.ones(n_p)) / (2 * n_p)
    return pts.reshape(-1, 3), w.reshape(-1)


@pytest.mark.parametrize("h", [1.0 * A, 1.3 * A, 2.0 * A, 5.0 * A, 40.0 * A])
def test_self_mobility_closed_form(h):
    """Faxen-corrected Blake self mobility (RPB): mu_par/mu0 = 1 - 9/16 x +
    1/8 x^3 - 1/16 x^5, mu_perp/mu0 = 1 - 9/8 x + 1/2 x^3 - 1/8 x^5, x = a/h."""
    M = om.pair_block([0.3, -1.2, h], [0.3, -1.2, h], P, same=True) / MU0
    x = A / h
    par = 1 - 9 / 16 * x + x**3 / 8 - x**5 / 16
    perp = 1 - 9 / 8 * x + x**3 / 2 - x**5 / 8
    np.testing.assert_allclose(np.diag(M), [par, par, perp], rtol=1e-13)
    off = M - np.diag(np.diag(M))
    assert np.max(np.abs(off)) < 1e-14


def test_blake_point_no_slip_and_reciprocity():
    rng = np.random.default_rng(11)
    for _ in range(20):
        y = np.array([*rng.uniform(-2, 2, 2), rng.uniform(0.2, 3)])
        x = np.array([*rng.uniform(-2, 2, 2), 0.0])
        assert np.max(np.abs(om.blake_point(x, y))) < 1e-12
        x[2] = rng.uniform(0.2, 3)
        G = om.blake_point(x, y)
        np.testing.assert_allclose(G, om.blake_point(y, x).T, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(G, blake_numpy(x, y), rtol=1e-12, atol=1e-14)


def test_blake_point_divergence_free():
    rng = np.random.default_rng(12)
    eps = 1e-5
    for _ in range(10):
        y = np.array([*rng.uniform(-1, 1, 2), rng.uniform(0.5, 2)])
        x = np.array([*rng.uniform(-1, 1, 2), rng.uniform(0.5, 2)])
        div = np.zeros(3)
        for c in range(3):
            e = np.zeros(3); e[c] = eps
            div += (om.blake_point(x + e, y)[c] - om.blake_point(x - e, y)[c]) / (2 * eps)
        assert np.max(np.abs(div)) < 1e-7 * np.max(np.abs(om.blake_point(x, y)))


def test_rpy_far_branch_is_surface_average_of_oseen():
    pts, w = sphere_rule(16, 32)
    rng = np.random.default_rng(13)
    for _ in range(4):
        d = rng.standard_normal(3)
        d *= rng.uniform(3.0, 6.0) * A / np.linalg.norm(d)
        xs = d + A * pts
        ys = A * pts
        v = xs[:, None, :] - ys[None, :, :]
        n = np.linalg.norm(v, axis=-1)
        S = np.eye(3) / n[..., None, None] + v[..., :, None] * v[..., None, :] / n[..., None, None] ** 3
        avg = np.einsum('i,j,ijab->ab', w, w, S) / (8 * np.pi * ETA)
        M = om.pair_block(d, [0, 0, 0], P0)
        np.testing.assert_allclose(M, avg, rtol=1e-9, atol=1e-9 * np.abs(M).max())


def test_wall_tensor_is_surface_average_of_blake():
    """For spheres clear of the wall and of each other, the RPY-Blake block
    equals the double surface average of Blake's Green's function."""
    pts, w = sphere_rule(20, 40)
    rng = np.random.default_rng(14)
    for _ in range(5):
        x = np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(1.6, 3.0) * A])
        y = np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(1.6, 3.0) * A])
        if np.linalg.norm(x - y) < 3.0 * A:
            continue
        xs = x + A * pts
        ys = y + A * pts
        G = blake_numpy(xs[:, None, :], ys[None, :, :])
        avg = np.einsum('i,j,ijab->ab', w, w, G) / (8 * np.pi * ETA)
        M = om.pair_block(x, y, P)
        np.testing.assert_allclose(M, avg, rtol=1e-7, atol=1e-8 * np.abs(M).max())


def test_rpy_continuity_at_2a():
    e = np.array([0.6, -0.48, 0.64])
    lo = om.pair_block(e * (2 * A * (1 - 1e-12)), [0, 0, 0], P0)
    hi = om.pair_block(e * (2 * A * (1 + 1e-12)), [0, 0, 0], P0)
    np.testing.assert_allclose(lo, hi, rtol=1e-10)
    # both branches give 7/(96 pi eta a) I + 1/(32 pi eta a) e e^T at r = 2a
    expect = 7 / (96 * np.pi * ETA * A) * np.eye(3) + np.outer(e, e) / (32 * np.pi * ETA * A)
    np.testing.assert_allclose(hi, expect, rtol=1e-10)


def test_rpy_overlap_limit_is_self():
    M = om.pair_block([1e-9, 0, 0], [0, 0, 0], P0)
    np.testing.assert_allclose(M, MU0 * np.eye(3), rtol=1e-8)


def test_free_space_limit_far_from_wall():
    rng = np.random.default_rng(15)
    for _ in range(5):
        d = rng.standard_normal(3) * 2
        Mf = om.pair_block(d, [0, 0, 0], P0)
        diffs = []
        for z in (1e3 * A, 1e4 * A, 1e5 * A):
            Mw = om.pair_block(np.array([0, 0, z]) + d, [0, 0, z], P)
            diffs.append(np.max(np.abs(Mw - Mf)))
        # the image part is O(1/z): tenfold height, tenfold smaller
        assert diffs[2] < 2e-4 * np.max(np.abs(Mf))
        assert 8 < diffs[0] / diffs[1] < 12 and 8 < diffs[1] / diffs[2] < 12


def test_symmetry_blocks():
    rng = np.random.default_rng(16)
    for _ in range(50):
        ri = np.array([*rng.uniform(-3, 3, 2), rng.uniform(-0.5, 3)])
        rj = np.array([*rng.uniform(-3, 3, 2), rng.uniform(-0.5, 3)])
        np.testing.assert_allclose(om.pair_block(ri, rj, P), om.pair_block(rj, ri, P).T,
                                   rtol=1e-12, atol=1e-12 * MU0)


def random_cluster(n, seed, zlo=-0.3, zhi=2.0, box=3.0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(zlo, zhi, n)])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spd_dense(seed):
    r = random_cluster(64, seed)
    M = om.dense(r, P)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * MU0)
    assert np.linalg.eigvalsh(M).min() > 0


def test_matvec_matches_dense_and_uFMu():
    r = random_cluster(40, 5)
    rng = np.random.default_rng(6)
    F = rng.standard_normal((2, 3, 40))
    U = om.apply(r, F, P)
    M = om.dense(r, P)
    for k in range(2):
        np.testing.assert_allclose(om.soa_to_blob(U[k]), M @ om.soa_to_blob(F[k]), rtol=1e-12,
                                   atol=1e-12 * np.abs(U).max())
    u = om.soa_to_blob(F[0]); f = om.soa_to_blob(F[1])
    assert abs(u @ M @ f - f @ M @ u) < 1e-13 * abs(u @ M @ f) + 1e-12
    rows = np.array([3, 17, 39])
    Ur = om.apply(r, F, P, rows=rows)
    np.testing.assert_allclose(Ur, U[:, :, rows], rtol=1e-14)


def test_far_field_decay_r3():
    """Blob mobility above the wall is screened: pair blocks decay like r^-3."""
    h = 1.5 * A
    vals = []
    for r in (200.0, 400.0):
        vals.append(np.abs(om.pair_block([r, 0, h], [0, 0, h], P)).max())
    assert 7.5 < vals[0] / vals[1] < 8.5


def test_regularisation_continuity_at_h_equals_a():
    lo = om.pair_block([0.7, 0.1, A * (1 - 1e-12)], [0, 0, 1.1], P)
    hi = om.pair_block([0.7, 0.1, A * (1 + 1e-12)], [0, 0, 1.1], P)
    np.testing.assert_allclose(lo, hi, rtol=1e-9)


def test_point_force_no_slip_limit():
    """With a -> 0 the block vanishes as the source approaches the wall."""
    p = om.Params(ETA, 1e-9, wall=True)
    M = om.pair_block([0.5, 0.2, 1.0], [0, 0, 1e-6], p)
    Mref = om.pair_block([0.5, 0.2, 1.0], [0, 0, 1.0], p)
    assert np.abs(M).max() < 1e-4 * np.abs(Mref).max()
