"""Pins of the oracle's pseudo-periodic sum (Sec. 4.2: every blob interacts
with the minimum image of every other blob and with its 8 nearest periodic
images, in x and y; the wall stays at z = 0)."""
import numpy as np

from oracle import mobility as om

ETA, A = 1e-3, 0.325
L = 12.0
PP = om.Params(ETA, A, Lx=L, Ly=L)
P0 = om.Params(ETA, A)


def test_image_set_is_minimum_image_plus_eight():
    ri = np.array([0.4, 0.2, 0.9])
    for rj in (np.array([0.4 + 0.9 * L, 0.2 - 0.3 * L, 1.4]), np.array([1.1, 0.5, 0.7])):
        d = ri - rj
        m = np.round(d[:2] / L)
        ref = np.zeros((3, 3))
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                img = rj + np.array([(m[0] + a) * L, (m[1] + b) * L, 0.0])
                ref += om.pair_block(ri, img, P0)
        np.testing.assert_allclose(om.pair_block(ri, rj, PP), ref, rtol=1e-13)
    # self: Stokes drag + wall self term + the blob's own 8 images
    ref = om.pair_block(ri, ri, P0, same=True)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a or b:
                ref += om.pair_block(ri, ri + np.array([a * L, b * L, 0.0]), P0)
    np.testing.assert_allclose(om.pair_block(ri, ri, PP, same=True), ref, rtol=1e-13)


def test_translation_by_a_cell_changes_nothing():
    rng = np.random.default_rng(0)
    n = 30
    r = np.stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(0.4, 2.5, n)])
    F = rng.standard_normal((3, n))
    U = om.apply(r, F, PP)
    r2 = r.copy()
    r2[0, 3] += L
    r2[1, 7] -= 2 * L
    np.testing.assert_allclose(om.apply(r2, F, PP), U, rtol=1e-12, atol=1e-12 * np.abs(U).max())


def test_huge_cell_is_open_space():
    rng = np.random.default_rng(1)
    n = 20
    r = np.stack([rng.uniform(0, 3, n), rng.uniform(0, 3, n), rng.uniform(0.4, 2.5, n)])
    F = rng.standard_normal((3, n))
    Ubig = om.apply(r, F, om.Params(ETA, A, Lx=1e6, Ly=1e6))
    np.testing.assert_allclose(Ubig, om.apply(r, F, P0), rtol=1e-9, atol=1e-9 * np.abs(Ubig).max())


def test_periodic_symmetric_and_spd():
    rng = np.random.default_rng(2)
    n = 48
    r = np.stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(0.4, 2.5, n)])
    M = om.dense(r, PP)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(M).min() > 0


def test_periodic_gradient_matches_fd():
    rng = np.random.default_rng(3)
    n = 10
    r = np.stack([rng.uniform(0, L, n), rng.uniform(0, L, n), rng.uniform(0.4, 2.0, n)])
    u, F = rng.standard_normal((2, 3, n))
    g = om.grad(r, u, F, PP)
    h = 1e-6 * A
    for k in range(n):
        for c in range(3):
            rp, rm = r.copy(), r.copy()
            rp[c, k] += h
            rm[c, k] -= h
            fd = (np.sum(u * om.apply(rp, F, PP)) - np.sum(u * om.apply(rm, F, PP))) / (2 * h)
            assert abs(g[c, k] - fd) <= 1e-6 * np.abs(g).max()
