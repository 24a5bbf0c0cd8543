"""Pin of the oracle RFD drift (Sec. 3, eqs. RFDcenter/RFDB): its mean over
random directions is the exact divergence of M, and at small delta a single
sample equals the directional derivative (dM . W) W."""
import numpy as np

from oracle import mobility as om, rfd

ETA, A = 1e-3, 0.325
P = om.Params(ETA, A, wall=True)


def test_single_sample_is_directional_derivative():
    rng = np.random.default_rng(0)
    n = 10
    r = np.stack([rng.uniform(0, 3, n), rng.uniform(0, 3, n), rng.uniform(0.4, 2, n)])
    W = rng.standard_normal((3, n))
    d = rfd.rfd_drift(r, W, 1e-5, P)
    # exact directional derivative from the per-pair derivative tensors
    ref = np.zeros((3, n))
    for i in range(n):
        for j in range(n):
            Dx, Dy = om.pair_dblock(r[:, i], r[:, j], P, same=(i == j))
            dM = np.einsum('cde,e->cd', Dx, W[:, i]) + np.einsum('cde,e->cd', Dy, W[:, j])
            ref[:, i] += dM @ W[:, j]
    np.testing.assert_allclose(d, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())


def test_mean_is_divergence():
    rng = np.random.default_rng(1)
    n = 4
    r = np.stack([rng.uniform(0, 1.5, n), rng.uniform(0, 1.5, n), rng.uniform(0.5, 1.2, n)])
    div = om.divergence(r, P)
    ns = 4000
    acc = np.zeros((ns, 3, n))
    for s in range(ns):
        W = rng.standard_normal((3, n))
        acc[s] = rfd.rfd_drift(r, W, 1e-4, P)
    mean = acc.mean(0)
    se = acc.std(0) / np.sqrt(ns)
    assert np.all(np.abs(mean - div) < 5 * se + 1e-9)
