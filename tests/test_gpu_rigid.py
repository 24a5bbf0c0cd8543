"""GPU parity of K, K^T, the force model and Philox normals."""
import numpy as np
import pytest

from oracle import philox, rigid, steps
from paper_1709_02410_gb300 import synth
from paper_1709_02410_gb300._native import F32, F64, Forces

from gpu_util import handle_for, positions, to_dev

pytestmark = pytest.mark.gpu


def test_K_and_KT():
    s = synth.boomerangs_1920()
    r = positions(s)
    rng = np.random.default_rng(0)
    U = rng.standard_normal((s.nb, 6))
    lam = rng.standard_normal((3, s.n))
    h = handle_for(s)
    Kd = h.K_apply(s.nper, to_dev(r), to_dev(s.q), to_dev(U)).cpu().numpy()
    np.testing.assert_allclose(Kd, rigid.K_apply(r, s.q, U, s.nper), rtol=1e-13, atol=1e-13)
    KTd = h.KT_apply(s.nper, to_dev(r), to_dev(s.q), to_dev(lam)).cpu().numpy()
    np.testing.assert_allclose(KTd, rigid.KT_apply(r, s.q, lam, s.nper), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n", [1, 3, 4, 5, 1001])
def test_philox_normals(n):
    s = synth.boomerangs_1920()
    h = handle_for(s)
    z = h.philox_normals(n, seed=0x1234567890ABCDEF, step=9, sid=1).cpu().numpy()
    np.testing.assert_allclose(z, philox.normals(n, 0x1234567890ABCDEF, 9, 1), rtol=1e-13, atol=1e-13)


def test_blob_forces():
    s = synth.boomerangs_1920()
    r = positions(s)
    fm = steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1)
    f = Forces(fm.weight, fm.wall_gamma, fm.wall_b, fm.h_floor, (0.0, 0.0, 0.0))
    h = handle_for(s)
    out = h.blob_forces(to_dev(r), f).cpu().numpy()
    np.testing.assert_allclose(out, steps.blob_forces(r, fm), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dtype,tol", [(F64, 1e-12), (F32, 1e-5)])
@pytest.mark.parametrize("r_cut", [0.0, 4.0])
def test_blob_forces_steric(r_cut, dtype, tol):
    """Blob-blob Yukawa repulsion between blobs of different bodies (FP64
    separations, force arithmetic in dtype) against the FP64 oracle."""
    s = synth.boomerangs_1920()
    r = positions(s)
    fm = steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1, steric_gamma=0.5,
                          steric_b=0.3, r_floor=0.1, r_cut=r_cut)
    f = Forces(fm.weight, fm.wall_gamma, fm.wall_b, fm.h_floor, (0.0, 0.0, 0.0), fm.steric_gamma, fm.steric_b,
               fm.r_floor, fm.r_cut)
    h = handle_for(s)
    out = h.blob_forces(to_dev(r), f, nper=s.nper, dtype=dtype).cpu().numpy()
    ref = steps.blob_forces(r, fm, s.nper)
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= tol * scale
    # the repulsion part is nonzero and momentum-conserving
    base = steps.blob_forces(r, steps.ForceModel(weight=0.05, wall_gamma=0.096, wall_b=0.162, h_floor=0.1))
    assert np.abs(ref - base).max() > 1e-3 * scale
    np.testing.assert_allclose((out - base).sum(axis=1), 0.0, atol=tol * scale * np.sqrt(s.n))


def test_blob_forces_steric_rejects_bad_args():
    s = synth.boomerangs_1920()
    h = handle_for(s)
    r = to_dev(positions(s))
    f = Forces(0.0, 0.0, 1.0, 0.1, (0.0, 0.0, 0.0), 1.0, 0.3, 0.1, 0.0)
    with pytest.raises(RuntimeError):
        h.blob_forces(r, f, nper=7)  # nper does not divide n
