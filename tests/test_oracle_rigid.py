"""Pins of the oracle rigid kinematics: K and K^T adjoint (Sec. 2.1), rigid
rotations, and the Rotate update of App. B.1 (eq. rotate)."""
import numpy as np

from oracle import rigid
from paper_1709_02410_gb300 import synth


def test_rotation_matrices_orthonormal():
    th = synth.random_quaternions(np.random.default_rng(0), 50)
    R = rigid.quat_to_rot(th)
    np.testing.assert_allclose(np.einsum('bij,bkj->bik', R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)


def test_rotation_quarter_turn_about_z():
    th = np.array([[np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)]])
    np.testing.assert_allclose(rigid.quat_to_rot(th)[0] @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_blob_positions_rigid():
    s = synth.boomerangs_1920(0)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    rb = r.T.reshape(s.nb, s.nper, 3)
    d = np.linalg.norm(rb[:, :, None] - rb[:, None], axis=-1)
    d0 = np.linalg.norm(s.shape[:, None] - s.shape[None], axis=-1)
    np.testing.assert_allclose(d, np.broadcast_to(d0, d.shape), atol=1e-12)
    np.testing.assert_allclose(rb[:, 0], s.q, atol=1e-14)      # cross-point is the tracking point


def test_K_KT_adjoint():
    s = synth.boomerang_suspension(7, 10.0, 3)
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((7, 6))
    lam = rng.standard_normal((3, s.n))
    lhs = np.sum(lam * rigid.K_apply(r, s.q, U, s.nper))
    rhs = np.sum(U * rigid.KT_apply(r, s.q, lam, s.nper))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    Kp = rigid.K_matrix_body(r[:, :15], s.q[0])
    v = rigid.K_apply(r[:, :15], s.q[:1], U[:1], 15)
    np.testing.assert_allclose(Kp @ U[0], v.T.reshape(-1), atol=1e-13)


def test_rotate_expansion_and_norm():
    """Rotate(theta, w dt) = theta + dt Psi w - dt^2/8 |w|^2 theta + O(dt^3)."""
    rng = np.random.default_rng(2)
    th = synth.random_quaternions(rng, 5)
    w = rng.standard_normal((5, 3))
    errs = []
    for dt in (1e-2, 5e-3):
        new = rigid.rotate(th, dt * w)
        np.testing.assert_allclose(np.linalg.norm(new, axis=1), 1.0, atol=1e-15)
        approx = th + dt * np.einsum('bij,bj->bi', rigid.psi(th), w) - dt**2 / 8 * np.sum(w * w, 1)[:, None] * th
        errs.append(np.abs(new - approx).max())
    assert 6 < errs[0] / errs[1] < 10     # third order remainder


def test_rotate_matches_rotation_of_blobs():
    rng = np.random.default_rng(3)
    th = synth.random_quaternions(rng, 1)
    phi = np.array([[0.0, 0.0, np.pi / 2]])
    R0 = rigid.quat_to_rot(th)[0]
    R1 = rigid.quat_to_rot(rigid.rotate(th, phi))[0]
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    np.testing.assert_allclose(R1, Rz @ R0, atol=1e-14)
