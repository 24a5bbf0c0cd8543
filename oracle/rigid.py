"""Oracle rigid-body kinematics (FP64, numpy).  TEST INFRASTRUCTURE.

Bodies all share one reference shape s [nper, 3]; blob i of body p sits at
index p * nper + i.  Blob vectors are SoA [3, n]; body vectors are [nb, 6]
rows (u, omega) or (f, tau).
"""
import numpy as np


def quat_to_rot(theta):
    """Rotation matrices [nb, 3, 3] of unit quaternions theta = (s, p)
    (App. B.1): R = (s^2 - p.p) I + 2 p p^T + 2 s [p]_x."""
    theta = np.atleast_2d(theta)
    s = theta[:, 0]
    p = theta[:, 1:]
    R = np.zeros((theta.shape[0], 3, 3))
    pp = np.einsum('bi,bi->b', p, p)
    for i in range(3):
        R[:, i, i] = s * s - pp
    R += 2.0 * np.einsum('bi,bj->bij', p, p)
    cx = np.zeros_like(R)
    cx[:, 0, 1], cx[:, 0, 2] = -p[:, 2], p[:, 1]
    cx[:, 1, 0], cx[:, 1, 2] = p[:, 2], -p[:, 0]
    cx[:, 2, 0], cx[:, 2, 1] = -p[:, 1], p[:, 0]
    R += 2.0 * s[:, None, None] * cx
    return R


def blob_positions(q, theta, shape):
    """r_i = q_p + R(theta_p) s_i for i in body p (Sec. 2.1, multiblob model).
    Returns SoA [3, nb * nper]."""
    R = quat_to_rot(theta)
    r = q[:, None, :] + np.einsum('bij,kj->bki', R, shape)
    return np.ascontiguousarray(r.reshape(-1, 3).T)


def K_apply(r, q, U, nper):
    """(K U)_i = u_p + omega_p x (r_i - q_p)   (eq. K, Sec. 2.1)."""
    nb = q.shape[0]
    rb = r.T.reshape(nb, nper, 3)
    d = rb - q[:, None, :]
    u = U[:, None, :3]
    w = np.broadcast_to(U[:, None, 3:], d.shape)
    v = u + np.cross(w, d)
    return np.ascontiguousarray(v.reshape(-1, 3).T)


def KT_apply(r, q, lam, nper):
    """K^T lambda: f_p = sum_i lambda_i, tau_p = sum_i (r_i - q_p) x lambda_i
    (force and torque balance, Sec. 2.1)."""
    nb = q.shape[0]
    rb = r.T.reshape(nb, nper, 3)
    lb = lam.T.reshape(nb, nper, 3)
    d = rb - q[:, None, :]
    f = lb.sum(axis=1)
    t = np.cross(d, lb).sum(axis=1)
    return np.concatenate([f, t], axis=1)


def K_matrix_body(r_body, q_p):
    """Dense K_p [3 nper, 6] of one body, rows blob-interleaved (3i + c)."""
    nper = r_body.shape[1]
    Kp = np.zeros((3 * nper, 6))
    for i in range(nper):
        d = r_body[:, i] - q_p
        Kp[3 * i:3 * i + 3, :3] = np.eye(3)
        # omega x d = -[d]_x omega
        Kp[3 * i:3 * i + 3, 3:] = np.array([[0.0, d[2], -d[1]],
                                            [-d[2], 0.0, d[0]],
                                            [d[1], -d[0], 0.0]])
    return Kp


def quat_mul(a, b):
    """Quaternion product a (x) b of [.., 4] arrays (s, p)."""
    sa, pa = a[..., :1], a[..., 1:]
    sb, pb = b[..., :1], b[..., 1:]
    s = sa * sb - np.sum(pa * pb, axis=-1, keepdims=True)
    p = sa * pb + sb * pa + np.cross(pa, pb)
    return np.concatenate([s, p], axis=-1)


def rotate(theta, phi):
    """Rotate(theta, phi) = [cos(|phi|/2), sin(|phi|/2) phi/|phi|] (x) theta
    (App. B.1, eq. rotate): rotation by the angle vector phi = omega dt."""
    theta = np.atleast_2d(theta)
    phi = np.atleast_2d(phi)
    ang = np.linalg.norm(phi, axis=1, keepdims=True)
    half = 0.5 * ang
    with np.errstate(invalid='ignore', divide='ignore'):
        sinc = np.where(ang > 0, np.sin(half) / np.where(ang > 0, ang, 1.0), 0.5)
    qw = np.concatenate([np.cos(half), sinc * phi], axis=1)
    return quat_mul(qw, theta)


def psi(theta):
    """Psi(theta) = 1/2 [-p^T; s I - P] (App. B.1), [nb, 4, 3]."""
    theta = np.atleast_2d(theta)
    s, p = theta[:, 0], theta[:, 1:]
    out = np.zeros((theta.shape[0], 4, 3))
    out[:, 0, :] = -p
    P = np.zeros((theta.shape[0], 3, 3))
    P[:, 0, 1], P[:, 0, 2] = -p[:, 2], p[:, 1]
    P[:, 1, 0], P[:, 1, 2] = p[:, 2], -p[:, 0]
    P[:, 2, 0], P[:, 2, 1] = -p[:, 1], p[:, 0]
    out[:, 1:, :] = s[:, None, None] * np.eye(3) - P
    return 0.5 * out


def advance(q, theta, U, dt):
    """Q + dt U on the body manifold: q += dt u; theta = Rotate(theta, dt omega)."""
    return q + dt * U[:, :3], rotate(theta, dt * U[:, 3:])
