"""Oracle mobility problem (eq. saddle, Sec. 2.1) at the blob/body level.
TEST INFRASTRUCTURE.

[M  -K][lam]   [-slip]
[-K^T 0][ U ] = [ -F  ]
Unknown vector x = [lam (3n, SoA flattened), U (6 nb)].
"""
import numpy as np

from . import krylov, mobility, precond, rigid


class Saddle:
    def __init__(self, r, q, nper, prm: mobility.Params, pc: precond.BlockPrecond = None):
        self.r, self.q, self.nper, self.prm = r, q, nper, prm
        self.n = r.shape[1]
        self.nb = q.shape[0]
        self.pc = pc if pc is not None else precond.BlockPrecond(r, q, nper, prm)
        self.matvecs = 0

    def split(self, x):
        return x[:3 * self.n].reshape(3, self.n), x[3 * self.n:].reshape(self.nb, 6)

    def join(self, lam, U):
        return np.concatenate([np.asarray(lam).reshape(-1), np.asarray(U).reshape(-1)])

    def A(self, x):
        lam, U = self.split(x)
        self.matvecs += 1
        top = mobility.apply(self.r, lam, self.prm) - rigid.K_apply(self.r, self.q, U, self.nper)
        bot = -rigid.KT_apply(self.r, self.q, lam, self.nper)
        return self.join(top, bot)

    def Pinv(self, x):
        a, b = self.split(x)
        lam, U = self.pc.saddle_solve(a, b)
        return self.join(lam, U)

    def solve(self, slip, F, tol, restart=50, max_iter=500):
        """Returns (lam [3, n], U [nb, 6], iterations, rel_residual)."""
        slip = np.zeros((3, self.n)) if slip is None else slip
        F = np.zeros((self.nb, 6)) if F is None else F
        b = self.join(-slip, -F)
        x, it, rel = krylov.gmres(self.A, self.Pinv, b, tol, restart, max_iter)
        lam, U = self.split(x)
        return lam.copy(), U.copy(), it, rel


def dense_solution(r, q, nper, prm, slip, F):
    """U = N F + N K^T M^-1 slip, lam = M^-1 (K U - slip) with
    N = (K^T M^-1 K)^-1 (eqs. sysDense, N_def), dense FP64."""
    n, nb = r.shape[1], q.shape[0]
    M = mobility.dense(r, prm)
    Kd = np.zeros((3 * n, 6 * nb))
    for p in range(nb):
        Kd[3 * nper * p:3 * nper * (p + 1), 6 * p:6 * p + 6] = rigid.K_matrix_body(r[:, p * nper:(p + 1) * nper], q[p])
    Minv = np.linalg.inv(M)
    N = np.linalg.inv(Kd.T @ Minv @ Kd)
    s = np.zeros(3 * n) if slip is None else mobility.soa_to_blob(slip)
    f = np.zeros(6 * nb) if F is None else np.asarray(F).reshape(-1)
    U = N @ (f + Kd.T @ Minv @ s)
    lam = Minv @ (Kd @ U - s)
    return mobility.blob_to_soa(lam), U.reshape(nb, 6), N
