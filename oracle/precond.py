"""Oracle body-block-diagonal preconditioner (FP64).  TEST INFRASTRUCTURE.

Sec. 2.2: hydrodynamic interactions between distinct bodies are dropped,
M~(pq) = delta_pq M(pp), where M(pp) is the dense blob mobility of body p
alone (wall included).  For Lanczos the preconditioner is the block Cholesky
factor L with M(pp) = L_p L_p^T; for the saddle system (eq. saddle) it is the
exact block solve using N_p = (K_p^T M(pp)^-1 K_p)^-1 (eq. N_def per body).
"""
import numpy as np

from . import mobility, rigid


class BlockPrecond:
    def __init__(self, r, q, nper, prm: mobility.Params):
        nb = q.shape[0]
        self.nb, self.nper = nb, nper
        self.L, self.Minv, self.N, self.K = [], [], [], []
        for p in range(nb):
            rb = r[:, p * nper:(p + 1) * nper]
            Mpp = mobility.dense(rb, prm)
            L = np.linalg.cholesky(Mpp)
            Kp = rigid.K_matrix_body(rb, q[p])
            Minv = np.linalg.inv(Mpp)
            Np = np.linalg.inv(Kp.T @ Minv @ Kp)
            self.L.append(L)
            self.Minv.append(Minv)
            self.N.append(Np)
            self.K.append(Kp)

    def _blocks(self, v):
        return mobility.soa_to_blob(v).reshape(self.nb, 3 * self.nper)

    def _unblocks(self, b):
        return mobility.blob_to_soa(b.reshape(-1))

    def L_apply(self, v):
        b = self._blocks(v)
        return self._unblocks(np.stack([self.L[p] @ b[p] for p in range(self.nb)]))

    def Linv_apply(self, v):
        b = self._blocks(v)
        return self._unblocks(np.stack([np.linalg.solve(self.L[p], b[p]) for p in range(self.nb)]))

    def LinvT_apply(self, v):
        b = self._blocks(v)
        return self._unblocks(np.stack([np.linalg.solve(self.L[p].T, b[p]) for p in range(self.nb)]))

    def saddle_solve(self, a, b):
        """Exact solve of the block-diagonal saddle system
        [M(pp) -K_p; -K_p^T 0][lam_p; U_p] = [a_p; b_p] for every body:
        U_p = -N_p (b_p + K_p^T M(pp)^-1 a_p), lam_p = M(pp)^-1 (a_p + K_p U_p)."""
        ab = self._blocks(a)
        lam = np.zeros_like(ab)
        U = np.zeros((self.nb, 6))
        for p in range(self.nb):
            Ma = self.Minv[p] @ ab[p]
            U[p] = -self.N[p] @ (b[p] + self.K[p].T @ Ma)
            lam[p] = self.Minv[p] @ (ab[p] + self.K[p] @ U[p])
        return self._unblocks(lam), U
