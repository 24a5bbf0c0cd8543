"""Oracle Krylov solvers (FP64, numpy).  TEST INFRASTRUCTURE.

lanczos_sqrt: the preconditioned Lanczos approximation of M^{1/2} W
  (Sec. 2.2; the paper cites the method and fixes the block Cholesky
  preconditioner L = M~^{1/2}, but prints no algorithm).  Reading: Lanczos on
  G = L^-1 M L^-T from v_1 = W/|W| with full reorthogonalisation;
  f(G) W ~ |W| V_m T_m^{1/2} e_1 with T_m^{1/2} from a symmetric eigen-
  decomposition; stop when |y_m - y_{m-1}| / |y_m| < tol; output L y_m, whose
  covariance is L G L^T = M.
gmres: right-preconditioned restarted GMRES(m) with modified Gram-Schmidt
  Arnoldi and Givens rotations, stopping on the relative residual of the
  unpreconditioned system (Sec. 2.1 solves eq. saddle this way with the
  block preconditioner of Sec. 2.2).
"""
import numpy as np


def lanczos_sqrt(apply_G, W, tol, max_iter):
    """Returns (y, iterations, last relative change). y ~ G^{1/2} W."""
    W = np.asarray(W, dtype=np.float64)
    shape = W.shape
    w0 = W.reshape(-1)
    beta0 = np.linalg.norm(w0)
    if beta0 == 0.0:
        return np.zeros(shape), 0, 0.0
    V = [w0 / beta0]
    alpha, beta = [], []
    c_prev = None
    change = np.inf
    m = 0
    for m in range(1, max_iter + 1):
        w = apply_G(V[-1].reshape(shape)).reshape(-1).astype(np.float64)
        a = float(w @ V[-1])
        w = w - a * V[-1]
        if m > 1:
            w = w - beta[-1] * V[-2]
        for v in V:                      # full reorthogonalisation
            w = w - (w @ v) * v
        alpha.append(a)
        b = float(np.linalg.norm(w))
        T = np.diag(alpha)
        for i in range(m - 1):
            T[i, i + 1] = T[i + 1, i] = beta[i]
        lam, Q = np.linalg.eigh(T)
        c = Q @ (np.sqrt(np.maximum(lam, 0.0)) * Q[0, :])
        if c_prev is not None:
            cp = np.zeros(m)
            cp[:m - 1] = c_prev
            change = np.linalg.norm(c - cp) / np.linalg.norm(c)
            if change < tol:
                break
        c_prev = c
        if b == 0.0 or m == max_iter:
            break
        beta.append(b)
        V.append(w / b)
    Vm = np.stack(V[:len(c)], axis=1)
    y = beta0 * (Vm @ c)
    return y.reshape(shape), m, change


def gmres(apply_A, apply_Pinv, b, tol, restart=50, max_iter=500):
    """Solve A x = b, right preconditioned: A P^-1 y = b, x = P^-1 y.
    Vectors are flat float64 arrays.  Returns (x, iterations, rel_residual)."""
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    total = 0
    rel = 1.0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= tol or total >= max_iter:
            break
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_used = 0
        for j in range(m):
            w = apply_A(apply_Pinv(V[j]))
            for i in range(j + 1):                  # modified Gram-Schmidt
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                      # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_used = j + 1
            rel = abs(g[j + 1]) / bnorm
            if rel <= tol or total >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), g[:j_used])
        x = x + apply_Pinv(V[:j_used].T @ y)
        if rel <= tol or total >= max_iter:
            r = b - apply_A(x)
            rel = np.linalg.norm(r) / bnorm
            break
    return x, total, rel
