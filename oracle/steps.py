"""Oracle time steps (FP64).  TEST INFRASTRUCTURE.

Algorithm 1 (EM-T, Sec. 3.1), Algorithm 2 (T-S, Sec. 3.2), Algorithm 3
(EM-RFD, App. A) and the trapezoidal-traction variant T-T (Sec. 3.2) written
in the paper's order and notation.  Random vectors are inputs; the caller draws them
(from oracle.philox to match the CUDA library's internal draws).

Solvers: mode="dense" uses the exact Schur solution (eq. sysDense) and the
exact limit of the preconditioned Lanczos iteration, L (L^-1 M L^-T)^{1/2} W;
mode="iterative" uses oracle.krylov with the given tolerances.

Readings where the paper is silent:
  * forces F(Q): per-blob gravity -w z^, blob-wall Yukawa repulsion
    U(h) = gamma exp(-h/b)/h on h = max(z, h_floor) (Sec. 4.1 uses this
    potential for the wall), and one constant torque on every body (Sec. 4.3);
  * Q +/- for the RFD: q +/- (delta/2) dq, theta rotated by +/- (delta/2) dw;
  * Q + dt U for quaternions: theta <- Rotate(theta, dt omega) (App. B.1).
"""
from dataclasses import dataclass

import numpy as np
import scipy.linalg

from . import krylov, mobility, precond, rigid, saddle


@dataclass
class ForceModel:
    weight: float = 0.0          # gravity per blob, along -z
    wall_gamma: float = 0.0      # Yukawa strength of the blob-wall repulsion
    wall_b: float = 1.0          # Yukawa (Debye) length
    h_floor: float = 0.1         # repulsion evaluated at max(z, h_floor)
    torque: tuple = (0.0, 0.0, 0.0)
    steric_gamma: float = 0.0    # blob-blob Yukawa between blobs of different bodies
    steric_b: float = 1.0
    r_floor: float = 0.1         # blob-blob repulsion evaluated at max(r, r_floor)
    r_cut: float = 0.0           # pairs farther than r_cut are skipped (0: no cut)


def blob_forces(r, fm: ForceModel, nper=None):
    """Per-blob forces (Sec. 4.1): gravity, the Yukawa wall repulsion on the
    blob height, and (when steric_gamma != 0, nper given) the Yukawa
    repulsion U = gamma exp(-r/b)/r between blobs of different bodies."""
    f = np.zeros_like(r)
    h = np.maximum(r[2], fm.h_floor)
    if fm.wall_gamma != 0.0:
        f[2] += fm.wall_gamma * np.exp(-h / fm.wall_b) * (1.0 / (fm.wall_b * h) + 1.0 / (h * h))
    f[2] -= fm.weight
    if fm.steric_gamma != 0.0 and nper is not None:
        n = r.shape[1]
        body = np.arange(n) // nper
        for i in range(n):
            d = r[:, [i]] - r                      # from every blob j to blob i
            dist = np.sqrt(np.sum(d * d, axis=0))
            mask = body != body[i]
            if fm.r_cut > 0:
                mask &= dist <= fm.r_cut
            re = np.maximum(dist[mask], fm.r_floor)
            mag = fm.steric_gamma * np.exp(-re / fm.steric_b) * (1.0 / (fm.steric_b * re) + 1.0 / (re * re))
            f[:, i] += np.sum(d[:, mask] / np.maximum(dist[mask], 1e-300) * mag, axis=1)
    return f


def body_forces(r, q, nper, fm: ForceModel):
    FT = rigid.KT_apply(r, q, blob_forces(r, fm, nper), nper)
    FT[:, 3:] += np.asarray(fm.torque)
    return FT


class Solver:
    def __init__(self, mode="dense", tol_gmres=1e-10, tol_lanczos=1e-10, max_iter=200, restart=50):
        self.mode, self.tol_gmres, self.tol_lanczos = mode, tol_gmres, tol_lanczos
        self.max_iter, self.restart = max_iter, restart

    def saddle(self, r, q, nper, prm, slip, F):
        if self.mode == "dense":
            lam, U, _ = saddle.dense_solution(r, q, nper, prm, slip, F)
            return lam, U
        S = saddle.Saddle(r, q, nper, prm)
        lam, U, it, rel = S.solve(slip, F, self.tol_gmres, self.restart, self.max_iter)
        return lam, U

    def sqrtM(self, r, q, nper, prm, W):
        pc = precond.BlockPrecond(r, q, nper, prm)
        if self.mode == "dense":
            n = r.shape[1]
            M = mobility.dense(r, prm)
            Lb = scipy.linalg.block_diag(*pc.L)
            G = np.linalg.solve(Lb, np.linalg.solve(Lb, M).T).T
            lam, Q = np.linalg.eigh(0.5 * (G + G.T))
            y = Q @ (np.sqrt(np.maximum(lam, 0)) * (Q.T @ mobility.soa_to_blob(W)))
            return mobility.blob_to_soa(Lb @ y)
        G = lambda v: pc.Linv_apply(mobility.apply(r, pc.LinvT_apply(v), prm))
        y, it, ch = krylov.lanczos_sqrt(G, W, self.tol_lanczos, self.max_iter)
        return pc.L_apply(y)


def _displace(q, theta, dQ, scale):
    return q + scale * dQ[:, :3], rigid.rotate(theta, scale * dQ[:, 3:])


def step_ts(q, theta, shape, prm, fm, dt, delta, Lp, Ws, W, solver: Solver, kT):
    """Algorithm 2 (T-S).  Ws, W: blob-level standard normals [3, n].
    Returns (q_new, theta_new, info)."""
    nper = shape.shape[0]
    r = rigid.blob_positions(q, theta, shape)
    # 1a: W^D = L_p W^s, W^F = kT / L_p W^s
    WD = Lp * Ws
    WF = (kT / Lp) * Ws
    # 1b: RFD displacement problem  [M -K; -K^T 0][lam; dQ] = [-W^D; 0]
    _, dQ = solver.saddle(r, q, nper, prm, WD, None)
    # 1c: Q+- = Q +- delta/2 dQ
    qp, tp = _displace(q, theta, dQ, +0.5 * delta)
    qm, tm = _displace(q, theta, dQ, -0.5 * delta)
    rp = rigid.blob_positions(qp, tp, shape)
    rm = rigid.blob_positions(qm, tm, shape)
    # 1d: D^F, D^S
    DF = (rigid.KT_apply(rp, qp, WF, nper) - rigid.KT_apply(rm, qm, WF, nper)) / delta
    DS = (mobility.apply(rp, WF, prm) - mobility.apply(rm, WF, prm)) / delta
    # 2: M^{1/2} W
    MhW = solver.sqrtM(r, q, nper, prm, W)
    c = np.sqrt(2.0 * kT / dt)
    # 3: predictor solve
    Fn = body_forces(r, q, nper, fm)
    _, Un = solver.saddle(r, q, nper, prm, c * MhW, Fn)
    # 4: predicted configuration
    qt, tt = _displace(q, theta, Un, dt)
    rt = rigid.blob_positions(qt, tt, shape)
    # 5: corrector solve at Q~ with slip 2 D^S + c M^{1/2} W and force F~ - 2 D^F
    Ft = body_forces(rt, qt, nper, fm)
    _, Ut = solver.saddle(rt, qt, nper, prm, 2.0 * DS + c * MhW, Ft - 2.0 * DF)
    # 6: trapezoidal update
    qn, tn = _displace(q, theta, 0.5 * (Un + Ut), dt)
    return qn, tn, dict(dQ=dQ, DF=DF, DS=DS, MhW=MhW, Un=Un, Ut=Ut)


def step_emt(q, theta, shape, prm, fm, dt, delta, Lp, Wf, Wt, W, solver: Solver, kT):
    """Algorithm 1 (EM-T).  Wf, Wt: body-level normals [nb, 3]; W: blob [3, n]."""
    nper = shape.shape[0]
    r = rigid.blob_positions(q, theta, shape)
    # 1a: W^FT = kT [W^f / L_p; W^tau]
    WFT = kT * np.concatenate([Wf / Lp, Wt], axis=1)
    # 1b: RFD mobility problem [M -K; -K^T 0][lam; U] = [0; -W^FT]
    lamR, UR = solver.saddle(r, q, nper, prm, None, WFT)
    # 1c: Q+- = Q +- delta/2 [L_p W^f; W^tau]
    dQ = np.concatenate([Lp * Wf, Wt], axis=1)
    qp, tp = _displace(q, theta, dQ, +0.5 * delta)
    qm, tm = _displace(q, theta, dQ, -0.5 * delta)
    rp = rigid.blob_positions(qp, tp, shape)
    rm = rigid.blob_positions(qm, tm, shape)
    # 1d: D^F, D^S
    DF = (rigid.KT_apply(rp, qp, lamR, nper) - rigid.KT_apply(rm, qm, lamR, nper)) / delta
    DS = ((mobility.apply(rp, lamR, prm) - mobility.apply(rm, lamR, prm))
          - (rigid.K_apply(rp, qp, UR, nper) - rigid.K_apply(rm, qm, UR, nper))) / delta
    # 2: M^{1/2} W
    MhW = solver.sqrtM(r, q, nper, prm, W)
    c = np.sqrt(2.0 * kT / dt)
    # 3: solve with slip D^S + c M^{1/2} W and force F - D^F
    Fn = body_forces(r, q, nper, fm)
    _, Un = solver.saddle(r, q, nper, prm, DS + c * MhW, Fn - DF)
    # 4: Euler-Maruyama update
    qn, tn = _displace(q, theta, Un, dt)
    return qn, tn, dict(lamR=lamR, UR=UR, DF=DF, DS=DS, MhW=MhW, Un=Un)


def step_emrfd(q, theta, shape, prm, fm, dt, delta, Lp, Wf, Wt, W, solver: Solver, kT):
    """Algorithm 3 (EM-RFD, App. A): RFD on N with two solves at Q+-."""
    nper = shape.shape[0]
    r = rigid.blob_positions(q, theta, shape)
    # 1a: W^FT = kT [W^f / L_p; W^tau]
    WFT = kT * np.concatenate([Wf / Lp, Wt], axis=1)
    # 1b: Q+- = Q +- delta/2 [L_p W^f; W^tau]
    dQ = np.concatenate([Lp * Wf, Wt], axis=1)
    qp, tp = _displace(q, theta, dQ, +0.5 * delta)
    qm, tm = _displace(q, theta, dQ, -0.5 * delta)
    rp = rigid.blob_positions(qp, tp, shape)
    rm = rigid.blob_positions(qm, tm, shape)
    # 1c: two mobility problems with force W^FT
    _, Up = solver.saddle(rp, qp, nper, prm, None, WFT)
    _, Um = solver.saddle(rm, qm, nper, prm, None, WFT)
    # 2: M^{1/2} W
    MhW = solver.sqrtM(r, q, nper, prm, W)
    c = np.sqrt(2.0 * kT / dt)
    # 3: slip c M^{1/2} W, force F^n
    Fn = body_forces(r, q, nper, fm)
    _, Un = solver.saddle(r, q, nper, prm, c * MhW, Fn)
    # 4: Q^{n+1} = Q^n + dt (U^n + (U+ - U-) / delta)
    qn, tn = _displace(q, theta, Un + (Up - Um) / delta, dt)
    return qn, tn, dict(Up=Up, Um=Um, MhW=MhW, Un=Un)


def step_tt(q, theta, shape, prm, fm, dt, delta, Lp, Wf, Wt, W, solver: Solver, kT):
    """Trapezoidal Traction (T-T, Sec. 3.2): D^F and D^S as in step 1 of
    Algorithm 1 without the U^RFD term, then the predictor-corrector of
    Algorithm 2 (steps 3-6) with those drifts."""
    nper = shape.shape[0]
    r = rigid.blob_positions(q, theta, shape)
    WFT = kT * np.concatenate([Wf / Lp, Wt], axis=1)
    lamR, UR = solver.saddle(r, q, nper, prm, None, WFT)
    dQ = np.concatenate([Lp * Wf, Wt], axis=1)
    qp, tp = _displace(q, theta, dQ, +0.5 * delta)
    qm, tm = _displace(q, theta, dQ, -0.5 * delta)
    rp = rigid.blob_positions(qp, tp, shape)
    rm = rigid.blob_positions(qm, tm, shape)
    DF = (rigid.KT_apply(rp, qp, lamR, nper) - rigid.KT_apply(rm, qm, lamR, nper)) / delta
    DS = (mobility.apply(rp, lamR, prm) - mobility.apply(rm, lamR, prm)) / delta
    MhW = solver.sqrtM(r, q, nper, prm, W)
    c = np.sqrt(2.0 * kT / dt)
    Fn = body_forces(r, q, nper, fm)
    _, Un = solver.saddle(r, q, nper, prm, c * MhW, Fn)
    qt, tt = _displace(q, theta, Un, dt)
    rt = rigid.blob_positions(qt, tt, shape)
    Ft = body_forces(rt, qt, nper, fm)
    _, Ut = solver.saddle(rt, qt, nper, prm, 2.0 * DS + c * MhW, Ft - 2.0 * DF)
    qn, tn = _displace(q, theta, 0.5 * (Un + Ut), dt)
    return qn, tn, dict(DF=DF, DS=DS, MhW=MhW, Un=Un, Ut=Ut)
