"""Full-size parity in the launch configurations the bench times: the
196,608-blob roller suspension (symmetric kernels at k = 1, 2, row-sampled),
and the 64-system uneven boomerang batch (471,495 blobs: the batched matvec
of the symmetric and the one-direction variants on sampled rows of every
system, and the graph-captured batched Lanczos over the whole batch checked
against the oracle's Lanczos on its smallest systems)."""
import numpy as np
import pytest
import torch

from oracle import krylov, mobility as om, precond, rigid
from paper_1709_02410_gb300 import synth

from gpu_util import DEV, handle_for, oracle_params, rel2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [1, 2])
def test_rollers_196608_row_sampled(k):
    s = synth.rollers_196608()
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    F = synth.gaussian(80 + k, (k, 3, s.n), np.float32)
    h = handle_for(s)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    h.close()
    rows = np.random.default_rng(81).choice(s.n, 32, replace=False)
    rows[0], rows[1] = 0, s.n - 1
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s), rows=rows)
    assert rel2(U[:, :, rows], Uo) <= 1e-5


def _batch():
    systems = synth.uneven_batch_64()
    rs = [rigid.blob_positions(sy.q, sy.theta, sy.shape) for sy in systems]
    off = np.concatenate([[0], np.cumsum([x.shape[1] for x in rs])]).astype(np.int64)
    return systems, rs, off, np.concatenate(rs, axis=1)


@pytest.mark.parametrize("variant", [3, 4])
def test_uneven_batch_471495_matvec_sampled(variant):
    systems, rs, off, r = _batch()
    assert off[-1] == 471495
    h = handle_for(systems[0])
    h.set_batch_variant(variant)
    F = synth.gaussian(82, (1, 3, r.shape[1]), np.float32)
    U = h.mobility_apply_batched(off, to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    h.close()
    rng = np.random.default_rng(83)
    for s, (sy, rr) in enumerate(zip(systems, rs)):
        n = rr.shape[1]
        rows = rng.choice(n, min(n, 4), replace=False)
        rows[0] = n - 1
        Fs = F[:, :, off[s]:off[s + 1]].astype(np.float64)
        Uo = om.apply(rr, Fs, oracle_params(sy), rows=rows)
        assert rel2(U[:, :, off[s] + rows], Uo) <= 1e-5, s


def test_uneven_batch_471495_lanczos_graph():
    """The graph-captured batched Lanczos over the whole 64-system batch.
    Checked on ten systems: the six smallest and the four nearest 4,000
    blobs.  Each system's answer is compared with the oracle's Lanczos run for
    exactly the same number of iterations (a tolerance it cannot reach), so
    both build the same Krylov space and differ only by the FP32 pair
    arithmetic of the GPU matvec (~1e-6 per apply, the FP32 parity level,
    propagated through a well-conditioned preconditioned operator): bound
    1e-4.  The stopping rule itself is checked on the three smallest systems:
    the oracle stops at tol = 1e-4 within one iteration of the GPU."""
    systems, rs, off, r = _batch()
    h = handle_for(systems[0])
    rd = to_dev(r)
    q = np.concatenate([sy.q for sy in systems])
    h.precond_build(15, rd, to_dev(q))
    W = synth.gaussian(84, (3, r.shape[1]))
    F = synth.gaussian(85, (3, r.shape[1]))
    out, U, iters = h.lanczos_sqrt_apply_batched(off, rd, to_dev(W), tol=1e-4, max_iter=60, use_graph=True,
                                                 F=to_dev(F))
    out, U = out.cpu().numpy(), U.cpu().numpy()
    h.close()
    assert all(1 <= it <= 60 for it in iters)
    sizes = np.array([rr.shape[1] for rr in rs])
    order = np.argsort(sizes)
    near4k = [s for s in np.argsort(np.abs(sizes - 4000)) if s not in order[:6]][:4]
    for rank, s in enumerate(list(order[:6]) + near4k):
        sy, rr = systems[s], rs[s]
        sl = slice(off[s], off[s + 1])
        prm = oracle_params(sy)
        pc = precond.BlockPrecond(rr, sy.q, sy.nper, prm)
        G = lambda v: pc.Linv_apply(om.apply(rr, pc.LinvT_apply(v), prm))
        y, it, _ = krylov.lanczos_sqrt(G, W[:, sl], 0.0, iters[s])
        assert it == iters[s]
        assert rel2(out[:, sl], pc.L_apply(y)) <= 1e-4, s
        assert rel2(U[:, sl], om.apply(rr, F[:, sl], prm)) <= 1e-5, s
        if rank < 3:
            _, it_tol, _ = krylov.lanczos_sqrt(G, W[:, sl], 1e-4, 60)
            assert abs(iters[s] - it_tol) <= 1, s


def test_boomerangs_65535_gmres_residual_sampled():
    """The saddle solve at full size in the bench's configuration (65,535
    boomerang blobs, FP32 pairs, GMRES tol 1e-6, restart 100, block-diagonal
    preconditioner), checked on 48 sampled bodies (720 blob rows) with the
    oracle: the velocity rows M lambda - K U + slip (oracle M lambda in FP64
    over all sources) and the force and torque balance K^T lambda = F.  The
    FP32 operator agrees with the oracle to ~1e-6 of |M lambda|, so the first
    residual is bounded by the FP32 parity tolerance (1e-5 of the sampled
    |M lambda|) plus GMRES's own 1e-6 |b|; the balance, formed in FP64, by
    the GMRES tolerance."""
    from paper_1709_02410_gb300 import F32
    s = synth.boomerangs_65535()
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    h = handle_for(s)
    FT = synth.gaussian(71, (s.nb, 6)) * 1e-2
    slip = synth.gaussian(72, (3, s.n)) * 1e-3
    lam, U, st = h.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), to_dev(slip), to_dev(FT), tol=1e-6,
                                     max_iter=300, restart=100, dtype=F32)
    assert st["status"] == 0, st
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    nper = s.nper
    bodies = np.sort(np.random.default_rng(73).choice(s.nb, 48, replace=False))
    rows = np.concatenate([np.arange(p * nper, (p + 1) * nper) for p in bodies])
    Ml = om.apply(r, lam, oracle_params(s), rows=rows)
    KU = np.concatenate([rigid.K_apply(r[:, p * nper:(p + 1) * nper], s.q[p:p + 1], U[p:p + 1], nper)
                         for p in bodies], axis=1)
    b_norm = np.sqrt(np.sum(slip ** 2) + np.sum(FT ** 2))
    res = Ml - KU + slip[:, rows]
    print(f"velocity rows: |res| {np.linalg.norm(res):.3e}, bound {1e-5 * np.linalg.norm(Ml) + 1e-6 * b_norm:.3e}")
    assert np.linalg.norm(res) <= 1e-5 * np.linalg.norm(Ml) + 1e-6 * b_norm
    KTl = np.concatenate([rigid.KT_apply(r[:, p * nper:(p + 1) * nper], s.q[p:p + 1],
                                         lam[:, p * nper:(p + 1) * nper], nper) for p in bodies])
    print(f"balance: |K^T lam - F| {np.linalg.norm(KTl - FT[bodies]):.3e}, bound {1e-5 * b_norm:.3e}")
    assert np.linalg.norm(KTl - FT[bodies]) <= 1e-5 * b_norm


def test_boomerangs_65535_lanczos_norm_identity():
    """The preconditioned Lanczos at full size in the bench's configuration
    (65,535 boomerang blobs, FP32 pairs, tol 1e-4): its output y = L G^{1/2} W
    with G = L^-1 M L^-T must satisfy |L^-1 y|^2 = W^T G W = z^T M z with
    z = L^-T W, a property that holds at any size.  L from the oracle's
    block preconditioner, M z from the FP64 matvec (pinned to the oracle at
    1e-12 elsewhere).  A relative error ~tol in y gives ~2 tol in the squared
    norm: bound 1e-3; a wrong factor or scale is off by O(1)."""
    from paper_1709_02410_gb300 import F32
    s = synth.boomerangs_65535()
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    h = handle_for(s)
    rd = to_dev(r)
    h.precond_build(s.nper, rd, to_dev(s.q))
    W = synth.gaussian(74, (3, s.n))
    y, st = h.lanczos_sqrt_apply(rd, to_dev(W), tol=1e-4, max_iter=60, dtype=F32)
    assert st["status"] == 0, st
    pc = precond.BlockPrecond(r, s.q, s.nper, oracle_params(s))
    u = pc.Linv_apply(y.cpu().numpy())
    z = pc.LinvT_apply(W)
    Mz = h.mobility_apply(rd, to_dev(z)).cpu().numpy()
    zMz = float(np.sum(z * Mz))
    print(f"|L^-1 y|^2 / z^T M z - 1 = {float(np.sum(u * u)) / zMz - 1:.3e} ({st['iterations']} iterations)")
    assert abs(float(np.sum(u * u)) - zMz) <= 1e-3 * zMz
