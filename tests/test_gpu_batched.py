"""GPU parity of the batched path (many uneven suspensions in one launch)
against the oracle per system, the autotuner, and the graph-captured batched
Lanczos against the oracle's Lanczos per system."""
import numpy as np
import pytest
import torch

from oracle import krylov, mobility as om, precond, rigid
from paper_1709_02410_gb300 import synth

from gpu_util import DEV, handle_for, oracle_params, rel2, to_dev

pytestmark = pytest.mark.gpu


def batch(counts, seed=0, box_per_body=2.5):
    systems = [synth.boomerang_suspension(c, max(4.0, np.sqrt(c) * box_per_body), seed * 100 + i)
               for i, c in enumerate(counts)]
    rs = [rigid.blob_positions(s.q, s.theta, s.shape) for s in systems]
    off = np.concatenate([[0], np.cumsum([r.shape[1] for r in rs])]).astype(np.int64)
    r = np.concatenate(rs, axis=1)
    return systems, rs, off, r


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("k", [1, 2, 3, 16])
def test_batched_matvec_matches_oracle_per_system(k, variant):
    """every tile variant (3: two targets per thread, packed FP32; 4: the packed
    symmetric kernel per system, k > 4 on variant 3), systems of 1 to 600
    blobs (ragged against the 256-blob home tile and the 256-target tile)"""
    systems, rs, off, r = batch([1, 2, 9, 40, 3])
    h = handle_for(systems[0])
    h.set_batch_variant(variant)
    F = synth.gaussian(5 + k, (k, 3, r.shape[1]), np.float32)
    U = h.mobility_apply_batched(off, to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    for s, (sy, rr) in enumerate(zip(systems, rs)):
        sl = slice(off[s], off[s + 1])
        ref = om.apply(rr, F[:, :, sl].astype(np.float64), oracle_params(sy))
        assert rel2(U[:, :, sl], ref) <= 1e-5


def test_autotune_and_variants_agree():
    """the default tile and the autotuned one both match the oracle; they
    differ only by FP32 rounding (the packed tile works in units of a)"""
    systems, rs, off, r = batch([30, 7, 64, 100, 12], seed=1)
    h = handle_for(systems[0])
    rd = to_dev(r)
    Fh = synth.gaussian(9, (1, 3, r.shape[1]), np.float32)
    F = to_dev(Fh, torch.float32)
    U0 = h.mobility_apply_batched(off, rd, F).cpu().numpy()
    v, ms = h.autotune_batched(off, rd, 1)
    assert 0 <= v <= 4 and ms > 0
    U1 = h.mobility_apply_batched(off, rd, F).cpu().numpy()
    assert rel2(U1, U0) <= 5e-6
    for s, (sy, rr) in enumerate(zip(systems, rs)):
        sl = slice(off[s], off[s + 1])
        ref = om.apply(rr, Fh[:, :, sl].astype(np.float64), oracle_params(sy))
        assert rel2(U0[:, :, sl], ref) <= 1e-5 and rel2(U1[:, :, sl], ref) <= 1e-5


@pytest.mark.parametrize("variant", [-1, 4])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_lanczos_matches_oracle(use_graph, variant):
    """default tile and the symmetric variant, eager and graph-replayed"""
    counts = [3, 11, 25, 6]
    systems, rs, off, r = batch(counts, seed=2)
    h = handle_for(systems[0])
    h.set_batch_variant(variant)
    rd = to_dev(r)
    # block preconditioner over all bodies of the batch (bodies never couple systems)
    q = np.concatenate([s.q for s in systems])
    h.precond_build(15, rd, to_dev(q))
    W = synth.gaussian(11, (3, r.shape[1]))
    F = synth.gaussian(12, (3, r.shape[1]))
    out, U, iters = h.lanczos_sqrt_apply_batched(off, rd, to_dev(W), tol=1e-5, max_iter=60, use_graph=use_graph,
                                                 F=to_dev(F))
    if use_graph:      # replay the captured graph on new inputs
        W = synth.gaussian(13, (3, r.shape[1]))
        out, U, iters = h.lanczos_sqrt_apply_batched(off, rd, to_dev(W), tol=1e-5, max_iter=60, use_graph=True,
                                                     F=to_dev(F))
    out, U = out.cpu().numpy(), U.cpu().numpy()
    for s, (sy, rr) in enumerate(zip(systems, rs)):
        sl = slice(off[s], off[s + 1])
        prm = oracle_params(sy)
        pc = precond.BlockPrecond(rr, sy.q, sy.nper, prm)
        G = lambda v: pc.Linv_apply(om.apply(rr, pc.LinvT_apply(v), prm))
        y, it, ch = krylov.lanczos_sqrt(G, W[:, sl], 1e-5, 60)
        ref = pc.L_apply(y)
        assert abs(iters[s] - it) <= 1
        assert rel2(out[:, sl], ref) <= 1e-4
        assert rel2(U[:, sl], om.apply(rr, F[:, sl], prm)) <= 1e-5


def test_graph_replay_after_the_single_system_workspace_grows():
    """A captured one-system batched Lanczos keeps working after an ordinary
    matvec on a larger suspension has regrown the handle's single-system
    buffers: the batched path owns its own buffers (and the graph cache checks
    them), so the replay reads no freed memory and matches the eager run."""
    systems, rs, off, r = batch([20], seed=3)
    h = handle_for(systems[0])
    h.set_batch_variant(4)
    rd = to_dev(r)
    h.precond_build(15, rd, to_dev(systems[0].q))
    W = to_dev(synth.gaussian(14, (3, r.shape[1])))
    F = to_dev(synth.gaussian(15, (3, r.shape[1])))
    ref, Uref, it_ref = h.lanczos_sqrt_apply_batched(off, rd, W, tol=1e-5, max_iter=60, use_graph=False, F=F)
    ref, Uref = ref.clone(), Uref.clone()
    h.lanczos_sqrt_apply_batched(off, rd, W, tol=1e-5, max_iter=60, use_graph=True, F=F)  # capture
    big = synth.boomerang_suspension(400, 60.0, 9)
    rb = to_dev(rigid.blob_positions(big.q, big.theta, big.shape))
    for k in (1, 2, 16):  # every single-system buffer grows past the batch's size
        h.mobility_apply(rb, to_dev(synth.gaussian(16 + k, (k, 3, big.n), np.float32), torch.float32))
    out, U, it = h.lanczos_sqrt_apply_batched(off, rd, W, tol=1e-5, max_iter=60, use_graph=True, F=F)
    assert it == it_ref
    assert rel2(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-13
    assert rel2(U.cpu().numpy(), Uref.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("k", [1, 2, 3])
def test_batched_symmetric_fixed_point_and_partials(k):
    """Batched variant 4 (the packed symmetric kernel over a batch): fixed
    point with one maximum force per system (the default) against the
    per-system partials, the oracle per system, and a bitwise repeat; one
    system's forces 1e6 times larger than the rest, so a shared scale would
    cost the small systems their accuracy."""
    rng = np.random.default_rng(600 + k)
    sizes = [1, 255, 257, 700, 2049, 31]
    rs, Fs = [], []
    for i, n in enumerate(sizes):
        box = max(2.0, np.sqrt(n))
        rs.append(np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)]))
        Fs.append(rng.standard_normal((k, 3, n)) * (1e6 if i == 3 else 1.0))
    r = np.concatenate(rs, axis=1)
    F = np.concatenate(Fs, axis=2).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    h.set_batch_variant(4)
    rd, Fd = to_dev(r), to_dev(F, torch.float32)
    Ufx = h.mobility_apply_batched(off, rd, Fd).cpu().numpy()
    assert np.array_equal(Ufx, h.mobility_apply_batched(off, rd, Fd).cpu().numpy())
    h.set_sym_partials(True)
    Upt = h.mobility_apply_batched(off, rd, Fd).cpu().numpy()
    for i in range(len(sizes)):
        sl = slice(off[i], off[i + 1])
        Uo = om.apply(rs[i], F[:, :, sl].astype(np.float64), oracle_params(s))
        assert rel2(Ufx[:, :, sl], Uo) <= 1e-5, i
        assert rel2(Upt[:, :, sl], Uo) <= 1e-5, i
        assert rel2(Ufx[:, :, sl], Upt[:, :, sl]) <= 1e-6, i
