"""Accuracy of single FP32 pair blocks by distance band.

Far from the target, the direct RPY term and the image system above the wall
agree in their leading digits (each ~1/r) while their sum is only
O(zi zj / r^3), so a block formed from the two in FP32 loses digits in
proportion to r^2 / (zi zj).  The matvec's rows hardly notice (such blocks
are tiny next to the near ones), so this is measured block by block:

one source blob carries the unit forces e_x, e_y, e_z (three right-hand
sides) and every other blob carries none, so each other blob's velocity is
one column of its block with the source.  Blobs sit in bands of horizontal
distance rho / a from 2.5 to 2,500, heights a + Exp(1.5 a); the oracle forms
the same blocks in FP64.  With the far-field mode (RPBD_OPT_FARFIELD: the
direct-minus-image differences written without cancellation) every band
stays within 1e-5 relative (Frobenius norm of the block; measured ~5e-7);
the default form stays within 1e-5 inside 10 a and degrades beyond, as
eps32 rho^2 / (zi zj) predicts (printed with -s, not bounded)."""
import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import synth

from gpu_util import handle_for, oracle_params, rel2, to_dev

pytestmark = pytest.mark.gpu

BANDS = [(2.5, 5), (5, 10), (10, 30), (30, 100), (100, 300), (300, 1000), (1000, 2500)]
PER_BAND = 150


def _blocks(far, z0_over_a, seed):
    a = synth.A_BOOMERANG
    rng = np.random.default_rng(seed)
    rho = np.concatenate([rng.uniform(lo, hi, PER_BAND) for lo, hi in BANDS]) * a
    ang = rng.uniform(0, 2 * np.pi, rho.size)
    z = a + rng.exponential(1.5 * a, rho.size)
    r = np.concatenate([[[0.0], [0.0], [z0_over_a * a]],
                        np.stack([rho * np.cos(ang), rho * np.sin(ang), z])], axis=1)
    n = r.shape[1]
    F = np.zeros((3, 3, n), dtype=np.float32)
    for c in range(3):
        F[c, c, 0] = 1.0
    s = synth.boomerang_suspension(1, 1.0, 0)   # parameters only (a, eta)
    h = handle_for(s)
    h.set_far_field(far)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy().astype(np.float64)
    Uo = om.apply(r, F.astype(np.float64), oracle_params(s))
    err = np.linalg.norm(U[:, :, 1:] - Uo[:, :, 1:], axis=(0, 1)) / np.linalg.norm(Uo[:, :, 1:], axis=(0, 1))
    return [float(err[b * PER_BAND:(b + 1) * PER_BAND].max()) for b in range(len(BANDS))]


@pytest.mark.parametrize("z0", [1.2, 2.5, 6.0])
def test_block_error_by_band(z0):
    acc = _blocks(True, z0, 90 + int(10 * z0))
    plain = _blocks(False, z0, 90 + int(10 * z0))
    for (lo, hi), e_acc, e_plain in zip(BANDS, acc, plain):
        print(f"z0 = {z0} a, rho/a in [{lo}, {hi}): far-field mode {e_acc:.2e}, default {e_plain:.2e}")
    assert max(acc) <= 1e-5
    # the default form holds to 1e-5 inside 10 a; beyond, its error grows like
    # eps32 rho^2 / (zi zj) (~5e-5 at 30 a for blobs near the wall), which the
    # far-field mode removes
    assert max(plain[:2]) <= 1e-5
    assert plain[-1] > 10 * acc[-1]


@pytest.mark.parametrize("k", [1, 2, 3, 16])
@pytest.mark.parametrize("n", [33, 700, 4500])
def test_far_field_mode_matvec_parity(k, n):
    """The far-field mode against the oracle at ragged sizes and every k
    (k > 4 in groups of four right-hand sides), blobs overlapping each other
    and the wall."""
    rng = np.random.default_rng(7 * n + k)
    box = max(2.0, np.sqrt(n))
    r = np.stack([rng.uniform(0, box, n), rng.uniform(0, box, n), rng.uniform(-0.2, 2.5, n)])
    F = rng.standard_normal((k, 3, n)).astype(np.float32)
    s = synth.boomerangs_1920()
    h = handle_for(s)
    h.set_far_field(True)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5
    Ud = h.mobility_apply(to_dev(r), to_dev(F.astype(np.float64)), dtype=1).cpu().numpy()  # FP64 vectors
    assert rel2(Ud, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


def test_far_field_mode_periodic_and_solver():
    s = synth.boomerang_suspension(40, 12.0, 5)
    from oracle import rigid, saddle
    r = rigid.blob_positions(s.q, s.theta, s.shape)
    prm = om.Params(synth.ETA, s.a, Lx=12.0, Ly=12.0)
    from paper_1709_02410_gb300 import Handle
    h = Handle(synth.ETA, s.a, synth.KT, Lx=12.0, Ly=12.0)
    h.set_far_field(True)
    F = synth.gaussian(6, (2, 3, s.n), np.float32)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), prm)) <= 1e-5
    h2 = handle_for(s)
    h2.set_far_field(True)
    FT = synth.gaussian(7, (s.nb, 6)) * 1e-2
    lam, Ub, st = h2.gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), None, to_dev(FT), tol=1e-6, dtype=1)
    _, Ud, _ = saddle.dense_solution(r, s.q, s.nper, oracle_params(s), None, FT)
    assert st["status"] == 0 and rel2(Ub.cpu().numpy(), Ud) <= 1e-4
