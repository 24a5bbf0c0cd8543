"""GPU parity of the pseudo-periodic suspension (Sec. 4.2: minimum image plus
the 8 nearest periodic images in x, y) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import mobility as om, saddle
from paper_1709_02410_gb300 import F32, F64, Handle, RpbdError, synth

from gpu_util import DEV, positions, rel2, to_dev

pytestmark = pytest.mark.gpu

L = 45.3   # the paper's 256-boomerang cell edge (Sec. 4.2)


def cell(nb, seed):
    s = synth.boomerang_suspension(nb, L, seed)
    return s, positions(s), om.Params(synth.ETA, s.a, Lx=L, Ly=L)


def handle(s):
    return Handle(synth.ETA, s.a, synth.KT, Lx=L, Ly=L)


@pytest.mark.parametrize("nb", [1, 3, 64])
def test_periodic_f64(nb):
    s, r, prm = cell(nb, 50 + nb)
    F = synth.gaussian(51, (2, 3, s.n))
    U = handle(s).mobility_apply(to_dev(r), to_dev(F)).cpu().numpy()
    assert rel2(U, om.apply(r, F, prm)) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 4, 16])
@pytest.mark.parametrize("sym,packed,variant", [(True, True, -1), (True, True, 4), (True, True, 5), (True, False, -1),
                                                (False, False, -1)])
def test_periodic_f32(k, sym, packed, variant):
    """FP32 in the periodic cell: packed symmetric kernel (default for k <= 4;
    variants 4, 5: four home blobs per thread), one-home symmetric kernel,
    one-direction kernel"""
    s, r, prm = cell(40, 52)
    F = synth.gaussian(53 + k, (k, 3, s.n), np.float32)
    h = handle(s)
    h.set_symmetric(sym)
    h.set_packed(packed)
    h.set_sym_variant(variant)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), prm)) <= 1e-5


def test_periodic_adjoint_and_divergence():
    s, r, prm = cell(12, 54)
    rng = np.random.default_rng(55)
    u, F = rng.standard_normal((2, 3, s.n))
    h = handle(s)
    g = h.mobility_adjoint(to_dev(r), to_dev(u), to_dev(F)).cpu().numpy()
    assert rel2(g, om.grad(r, u, F, prm)) <= 1e-11
    d = h.mobility_divergence(to_dev(r)).cpu().numpy()
    assert rel2(d, om.divergence(r, prm)) <= 1e-10
    g32 = h.mobility_adjoint(to_dev(r), to_dev(u), to_dev(F), dtype=F32).cpu().numpy()
    assert rel2(g32, om.grad(r, u, F, prm)) <= 1e-5


def test_periodic_gmres():
    s, r, prm = cell(10, 56)
    FT = synth.gaussian(57, (s.nb, 6)) * 1e-2
    lam_d, U_d, _ = saddle.dense_solution(r, s.q, s.nper, prm, None, FT)
    lam, U, st = handle(s).gmres_rigid_solve(s.nper, to_dev(r), to_dev(s.q), None, to_dev(FT), tol=1e-12,
                                             max_iter=300, restart=60)
    assert st["status"] == 0
    assert rel2(U.cpu().numpy(), U_d) <= 1e-9


def test_periodic_argument_checks():
    with pytest.raises(RpbdError):
        Handle(synth.ETA, 0.325, Lx=L, Ly=0.0)
    with pytest.raises(RpbdError):
        Handle(synth.ETA, 0.325, wall=False, Lx=L, Ly=L)
    s, r, prm = cell(4, 58)
    h = handle(s)
    off = np.array([0, s.n], dtype=np.int64)
    F = torch.zeros((1, 3, s.n), dtype=torch.float32, device=DEV)
    with pytest.raises(RpbdError):
        h.mobility_apply_batched(off, to_dev(r), F)


@pytest.mark.parametrize("k", [1, 2])
def test_periodic_full_size_row_sampled(k):
    """The periodic cell at full size in the bench's configuration: the
    65,535-blob boomerang suspension in its own 233.7 um square cell (minimum
    image + 8 nearest images per pair), packed symmetric kernel with
    fixed-point accumulation; 64 sampled rows, the first and the last blob
    included, against the oracle's image sum."""
    s = synth.boomerangs_65535()
    Lc = 40.0 * np.sqrt(s.nb / 128)
    r = positions(s)
    F = synth.gaussian(510 + k, (k, 3, s.n), np.float32)
    h = Handle(synth.ETA, s.a, synth.KT, Lx=Lc, Ly=Lc)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    rows = np.random.default_rng(512).choice(s.n, 64, replace=False)
    rows[0], rows[1] = 0, s.n - 1
    Uo = om.apply(r, F.astype(np.float64), om.Params(synth.ETA, s.a, Lx=Lc, Ly=Lc), rows=rows)
    assert rel2(U[:, :, rows], Uo) <= 1e-5
