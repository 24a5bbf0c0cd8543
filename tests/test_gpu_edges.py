"""Degenerate inputs on a GPU: empty suspensions (n = 0) launch nothing and
return success, batches may hold empty systems and one-blob systems (every
batched variant against the oracle per system), and a lone blob's matvec is
its self mobility (the near-wall closed form of the pair block's self term)."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import mobility as om, rigid
from paper_1709_02410_gb300 import synth

from gpu_util import DEV, handle_for, oracle_params, rel2, to_dev

pytestmark = pytest.mark.gpu


def test_empty_suspension_launches_nothing():
    s = synth.boomerangs_1920()
    h = handle_for(s)
    r = torch.zeros((3, 0), dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    before = h.lib.rpbd_launch_count()
    for dt in (torch.float32, torch.float64):
        U = h.mobility_apply(r, torch.zeros((2, 3, 0), dtype=dt, device=DEV))
        assert U.shape == (2, 3, 0)
    g = h.mobility_adjoint(r, torch.zeros((3, 0), dtype=torch.float64, device=DEV),
                           torch.zeros((3, 0), dtype=torch.float64, device=DEV))
    assert g.shape == (3, 0)
    assert h.lib.rpbd_launch_count() == before


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_batch_with_empty_and_single_blob_systems(variant):
    counts = [0, 1, 0, 30, 1, 0]          # bodies of one blob each after slicing below
    systems = [synth.boomerang_suspension(max(c, 1), 6.0, 300 + i) for i, c in enumerate(counts)]
    rs = []
    for c, sy in zip(counts, systems):
        rr = rigid.blob_positions(sy.q, sy.theta, sy.shape)
        rs.append(rr[:, :c])              # 0, 1 or 30 blobs
    off = np.concatenate([[0], np.cumsum([x.shape[1] for x in rs])]).astype(np.int64)
    r = np.concatenate(rs, axis=1)
    h = handle_for(systems[0])
    h.set_batch_variant(variant)
    F = synth.gaussian(31, (2, 3, r.shape[1]), np.float32)
    U = h.mobility_apply_batched(off, to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    for s_, rr in enumerate(rs):
        if rr.shape[1] == 0:
            continue
        sl = slice(off[s_], off[s_ + 1])
        ref = om.apply(rr, F[:, :, sl].astype(np.float64), oracle_params(systems[0]))
        assert rel2(U[:, :, sl], ref) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lone_blob_is_its_self_mobility(dtype):
    """One blob at height h: U = mu(h) F with the near-wall self mobility
    mu_par = (1 - 9/16 x + 1/8 x^3 - 1/16 x^5) / (6 pi eta a),
    mu_perp = (1 - 9/8 x + 1/2 x^3 - 1/8 x^5) / (6 pi eta a), x = a / h."""
    s = synth.boomerangs_1920()
    a, eta = s.a, synth.ETA
    h = handle_for(s)
    for height in (1.0 * a, 1.7 * a, 5.0 * a):
        r = np.array([[0.3], [-0.2], [height]])
        F = np.array([[1.0], [-2.0], [0.5]])
        U = h.mobility_apply(to_dev(r), to_dev(F, dtype)).cpu().numpy().astype(np.float64)
        x = a / height
        mpar = (1 - 9 / 16 * x + x ** 3 / 8 - x ** 5 / 16) / (6 * np.pi * eta * a)
        mperp = (1 - 9 / 8 * x + x ** 3 / 2 - x ** 5 / 8) / (6 * np.pi * eta * a)
        ref = np.array([[mpar * 1.0], [mpar * -2.0], [mperp * 0.5]])
        assert rel2(U, ref) <= (1e-12 if dtype == torch.float64 else 1e-6)
