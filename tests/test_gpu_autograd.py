"""GPU: the autograd Function's backward (the adjoint kernel) against
torch.autograd.gradcheck and against the oracle gradient."""
import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import synth
from paper_1709_02410_gb300.autograd import mobility_apply

from gpu_util import handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def test_gradcheck_small():
    s = synth.boomerang_suspension(2, 3.0, 40)
    h = handle_for(s)
    r = to_dev(positions(s)).requires_grad_(True)
    F = to_dev(synth.gaussian(41, (3, s.n))).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda rr, ff: mobility_apply(h, rr, ff), (r, F), eps=1e-6, atol=1e-6,
                                    rtol=1e-5)


def test_backward_matches_oracle():
    s = synth.boomerang_suspension(20, 8.0, 42, lift=False)
    h = handle_for(s)
    rn = positions(s)
    r = to_dev(rn).requires_grad_(True)
    Fn = synth.gaussian(43, (2, 3, s.n))
    F = to_dev(Fn)
    G = synth.gaussian(44, (2, 3, s.n))
    U = mobility_apply(h, r, F)
    (U * to_dev(G)).sum().backward()
    ref = om.grad(rn, G[0], Fn[0], oracle_params(s)) + om.grad(rn, G[1], Fn[1], oracle_params(s))
    assert rel2(r.grad.cpu().numpy(), ref) <= 1e-11
