"""The binding and the multi-right-hand-side adjoint on a GPU.

* Every malformed argument (wrong dtype, shape, device or layout) raises
  RpbdError in the binding before any kernel is launched: the library's
  launch counter does not move.
* rpbd_mobility_adjoint_multi gives d(sum_m u_m^T M F_m)/dr, summed over the
  k right-hand-side pairs on the device, and the autograd backward uses it
  as one call; both are checked against the oracle's gradient summed over m
  (FP64 <= 1e-11, FP32 <= 1e-5 relative 2-norm)."""
import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import F32, F64, synth
from paper_1709_02410_gb300.api import RpbdError
from paper_1709_02410_gb300.autograd import mobility_apply

from gpu_util import DEV, handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def _small():
    s = synth.boomerang_suspension(12, 8.0, 41)
    return s, handle_for(s), positions(s)


def test_bad_arguments_raise_without_a_launch():
    s, h, r = _small()
    n = s.n
    rd = to_dev(r)
    F32v = torch.zeros((3, n), dtype=torch.float32, device=DEV)
    F64v = torch.zeros((3, n), dtype=torch.float64, device=DEV)
    bad_calls = [
        ("F float16", lambda: h.mobility_apply(rd, F32v.half())),
        ("F bfloat16", lambda: h.mobility_apply(rd, F32v.bfloat16())),
        ("F int32", lambda: h.mobility_apply(rd, torch.zeros((3, n), dtype=torch.int32, device=DEV))),
        ("F wrong n", lambda: h.mobility_apply(rd, torch.zeros((3, n - 1), dtype=torch.float32, device=DEV))),
        ("F wrong rank", lambda: h.mobility_apply(rd, torch.zeros((2, 2, 3, n), dtype=torch.float32, device=DEV))),
        ("F on the host", lambda: h.mobility_apply(rd, torch.zeros((3, n), dtype=torch.float32))),
        ("F strided", lambda: h.mobility_apply(rd, torch.zeros((n, 3), dtype=torch.float32, device=DEV).t())),
        ("out dtype", lambda: h.mobility_apply(rd, F32v, out=F64v)),
        ("out shape", lambda: h.mobility_apply(rd, F32v, out=torch.zeros((1, 3, n), dtype=torch.float32,
                                                                          device=DEV))),
        ("mixed mode F32 vectors", lambda: h.mobility_apply(rd, F32v, dtype=F32)),
        ("r float32", lambda: h.mobility_apply(rd.float(), F32v)),
        ("r shape", lambda: h.mobility_apply(rd.t().contiguous(), F32v)),
        ("adjoint u shape", lambda: h.mobility_adjoint(rd, torch.zeros((2, 3, n), dtype=torch.float64,
                                                                       device=DEV), F64v)),
        ("adjoint float32", lambda: h.mobility_adjoint(rd, F32v, F32v)),
        ("adjoint out shape", lambda: h.mobility_adjoint(rd, F64v, F64v, out=torch.zeros((3, n + 1),
                                                                                        dtype=torch.float64,
                                                                                        device=DEV))),
        ("lanczos W float32", lambda: h.lanczos_sqrt_apply(rd, F32v, tol=1e-4)),
        ("rfd W shape", lambda: h.rfd_drift(rd, F64v[:, :-1].contiguous(), 1e-6)),
        ("gmres FT shape", lambda: h.gmres_rigid_solve(s.nper, rd, to_dev(s.q), None,
                                                       torch.zeros((s.nb, 3), dtype=torch.float64, device=DEV))),
        ("bodies do not match r", lambda: h.K_apply(s.nper + 1, rd, to_dev(s.q),
                                                    torch.zeros((s.nb, 6), dtype=torch.float64, device=DEV))),
        ("batched F float64", lambda: h.mobility_apply_batched([0, n], rd, F64v)),
        ("batched offsets end", lambda: h.mobility_apply_batched([0, n - 3], rd, F32v)),
    ]
    torch.cuda.synchronize()
    before = h.lib.rpbd_launch_count()
    for what, call in bad_calls:
        with pytest.raises(RpbdError):
            call()
        assert h.lib.rpbd_launch_count() == before, what
    # and the handle works afterwards
    F = synth.gaussian(5, (3, n), np.float32)
    U = h.mobility_apply(rd, to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_adjoint_multi_matches_summed_oracle_gradient(k, dtype):
    s = synth.boomerang_suspension(30, 9.0, 43 + k, lift=False)   # some blobs below a
    r = positions(s)
    rng = np.random.default_rng(44 + k)
    u, F = rng.standard_normal((2, k, 3, s.n))
    h = handle_for(s)
    g = h.mobility_adjoint(to_dev(r), to_dev(u), to_dev(F), dtype=dtype).cpu().numpy()
    go = sum(om.grad(r, u[m], F[m], oracle_params(s)) for m in range(k))
    assert rel2(g, go) <= (1e-11 if dtype == F64 else 1e-5)


def test_autograd_k_rhs_single_call():
    s, h, r = _small()
    rng = np.random.default_rng(47)
    F = rng.standard_normal((3, 3, s.n))
    G = rng.standard_normal((3, 3, s.n))
    rd = to_dev(r).requires_grad_(True)
    Fd = to_dev(F).requires_grad_(True)
    U = mobility_apply(h, rd, Fd)
    torch.cuda.synchronize()
    before = h.lib.rpbd_launch_count()
    (U * to_dev(G)).sum().backward()
    torch.cuda.synchronize()
    # the k = 3 position gradient is one FP64 adjoint launch; dL/dF one matvec
    # (pack, pair kernel, reduction)
    assert h.lib.rpbd_launch_count() - before <= 1 + 3
    go = sum(om.grad(r, G[m], F[m], oracle_params(s)) for m in range(3))
    assert rel2(rd.grad.cpu().numpy(), go) <= 1e-11
    gF = np.stack([om.apply(r, G[m], oracle_params(s)) for m in range(3)])
    assert rel2(Fd.grad.cpu().numpy(), gF) <= 1e-12
