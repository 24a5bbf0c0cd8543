"""Failure detection on a GPU without a fault: the pair kernels' bounded
waits for their source copies are made to run out on purpose.

With the handle's test option RPBD_OPT_TEST_STALL set, the pair kernels
leave the barrier of their first source stage without a copy (a barrier that
nothing completes) and wait on it with a short limit (about 0.1 ms).  The
kernel records the timeout in the handle's device flag, lets its copies that
are in flight land, and exits; the synchronising calls then return
RPBD_TIMEOUT.  After the option is cleared, the same handle must give
oracle-correct results again (no lost context, no stale flag)."""
import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import F32, F64, synth
from paper_1709_02410_gb300.api import RpbdError

from gpu_util import handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def _check_healthy(h, s, r):
    for dt, tol in ((torch.float32, 1e-5), (torch.float64, 1e-12)):
        F = synth.gaussian(3, (2, 3, s.n))
        U = h.mobility_apply(to_dev(r), to_dev(F, dt)).cpu().numpy()
        ref = om.apply(r, F.astype(np.float32).astype(np.float64) if dt == torch.float32 else F, oracle_params(s))
        assert rel2(U, ref) <= tol


@pytest.mark.parametrize("dtype", [F32, F64])
def test_lanczos_and_gmres_report_timeout_then_recover(dtype):
    s = synth.boomerang_suspension(40, 10.0, 51)
    r = positions(s)
    h = handle_for(s)
    rd = to_dev(r)
    W = to_dev(synth.gaussian(52, (3, s.n)))
    FT = to_dev(synth.gaussian(53, (s.nb, 6)) * 1e-2)
    h.precond_build(s.nper, rd, to_dev(s.q))
    h.set_test_stall(True)
    with pytest.raises(RpbdError, match="timed out"):
        h.lanczos_sqrt_apply(rd, W, tol=1e-4, max_iter=40, dtype=dtype)
    with pytest.raises(RpbdError, match="timed out"):
        h.gmres_rigid_solve(s.nper, rd, to_dev(s.q), None, FT, tol=1e-6, dtype=dtype)
    h.set_test_stall(False)
    torch.cuda.synchronize()
    _check_healthy(h, s, r)
    # the solvers run to convergence again on the same handle
    _, st = h.lanczos_sqrt_apply(rd, W, tol=1e-4, max_iter=40, dtype=dtype)
    assert st["status"] == 0
    _, _, st = h.gmres_rigid_solve(s.nper, rd, to_dev(s.q), None, FT, tol=1e-6, dtype=dtype)
    assert st["status"] == 0


def test_time_step_reports_timeout_then_recovers():
    from paper_1709_02410_gb300 import Forces, StepParams
    s = synth.boomerang_suspension(6, 6.0, 54)
    h = handle_for(s)
    shape = to_dev(s.shape)
    f = Forces(0.05, 0.0, 1.0, 0.1, (0.0, 0.0, 0.0), 0.0, 1.0, 0.1, 0.0)
    sp = StepParams(0.01, 1e-3, 14.7 * s.a, 1e-6, 1e-4, 200, 50, 60, F32, 7, 0, 0)
    q, th = to_dev(s.q), to_dev(s.theta)
    h.set_test_stall(True)
    with pytest.raises(RpbdError, match="timed out"):
        h.step_ts(shape, q.clone(), th.clone(), f, sp)
    h.set_test_stall(False)
    stats, status = h.step_ts(shape, q, th, f, sp)
    assert status == 0 and all(x["status"] == 0 for x in stats)
    assert torch.isfinite(q).all() and torch.isfinite(th).all()
    _check_healthy(h, s, positions(s))
