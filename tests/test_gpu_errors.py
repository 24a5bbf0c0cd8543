"""Error behaviour of the C ABI on a GPU: argument checks return RPBD_BAD_ARG,
non-finite positions in the synchronising calls return RPBD_BAD_INPUT, an
unconverged Lanczos run returns RPBD_NOT_CONVERGED with its last iterate, and
the handle stays usable after every error."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import F32, F64, synth
from paper_1709_02410_gb300.api import RpbdError

from gpu_util import DEV, handle_for, oracle_params, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def _setup():
    s = synth.boomerangs_1920()
    return s, handle_for(s), positions(s)


def _still_works(h, s, r):
    F = synth.gaussian(90, (1, 3, s.n), np.float32)
    U = h.mobility_apply(to_dev(r), to_dev(F, torch.float32)).cpu().numpy()
    assert rel2(U, om.apply(r, F.astype(np.float64), oracle_params(s))) <= 1e-5


def test_matvec_argument_checks():
    s, h, r = _setup()
    F = torch.zeros((17, 3, s.n), dtype=torch.float32, device=DEV)
    with pytest.raises(RpbdError, match="F: expected shape"):
        h.mobility_apply(to_dev(r), F)  # k = 17 > 16, caught by the binding
    # the library's own checks: k out of range, null pointers
    st = h.lib.rpbd_mobility_apply(h.h, s.n, C.c_void_p(to_dev(r).data_ptr()), C.c_void_p(F.data_ptr()),
                                   C.c_void_p(F.data_ptr()), 17, F32, None)
    assert st == -1 and b"k must be" in h.lib.rpbd_last_error(h.h)
    st = h.lib.rpbd_mobility_apply(h.h, s.n, None, None, None, 1, F64, None)
    assert st == -1 and b"null" in h.lib.rpbd_last_error(h.h)
    _still_works(h, s, r)


def test_batched_argument_checks():
    s, h, r = _setup()
    F = torch.zeros((1, 3, s.n), dtype=torch.float32, device=DEV)
    rd = to_dev(r)
    for off in ([0, 1000, 900, s.n], [5, s.n]):  # decreasing; not starting at 0
        with pytest.raises(RpbdError, match="offsets"):
            h.mobility_apply_batched(np.array(off, dtype=np.int64), rd, F)
        # the library rejects them too
        o = np.array(off, dtype=np.int64)
        st = h.lib.rpbd_mobility_apply_batched(h.h, o.size - 1, o.ctypes.data_as(C.c_void_p),
                                               C.c_void_p(rd.data_ptr()), C.c_void_p(F.data_ptr()),
                                               C.c_void_p(F.data_ptr()), 1, None)
        assert st == -1
    _still_works(h, s, r)


def test_non_finite_positions_in_solvers():
    s, h, r = _setup()
    rb = r.copy()
    rb[2, 17] = np.nan
    W = to_dev(synth.gaussian(91, (3, s.n)))
    with pytest.raises(RpbdError, match="bad input"):
        h.lanczos_sqrt_apply(to_dev(rb), W, tol=1e-4, max_iter=40, use_precond=False)
    rb[2, 17] = np.inf
    FT = to_dev(synth.gaussian(92, (s.nb, 6)) * 1e-2)
    with pytest.raises(RpbdError, match="bad input"):
        h.gmres_rigid_solve(s.nper, to_dev(rb), to_dev(s.q), None, FT, tol=1e-6, dtype=F32)
    _still_works(h, s, r)
    # and the solvers still run on good positions
    _, st = h.lanczos_sqrt_apply(to_dev(r), W, tol=1e-4, max_iter=40, use_precond=False)
    assert st["status"] == 0


def test_lanczos_not_converged_keeps_last_iterate():
    s, h, r = _setup()
    W = to_dev(synth.gaussian(93, (3, s.n)))
    y2, st2 = h.lanczos_sqrt_apply(to_dev(r), W, tol=1e-14, max_iter=2, use_precond=False)
    assert st2["status"] == -4 and st2["iterations"] == 2
    y3, st3 = h.lanczos_sqrt_apply(to_dev(r), W, tol=1e-14, max_iter=3, use_precond=False)
    # the iterate after two steps differs from the one after three by the reported change
    d = float(torch.linalg.norm(y3 - y2) / torch.linalg.norm(y3))
    assert abs(d - st3["residual"]) <= 1e-6 * max(1.0, d)
    with pytest.raises(RpbdError, match="bad argument"):
        h.lanczos_sqrt_apply(to_dev(r), W, tol=1e-4, max_iter=81, use_precond=False)
    _still_works(h, s, r)


def test_blob_forces_argument_checks():
    s, h, r = _setup()
    from paper_1709_02410_gb300 import Forces
    f = Forces(1.0, 0.0, 1.0, 0.1, (0.0, 0.0, 0.0), 1.0, 0.3, 0.1, 0.0)  # steric on: needs the bodies
    with pytest.raises(RpbdError, match="bad argument"):
        h.blob_forces(to_dev(r), f, nper=7)  # nper does not divide n
    bad = Forces(1.0, 0.0, 1.0, 0.1, (0.0, 0.0, 0.0), 1.0, -0.3, 0.1, 0.0)
    with pytest.raises(RpbdError, match="bad argument"):
        h.blob_forces(to_dev(r), bad, nper=s.nper)  # negative steric range
    _still_works(h, s, r)
