"""GPU test of the allocation-free matvec entry point.

rpbd_mobility_apply_f32_noalloc serves callers that must not call the CUDA
allocator (for example code running inside a host framework that owns all
device memory, or a real-time loop that cannot afford an allocation): it
keeps its scratch in a fixed device array compiled into the library.  This
test calls it through the C ABI twice in a row, with different inputs and
right-hand-side counts, and checks each result against the ordinary
workspace-based rpbd_mobility_apply within the FP32 parity tolerance
(relative 2-norm error <= 1e-5) and, on sampled rows, against the FP64
oracle.  A third call with the same sizes must leave the device's free memory
exactly as it was (nothing allocated, nothing freed).  It also checks the
size limit."""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import mobility as om
from paper_1709_02410_gb300 import Handle, _native, synth

from gpu_util import DEV, positions, rel2, to_dev

pytestmark = pytest.mark.gpu


def _call(lib, prm, r, F, U, k, n=None):
    return lib.rpbd_mobility_apply_f32_noalloc(C.byref(prm), r.shape[1] if n is None else n,
                                               C.c_void_p(r.data_ptr()), C.c_void_p(F.data_ptr()),
                                               C.c_void_p(U.data_ptr()), k,
                                               C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_workspace_path_twice():
    lib = _native.load()
    s = synth.blobs_16384()           # 16,380 blobs, just under the 16,384 limit
    rh = positions(s)
    r = to_dev(rh)
    prm = _native.Params(synth.ETA, s.a, synth.KT, 1, 1e-3)
    h = Handle(synth.ETA, s.a, synth.KT)
    rows = np.random.default_rng(7).choice(s.n, 16, replace=False)
    for k, seed in ((16, 101), (3, 202)):
        Fh = synth.gaussian(seed, (k, 3, s.n), np.float32)
        F = to_dev(Fh, torch.float32)
        U = torch.full_like(F, float("nan"))
        assert _call(lib, prm, r, F, U, k) == 0
        ref = h.mobility_apply(r, F)
        torch.cuda.synchronize()
        U, ref = U.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(U).all()
        for m in range(k):
            assert rel2(U[m], ref[m]) <= 1e-5
        orc = om.apply(rh, Fh[:2].astype(np.float64), om.Params(synth.ETA, s.a), rows=rows)
        assert rel2(U[:2][:, :, rows], orc) <= 1e-5


def test_noalloc_allocates_nothing():
    lib = _native.load()
    s = synth.boomerang_suspension(300, 40.0, 8)
    r = to_dev(positions(s))
    prm = _native.Params(synth.ETA, s.a, synth.KT, 1, 1e-3)
    F = to_dev(synth.gaussian(303, (4, 3, s.n), np.float32), torch.float32)
    U = torch.empty_like(F)
    assert _call(lib, prm, r, F, U, 4) == 0   # the first call may load the kernels' code
    torch.cuda.synchronize()
    U1 = U.clone()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(lib, prm, r, F, U, 4) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(U, U1)  # deterministic: the same inputs give the same bits


def test_noalloc_rejects_oversize():
    lib = _native.load()
    prm = _native.Params(synth.ETA, 0.325, synth.KT, 1, 1e-3)
    n = 16385
    r = torch.zeros((3, n), dtype=torch.float64, device=DEV)
    F = torch.zeros((1, 3, n), dtype=torch.float32, device=DEV)
    U = torch.zeros_like(F)
    assert _call(lib, prm, r, F, U, 1) == -7
    r2 = torch.zeros((3, 8), dtype=torch.float64, device=DEV)
    F2 = torch.zeros((17, 3, 8), dtype=torch.float32, device=DEV)
    assert _call(lib, prm, r2, F2, torch.zeros_like(F2), 17) == -7
    assert lib.rpbd_status_string(-7).startswith(b"size beyond")
