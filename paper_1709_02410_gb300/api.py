"""Torch-facing binding of the C ABI (argument marshalling only).

Tensors must be contiguous CUDA tensors on the handle's device; positions
are [3, n] float64 (SoA), blob vectors [k, 3, n] or [3, n], body vectors
[nb, 6], q [nb, 3], theta [nb, 4].  Calls run on torch's current stream.
"""
import ctypes as C

import torch

from . import _native
from ._native import F32, F64, Forces, Params, Stats, StepParams


class RpbdError(RuntimeError):
    pass


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise RpbdError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise RpbdError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, dtype, shape=None, name="tensor"):
    if t.dtype != dtype:
        raise RpbdError(f"{name}: expected {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise RpbdError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")


class Handle:
    """Owns an rpbd_handle (device workspace + physical parameters)."""

    def __init__(self, eta, a, kT=0.0, wall=True, s_min=1e-3, Lx=0.0, Ly=0.0):
        self.lib = _native.load()
        self.params = Params(eta, a, kT, int(bool(wall)), s_min, Lx, Ly)
        h = C.c_void_p()
        st = self.lib.rpbd_create(C.byref(h), C.byref(self.params))
        if st != 0:
            raise RpbdError(f"rpbd_create failed: {_native.STATUS.get(st, st)}")
        self.h = h

    def close(self):
        """Destroy the handle and free its device workspace (idempotent)."""
        if getattr(self, "h", None):
            self.lib.rpbd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.rpbd_last_error(self.h).decode(errors="replace")
            raise RpbdError(f"{what}: {_native.STATUS.get(st, st)}: {msg}")
        return st

    def set_batch_variant(self, v: int):
        """tile variant of the batched kernel (-1 default, 0..4; 3: packed two targets per thread;
        4: packed symmetric kernel for k <= 4)"""
        self._check(self.lib.rpbd_set_option(self.h, 4, int(v)), "set_option")

    def set_packed(self, on: bool):
        """k <= 4 symmetric matvecs with the wall: packed two-homes-per-thread kernel (default) or not."""
        self._check(self.lib.rpbd_set_option(self.h, 3, int(bool(on))), "set_option")

    def set_symmetric(self, on: bool):
        """FP32 matvecs with k <= 4: symmetric kernel (default) or one-direction."""
        self._check(self.lib.rpbd_set_option(self.h, 1, int(bool(on))), "set_option")

    def set_sym_variant(self, v: int):
        """Loop-unroll / occupancy variant 0..3 of the symmetric kernels (-1: the default)."""
        self._check(self.lib.rpbd_set_option(self.h, 2, int(v)), "set_option")

    def measure_fma_peak(self, dtype=F32):
        """FMA throughput of this GPU in TFLOP/s (FMA = 2), measured by the library."""
        v = C.c_double()
        self._check(self.lib.rpbd_measure_fma_peak(self.h, dtype, C.byref(v), _stream()), "measure_fma_peak")
        return v.value

    def autotune(self, r, k=1):
        """Pick the fastest FP32 kernel for this n and k; returns (choice, ms per launch)."""
        ms = C.c_double()
        c = self.lib.rpbd_autotune(self.h, r.shape[1], _ptr(r), k, C.byref(ms), _stream())
        if c < 0:
            self._check(c, "autotune")
        return c, ms.value

    # ---- a1
    def blobs_from_bodies(self, shape, q, theta, out=None):
        """Blob positions r = q_p + R(theta_p) s_i (Sec. 2.1) as [3, nb * nper] FP64 SoA."""
        nb, nper = q.shape[0], shape.shape[0]
        out = torch.empty((3, nb * nper), dtype=torch.float64, device=q.device) if out is None else out
        for t, n in ((shape, "shape"), (q, "q"), (theta, "theta")):
            _need(t, torch.float64, name=n)
        self._check(self.lib.rpbd_blobs_from_bodies(self.h, nb, nper, _ptr(shape), _ptr(q), _ptr(theta),
                                                    _ptr(out), _stream()), "blobs_from_bodies")
        return out

    # ---- a2
    def mobility_apply(self, r, F, dtype=None, out=None):
        """U = M(r) F.  F [k,3,n] or [3,n]; float64 -> FP64 kernel, float32 ->
        FP32 kernel.  dtype=F32 with float64 F runs FP32 pairs on FP64 vectors."""
        n = r.shape[1]
        _need(r, torch.float64, (3, n), "r")
        squeeze = F.dim() == 2
        k = 1 if squeeze else F.shape[0]
        out = torch.empty_like(F) if out is None else out
        if dtype is None:
            dt = F64 if F.dtype == torch.float64 else F32
            fn = self.lib.rpbd_mobility_apply
        else:
            dt = dtype
            if F.dtype != torch.float64:
                raise RpbdError("mixed mode needs float64 vectors")
            fn = self.lib.rpbd_mobility_apply_mixed
        self._check(fn(self.h, n, _ptr(r), _ptr(F), _ptr(out), k, dt, _stream()), "mobility_apply")
        return out

    # ---- a7
    def mobility_adjoint(self, r, u, F, out=None, dtype=F64):
        """d(u^T M(r) F)/dr, FP64 vectors; dtype F32 evaluates the pair derivative in FP32."""
        n = r.shape[1]
        out = torch.empty((3, n), dtype=torch.float64, device=r.device) if out is None else out
        fn = self.lib.rpbd_mobility_adjoint_f32 if dtype == F32 else self.lib.rpbd_mobility_adjoint
        self._check(fn(self.h, n, _ptr(r), _ptr(u), _ptr(F), _ptr(out), _stream()), "mobility_adjoint")
        return out

    def mobility_divergence(self, r, out=None):
        """div M (the thermal drift that the RFD of Sec. 3 estimates), exact, FP64, [3, n]."""
        n = r.shape[1]
        out = torch.empty((3, n), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_mobility_divergence(self.h, n, _ptr(r), _ptr(out), _stream()),
                    "mobility_divergence")
        return out

    # ---- rigid
    def K_apply(self, nper, r, q, U, out=None):
        """Blob velocities K U of rigid-body motions U [nb, 6] (Sec. 2.1), [3, n]."""
        nb = q.shape[0]
        out = torch.empty((3, nb * nper), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_K_apply(self.h, nb, nper, _ptr(r), _ptr(q), _ptr(U), _ptr(out), _stream()),
                    "K_apply")
        return out

    def KT_apply(self, nper, r, q, lam, out=None):
        """Total force and torque K^T lambda per body of blob forces lambda [3, n], [nb, 6]."""
        nb = q.shape[0]
        out = torch.empty((nb, 6), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_KT_apply(self.h, nb, nper, _ptr(r), _ptr(q), _ptr(lam), _ptr(out), _stream()),
                    "KT_apply")
        return out

    # ---- a3
    def precond_build(self, nper, r, q):
        """Build the body-block-diagonal preconditioner (Sec. 2.2) at r; kept until the next build."""
        self._check(self.lib.rpbd_precond_build(self.h, q.shape[0], nper, _ptr(r), _ptr(q), _stream()),
                    "precond_build")

    def precond_apply(self, mode, x, out=None):
        """Apply a stored factor per body: mode 0 L, 1 L^-1, 2 L^-T, 3 M~^-1."""
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.rpbd_precond_apply(self.h, mode, _ptr(x), _ptr(out), _stream()), "precond_apply")
        return out

    # ---- a4
    def lanczos_sqrt_apply(self, r, W, tol, max_iter=80, dtype=F64, use_precond=True, out=None):
        """M^{1/2} W by preconditioned Lanczos (Sec. 2.2); returns (out, stats).  A run that stops
        at max_iter returns its last iterate with stats status -4 (not converged)."""
        n = r.shape[1]
        out = torch.empty_like(W) if out is None else out
        st = Stats()
        s = self.lib.rpbd_lanczos_sqrt_apply(self.h, n, _ptr(r), _ptr(W), _ptr(out), tol, max_iter, dtype,
                                             int(bool(use_precond)), C.byref(st), _stream())
        if s not in (0, -4):
            self._check(s, "lanczos_sqrt_apply")
        return out, st.as_dict()

    # ---- a5
    def gmres_rigid_solve(self, nper, r, q, slip=None, FT=None, tol=1e-6, max_iter=200, restart=50, dtype=F64,
                          build_precond=True, x0=None):
        """x0 = (lambda0, U0): initial guess (GMRES warm start); default zero."""
        nb = q.shape[0]
        n = nb * nper
        if x0 is None:
            lam = torch.empty((3, n), dtype=torch.float64, device=r.device)
            U = torch.empty((nb, 6), dtype=torch.float64, device=r.device)
        else:
            lam, U = x0[0].clone(), x0[1].clone()
        st = Stats()
        s = self.lib.rpbd_gmres_rigid_solve(self.h, nb, nper, _ptr(r), _ptr(q), _ptr(slip), _ptr(FT), _ptr(lam),
                                            _ptr(U), tol, max_iter, restart, dtype, int(bool(build_precond)),
                                            int(x0 is not None), C.byref(st), _stream())
        if s not in (0, -4):
            self._check(s, "gmres_rigid_solve")
        return lam, U, st.as_dict()

    def lanczos_sqrt_apply_multi(self, r, Ws, tol=1e-4, max_iter=60, dtype=F64, use_precond=True):
        """1..4 Lanczos square roots M^{1/2} W at the same positions, in lockstep
        (shared multi-RHS matvecs).  Returns a list of (out, stats)."""
        n = r.shape[1]
        ns = len(Ws)
        outs = [torch.empty((3, n), dtype=torch.float64, device=r.device) for _ in range(ns)]
        arr = C.c_void_p * ns
        st = (Stats * ns)()
        s = self.lib.rpbd_lanczos_sqrt_apply_multi(self.h, n, _ptr(r), ns, arr(*[_ptr(w) for w in Ws]),
                                                   arr(*[_ptr(o) for o in outs]), tol, max_iter, dtype,
                                                   int(bool(use_precond)), st, _stream())
        if s not in (0, -4):
            self._check(s, "lanczos_sqrt_apply_multi")
        return [(o, st[i].as_dict()) for i, o in enumerate(outs)]

    def gmres_rigid_solve_multi(self, nper, r, q, problems, tol=1e-6, max_iter=200, restart=50, dtype=F64,
                                build_precond=True):
        """problems: list of 1..4 (slip, FT) pairs (either None) at the same
        positions; solved in lockstep with shared multi-RHS matvecs.  Returns a
        list of (lambda, U, stats)."""
        nb = q.shape[0]
        n = nb * nper
        ns = len(problems)
        outs = [(torch.empty((3, n), dtype=torch.float64, device=r.device),
                 torch.empty((nb, 6), dtype=torch.float64, device=r.device)) for _ in range(ns)]
        arr = C.c_void_p * ns
        slips = arr(*[_ptr(p[0]) for p in problems])
        fts = arr(*[_ptr(p[1]) for p in problems])
        lams = arr(*[_ptr(o[0]) for o in outs])
        us = arr(*[_ptr(o[1]) for o in outs])
        st = (Stats * ns)()
        s = self.lib.rpbd_gmres_rigid_solve_multi(self.h, nb, nper, _ptr(r), _ptr(q), ns, slips, fts, lams, us, tol,
                                                  max_iter, restart, dtype, int(bool(build_precond)), st, _stream())
        if s not in (0, -4):
            self._check(s, "gmres_rigid_solve_multi")
        return [(o[0], o[1], st[i].as_dict()) for i, o in enumerate(outs)]

    # ---- a6
    def rfd_drift(self, r, W, delta, dtype=F64, out=None):
        """Blob-level centred RFD (Sec. 3): [M(r + delta/2 W) - M(r - delta/2 W)] W / delta; mean div M."""
        n = r.shape[1]
        out = torch.empty_like(W) if out is None else out
        self._check(self.lib.rpbd_rfd_drift(self.h, n, _ptr(r), _ptr(W), delta, _ptr(out), dtype, _stream()),
                    "rfd_drift")
        return out

    # ---- batched suspensions
    @staticmethod
    def _offsets(offsets):
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        return off, off.ctypes.data_as(C.c_void_p)

    def mobility_apply_batched(self, offsets, r, F, out=None):
        """U = M(r_s) F_s for independent systems concatenated at blob offsets (FP32 [k, 3, n])."""
        off, op = self._offsets(offsets)
        n_sys = off.size - 1
        k = 1 if F.dim() == 2 else F.shape[0]
        _need(F, torch.float32, name="F")
        out = torch.empty_like(F) if out is None else out
        self._check(self.lib.rpbd_mobility_apply_batched(self.h, n_sys, op, _ptr(r), _ptr(F), _ptr(out), k,
                                                         _stream()), "mobility_apply_batched")
        return out

    def autotune_batched(self, offsets, r, k=1):
        """Time the batched variants on this batch and keep the fastest; returns (variant, ms)."""
        off, op = self._offsets(offsets)
        ms = C.c_double()
        v = self.lib.rpbd_autotune_batched(self.h, off.size - 1, op, _ptr(r), k, C.byref(ms), _stream())
        if v < 0:
            self._check(v, "autotune_batched")
        return v, ms.value

    def lanczos_sqrt_apply_batched(self, offsets, r, W, tol, max_iter=40, use_precond=True, use_graph=True,
                                   F=None, out=None, U=None):
        """One preconditioned Lanczos M^{1/2} W per system of a batch, in lockstep (one CUDA graph when
        use_graph), and optionally U = M F per system; returns (out, U, iterations per system)."""
        off, op = self._offsets(offsets)
        n_sys = off.size - 1
        out = torch.empty_like(W) if out is None else out
        if F is not None and U is None:
            U = torch.empty_like(F)
        iters = (C.c_int * n_sys)()
        self._check(self.lib.rpbd_lanczos_sqrt_apply_batched(self.h, n_sys, op, _ptr(r), _ptr(W), _ptr(out), _ptr(F),
                                                             _ptr(U), tol, max_iter, int(bool(use_precond)),
                                                             int(bool(use_graph)), iters, _stream()),
                    "lanczos_sqrt_apply_batched")
        return out, U, list(iters)

    # ---- random numbers
    def philox_normals(self, n, seed, step, sid, device="cuda"):
        """n N(0,1) draws of Philox4x32-10 keyed by (seed, step, stream id), as the time steps draw them."""
        out = torch.empty(n, dtype=torch.float64, device=device)
        self._check(self.lib.rpbd_philox_normals(self.h, seed, step, sid, n, _ptr(out), _stream()),
                    "philox_normals")
        return out

    # ---- a8
    def _step(self, fn, nstats, shape, q, theta, forces: Forces, sp: StepParams):
        st = (Stats * nstats)()
        s = fn(self.h, q.shape[0], shape.shape[0], _ptr(shape), _ptr(q), _ptr(theta), C.byref(forces),
               C.byref(sp), st, _stream())
        if s not in (0, -4):
            self._check(s, "step")
        return [x.as_dict() for x in st], s

    def step_ts(self, shape, q, theta, forces, sp):
        """One trapezoidal-slip step (Alg. 2) in place on q, theta; returns (statistics per solve, status)."""
        return self._step(self.lib.rpbd_step_ts, 4, shape, q, theta, forces, sp)

    def step_emt(self, shape, q, theta, forces, sp):
        """One Euler-Maruyama traction step (Alg. 1) in place on q, theta; returns (statistics per solve, status)."""
        return self._step(self.lib.rpbd_step_emt, 3, shape, q, theta, forces, sp)

    def step_emrfd(self, shape, q, theta, forces, sp):
        """One Euler-Maruyama RFD step (Alg. 3, App. A) in place on q, theta; returns (statistics per solve, status)."""
        return self._step(self.lib.rpbd_step_emrfd, 4, shape, q, theta, forces, sp)

    def step_tt(self, shape, q, theta, forces, sp):
        """One trapezoidal traction step (Sec. 3.2) in place on q, theta; returns (statistics per solve, status)."""
        return self._step(self.lib.rpbd_step_tt, 4, shape, q, theta, forces, sp)

    def blob_forces(self, r, forces: Forces, nper=0, dtype=F64, out=None):
        """Per-blob forces (gravity, blob-wall and, with nper, blob-blob Yukawa repulsion; Sec. 4.1), [3, n]."""
        out = torch.empty_like(r) if out is None else out
        self._check(self.lib.rpbd_blob_forces(self.h, r.shape[1], nper, _ptr(r), C.byref(forces), dtype,
                                              _ptr(out), _stream()), "blob_forces")
        return out
