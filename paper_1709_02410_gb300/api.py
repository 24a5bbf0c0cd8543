"""Torch-facing binding of the C ABI (argument marshalling only).

Tensors must be contiguous CUDA tensors on the handle's device; positions
are [3, n] float64 (SoA), blob vectors [k, 3, n] or [3, n], body vectors
[nb, 6], q [nb, 3], theta [nb, 4].  Calls run on torch's current stream.
Every tensor's dtype, shape and device is checked here before the library is
called, so a wrong argument raises RpbdError and launches nothing.
"""
import ctypes as C

import torch

from . import _native
from ._native import F32, F64, Forces, Params, Stats, StepParams


class RpbdError(RuntimeError):
    pass


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _kvec(t, n, name):
    """k of a blob vector [3, n] (k = 1) or [k, 3, n] (1 <= k <= 16)."""
    if t.dim() == 2 and tuple(t.shape) == (3, n):
        return 1
    if t.dim() == 3 and t.shape[1:] == (3, n) and 1 <= t.shape[0] <= 16:
        return t.shape[0]
    raise RpbdError(f"{name}: expected shape (3, {n}) or (k, 3, {n}) with 1 <= k <= 16, got {tuple(t.shape)}")


class Handle:
    """Owns an rpbd_handle (device workspace + physical parameters), bound to
    the CUDA device that is current when it is created."""

    def __init__(self, eta, a, kT=0.0, wall=True, s_min=1e-3, Lx=0.0, Ly=0.0):
        self.lib = _native.load()
        self.params = Params(eta, a, kT, int(bool(wall)), s_min, Lx, Ly)
        self.device = torch.device("cuda", torch.cuda.current_device())
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

    def _p(self, t, name, dtypes=(torch.float64,), shape=None):
        """Device pointer of t after checking dtype, shape, device and layout
        (None passes through as NULL)."""
        if t is None:
            return None
        if not isinstance(t, torch.Tensor):
            raise RpbdError(f"{name}: expected a torch tensor")
        if not t.is_cuda or t.device != self.device:
            raise RpbdError(f"{name}: expected a tensor on {self.device}, got {t.device}")
        if t.dtype not in dtypes:
            raise RpbdError(f"{name}: expected dtype {' or '.join(str(d) for d in dtypes)}, got {t.dtype}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise RpbdError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise RpbdError(f"{name}: expected a contiguous tensor")
        return C.c_void_p(t.data_ptr())

    def _r(self, r):
        if not isinstance(r, torch.Tensor) or r.dim() != 2 or r.shape[0] != 3:
            raise RpbdError(f"r: expected positions of shape (3, n), got {getattr(r, 'shape', type(r))}")
        return r.shape[1], self._p(r, "r", shape=(3, r.shape[1]))

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

    def set_test_stall(self, on: bool):
        """Failure-path test only: the pair kernels' first source wait runs out
        (RPBD_TIMEOUT from the synchronising calls) until this is set back off."""
        self._check(self.lib.rpbd_set_option(self.h, 5, int(bool(on))), "set_option")

    def set_far_field(self, on: bool):
        """FP32 matvecs with the wall: form every pair block with the cancellation-free
        direct-minus-image differences (FP32 accuracy at any separation, ~9% slower)."""
        self._check(self.lib.rpbd_set_option(self.h, 6, int(bool(on))), "set_option")

    def set_sym_partials(self, on: bool):
        """FP32 matvec of one system: partial sums with the fixed-order reduction (per home tile
        in the packed symmetric kernel, per source chunk in the one-direction kernel; memory
        O(n^2)) instead of the default fixed-point accumulation (memory O(n))."""
        self._check(self.lib.rpbd_set_option(self.h, 7, int(bool(on))), "set_option")

    def measure_fma_peak(self, dtype=F32):
        """FMA throughput of this GPU in TFLOP/s (FMA = 2), measured by the library."""
        v = C.c_double()
        self._check(self.lib.rpbd_measure_fma_peak(self.h, dtype, C.byref(v), _stream()), "measure_fma_peak")
        return v.value

    def autotune(self, r, k=1):
        """Pick the fastest FP32 kernel for this n and k; returns (choice, ms per launch)."""
        n, rp = self._r(r)
        ms = C.c_double()
        c = self.lib.rpbd_autotune(self.h, n, rp, k, C.byref(ms), _stream())
        if c < 0:
            self._check(c, "autotune")
        return c, ms.value

    # ---- a1
    def blobs_from_bodies(self, shape, q, theta, out=None):
        """Blob positions r = q_p + R(theta_p) s_i (Sec. 2.1) as [3, nb * nper] FP64 SoA."""
        nb, nper = q.shape[0], shape.shape[0]
        out = torch.empty((3, nb * nper), dtype=torch.float64, device=q.device) if out is None else out
        args = (self._p(shape, "shape", shape=(nper, 3)), self._p(q, "q", shape=(nb, 3)),
                self._p(theta, "theta", shape=(nb, 4)), self._p(out, "out", shape=(3, nb * nper)))
        self._check(self.lib.rpbd_blobs_from_bodies(self.h, nb, nper, *args, _stream()), "blobs_from_bodies")
        return out

    # ---- a2
    def mobility_apply(self, r, F, dtype=None, out=None):
        """U = M(r) F.  F [k,3,n] or [3,n]; float64 -> FP64 kernel, float32 ->
        FP32 kernel.  dtype=F32 with float64 F runs FP32 pairs on FP64 vectors."""
        n, rp = self._r(r)
        k = _kvec(F, n, "F")
        if dtype is None:
            Fp = self._p(F, "F", (torch.float32, torch.float64))
            dt = F64 if F.dtype == torch.float64 else F32
            fn = self.lib.rpbd_mobility_apply
        else:
            if dtype not in (F32, F64):
                raise RpbdError("dtype: expected F32 or F64")
            Fp = self._p(F, "F (mixed mode)")
            dt = dtype
            fn = self.lib.rpbd_mobility_apply_mixed
        out = torch.empty_like(F) if out is None else out
        Up = self._p(out, "out", (F.dtype,), tuple(F.shape))
        self._check(fn(self.h, n, rp, Fp, Up, k, dt, _stream()), "mobility_apply")
        return out

    # ---- a7
    def mobility_adjoint(self, r, u, F, out=None, dtype=F64):
        """d(sum_m u_m^T M(r) F_m)/dr, FP64 vectors u, F of shape [3, n] or [k, 3, n]
        (the sum over the k pairs runs on the device); dtype F32 evaluates the pair
        derivative in FP32."""
        n, rp = self._r(r)
        k = _kvec(F, n, "F")
        if tuple(u.shape) != tuple(F.shape):
            raise RpbdError(f"u: expected the shape of F {tuple(F.shape)}, got {tuple(u.shape)}")
        if dtype not in (F32, F64):
            raise RpbdError("dtype: expected F32 or F64")
        out = torch.empty((3, n), dtype=torch.float64, device=r.device) if out is None else out
        args = (self._p(u, "u"), self._p(F, "F"), k, self._p(out, "out", shape=(3, n)))
        self._check(self.lib.rpbd_mobility_adjoint_multi(self.h, n, rp, *args, dtype, _stream()), "mobility_adjoint")
        return out

    def mobility_divergence(self, r, out=None):
        """div M (the thermal drift that the RFD of Sec. 3 estimates), exact, FP64, [3, n]."""
        n, rp = self._r(r)
        out = torch.empty((3, n), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_mobility_divergence(self.h, n, rp, self._p(out, "out", shape=(3, n)), _stream()),
                    "mobility_divergence")
        return out

    # ---- rigid
    def _bodies(self, nper, r, q):
        n, rp = self._r(r)
        nb = q.shape[0]
        if nper <= 0 or nb * nper != n:
            raise RpbdError(f"bodies: {nb} bodies of {nper} blobs do not match r with {n} blobs")
        return n, nb, rp, self._p(q, "q", shape=(nb, 3))

    def K_apply(self, nper, r, q, U, out=None):
        """Blob velocities K U of rigid-body motions U [nb, 6] (Sec. 2.1), [3, n]."""
        n, nb, rp, qp = self._bodies(nper, r, q)
        out = torch.empty((3, n), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_K_apply(self.h, nb, nper, rp, qp, self._p(U, "U", shape=(nb, 6)),
                                          self._p(out, "out", shape=(3, n)), _stream()), "K_apply")
        return out

    def KT_apply(self, nper, r, q, lam, out=None):
        """Total force and torque K^T lambda per body of blob forces lambda [3, n], [nb, 6]."""
        n, nb, rp, qp = self._bodies(nper, r, q)
        out = torch.empty((nb, 6), dtype=torch.float64, device=r.device) if out is None else out
        self._check(self.lib.rpbd_KT_apply(self.h, nb, nper, rp, qp, self._p(lam, "lam", shape=(3, n)),
                                           self._p(out, "out", shape=(nb, 6)), _stream()), "KT_apply")
        return out

    # ---- a3
    def precond_build(self, nper, r, q):
        """Build the body-block-diagonal preconditioner (Sec. 2.2) at r; kept until the next build."""
        n, nb, rp, qp = self._bodies(nper, r, q)
        self._n_prec = n
        self._check(self.lib.rpbd_precond_build(self.h, nb, nper, rp, qp, _stream()), "precond_build")

    def precond_apply(self, mode, x, out=None):
        """Apply a stored factor per body: mode 0 L, 1 L^-1, 2 L^-T, 3 M~^-1."""
        n = getattr(self, "_n_prec", None)
        if n is None:
            raise RpbdError("precond_apply: no preconditioner built through this handle")
        out = torch.empty_like(x) if out is None else out
        self._check(self.lib.rpbd_precond_apply(self.h, mode, self._p(x, "x", shape=(3, n)),
                                                self._p(out, "out", shape=(3, n)), _stream()), "precond_apply")
        return out

    # ---- a4
    def lanczos_sqrt_apply(self, r, W, tol, max_iter=80, dtype=F64, use_precond=True, out=None):
        """M^{1/2} W by preconditioned Lanczos (Sec. 2.2); returns (out, stats).  A run that stops
        at max_iter returns its last iterate with stats status -4 (not converged)."""
        n, rp = self._r(r)
        Wp = self._p(W, "W", shape=(3, n))
        out = torch.empty_like(W) if out is None else out
        st = Stats()
        s = self.lib.rpbd_lanczos_sqrt_apply(self.h, n, rp, Wp, self._p(out, "out", shape=(3, n)), tol, max_iter,
                                             dtype, int(bool(use_precond)), C.byref(st), _stream())
        if s not in (0, -4):
            self._check(s, "lanczos_sqrt_apply")
        return out, st.as_dict()

    # ---- a5
    def gmres_rigid_solve(self, nper, r, q, slip=None, FT=None, tol=1e-6, max_iter=200, restart=50, dtype=F64,
                          build_precond=True, x0=None):
        """x0 = (lambda0, U0): initial guess (GMRES warm start); default zero."""
        n, nb, rp, qp = self._bodies(nper, r, q)
        if x0 is None:
            lam = torch.empty((3, n), dtype=torch.float64, device=r.device)
            U = torch.empty((nb, 6), dtype=torch.float64, device=r.device)
        else:
            lam, U = x0[0].clone(), x0[1].clone()
        st = Stats()
        if build_precond:
            self._n_prec = n
        s = self.lib.rpbd_gmres_rigid_solve(self.h, nb, nper, rp, qp, self._p(slip, "slip", shape=(3, n)),
                                            self._p(FT, "FT", shape=(nb, 6)), self._p(lam, "lambda", shape=(3, n)),
                                            self._p(U, "U", shape=(nb, 6)), tol, max_iter, restart, dtype,
                                            int(bool(build_precond)), int(x0 is not None), C.byref(st), _stream())
        if s not in (0, -4):
            self._check(s, "gmres_rigid_solve")
        return lam, U, st.as_dict()

    def lanczos_sqrt_apply_multi(self, r, Ws, tol=1e-4, max_iter=60, dtype=F64, use_precond=True):
        """1..4 Lanczos square roots M^{1/2} W at the same positions, in lockstep
        (shared multi-RHS matvecs).  Returns a list of (out, stats)."""
        n, rp = self._r(r)
        ns = len(Ws)
        if not 1 <= ns <= 4:
            raise RpbdError("lanczos_sqrt_apply_multi: 1..4 vectors W")
        outs = [torch.empty((3, n), dtype=torch.float64, device=r.device) for _ in range(ns)]
        arr = C.c_void_p * ns
        st = (Stats * ns)()
        s = self.lib.rpbd_lanczos_sqrt_apply_multi(self.h, n, rp, ns,
                                                   arr(*[self._p(w, "W", shape=(3, n)) for w in Ws]),
                                                   arr(*[self._p(o, "out") for o in outs]), tol, max_iter, dtype,
                                                   int(bool(use_precond)), st, _stream())
        if s not in (0, -4):
            self._check(s, "lanczos_sqrt_apply_multi")
        return [(o, st[i].as_dict()) for i, o in enumerate(outs)]

    def gmres_rigid_solve_multi(self, nper, r, q, problems, tol=1e-6, max_iter=200, restart=50, dtype=F64,
                                build_precond=True):
        """problems: list of 1..4 (slip, FT) pairs (either None) at the same
        positions; solved in lockstep with shared multi-RHS matvecs.  Returns a
        list of (lambda, U, stats)."""
        n, nb, rp, qp = self._bodies(nper, r, q)
        ns = len(problems)
        if not 1 <= ns <= 4:
            raise RpbdError("gmres_rigid_solve_multi: 1..4 problems")
        outs = [(torch.empty((3, n), dtype=torch.float64, device=r.device),
                 torch.empty((nb, 6), dtype=torch.float64, device=r.device)) for _ in range(ns)]
        arr = C.c_void_p * ns
        slips = arr(*[self._p(p[0], "slip", shape=(3, n)) for p in problems])
        fts = arr(*[self._p(p[1], "FT", shape=(nb, 6)) for p in problems])
        lams = arr(*[self._p(o[0], "lambda") for o in outs])
        us = arr(*[self._p(o[1], "U") for o in outs])
        st = (Stats * ns)()
        if build_precond:
            self._n_prec = n
        s = self.lib.rpbd_gmres_rigid_solve_multi(self.h, nb, nper, rp, qp, ns, slips, fts, lams, us, tol,
                                                  max_iter, restart, dtype, int(bool(build_precond)), st, _stream())
        if s not in (0, -4):
            self._check(s, "gmres_rigid_solve_multi")
        return [(o[0], o[1], st[i].as_dict()) for i, o in enumerate(outs)]

    # ---- a6
    def rfd_drift(self, r, W, delta, dtype=F64, out=None):
        """Blob-level centred RFD (Sec. 3): [M(r + delta/2 W) - M(r - delta/2 W)] W / delta; mean div M."""
        n, rp = self._r(r)
        Wp = self._p(W, "W", shape=(3, n))
        out = torch.empty_like(W) if out is None else out
        self._check(self.lib.rpbd_rfd_drift(self.h, n, rp, Wp, delta, self._p(out, "out", shape=(3, n)), dtype,
                                            _stream()), "rfd_drift")
        return out

    # ---- batched suspensions
    @staticmethod
    def _offsets(offsets):
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if off.ndim != 1 or off.size < 2 or off[0] != 0 or np.any(np.diff(off) < 0):
            raise RpbdError("offsets: expected a non-decreasing 1-D array starting at 0 with >= 2 entries")
        return off, off.ctypes.data_as(C.c_void_p)

    def mobility_apply_batched(self, offsets, r, F, out=None):
        """U = M(r_s) F_s for independent systems concatenated at blob offsets (FP32 [k, 3, n])."""
        off, op = self._offsets(offsets)
        n_sys = off.size - 1
        n, rp = self._r(r)
        if n != off[-1]:
            raise RpbdError(f"r: {n} blobs, offsets end at {off[-1]}")
        k = _kvec(F, n, "F")
        Fp = self._p(F, "F", (torch.float32,))
        out = torch.empty_like(F) if out is None else out
        self._check(self.lib.rpbd_mobility_apply_batched(self.h, n_sys, op, rp, Fp,
                                                         self._p(out, "out", (torch.float32,), tuple(F.shape)), k,
                                                         _stream()), "mobility_apply_batched")
        return out

    def autotune_batched(self, offsets, r, k=1):
        """Time the batched variants on this batch and keep the fastest; returns (variant, ms)."""
        off, op = self._offsets(offsets)
        n, rp = self._r(r)
        if n != off[-1]:
            raise RpbdError(f"r: {n} blobs, offsets end at {off[-1]}")
        ms = C.c_double()
        v = self.lib.rpbd_autotune_batched(self.h, off.size - 1, op, rp, k, C.byref(ms), _stream())
        if v < 0:
            self._check(v, "autotune_batched")
        return v, ms.value

    def lanczos_sqrt_apply_batched(self, offsets, r, W, tol, max_iter=40, use_precond=True, use_graph=True,
                                   F=None, out=None, U=None):
        """One preconditioned Lanczos M^{1/2} W per system of a batch, in lockstep (one CUDA graph when
        use_graph), and optionally U = M F per system; returns (out, U, iterations per system)."""
        off, op = self._offsets(offsets)
        n_sys = off.size - 1
        n, rp = self._r(r)
        if n != off[-1]:
            raise RpbdError(f"r: {n} blobs, offsets end at {off[-1]}")
        Wp = self._p(W, "W", shape=(3, n))
        out = torch.empty_like(W) if out is None else out
        if F is not None and U is None:
            U = torch.empty_like(F)
        iters = (C.c_int * n_sys)()
        self._check(self.lib.rpbd_lanczos_sqrt_apply_batched(self.h, n_sys, op, rp, Wp,
                                                             self._p(out, "out", shape=(3, n)),
                                                             self._p(F, "F", shape=(3, n)),
                                                             self._p(U, "U", shape=(3, n)), tol, max_iter,
                                                             int(bool(use_precond)), int(bool(use_graph)), iters,
                                                             _stream()),
                    "lanczos_sqrt_apply_batched")
        return out, U, list(iters)

    # ---- random numbers
    def philox_normals(self, n, seed, step, sid, device=None):
        """n N(0,1) draws of Philox4x32-10 keyed by (seed, step, stream id), as the time steps draw them."""
        out = torch.empty(n, dtype=torch.float64, device=self.device if device is None else device)
        self._check(self.lib.rpbd_philox_normals(self.h, seed, step, sid, n, self._p(out, "out"), _stream()),
                    "philox_normals")
        return out

    # ---- a8
    def _step(self, fn, nstats, shape, q, theta, forces: Forces, sp: StepParams):
        nb, nper = q.shape[0], shape.shape[0]
        args = (self._p(shape, "shape", shape=(nper, 3)), self._p(q, "q", shape=(nb, 3)),
                self._p(theta, "theta", shape=(nb, 4)))
        st = (Stats * nstats)()
        self._n_prec = nb * nper  # every step builds the preconditioner
        s = fn(self.h, nb, nper, *args, C.byref(forces), C.byref(sp), st, _stream())
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
        n, rp = self._r(r)
        out = torch.empty_like(r) if out is None else out
        self._check(self.lib.rpbd_blob_forces(self.h, n, nper, rp, C.byref(forces), dtype,
                                              self._p(out, "out", shape=(3, n)), _stream()), "blob_forces")
        return out
