"""ctypes binding of librpbd.so (include/rpbd.h).  Argument marshalling only:
every step of the computation runs in the CUDA library."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librpbd.so")

F64, F32 = 0, 1
STATUS = {0: "ok", -1: "bad argument", -2: "bad input", -3: "CUDA error", -4: "not converged",
          -5: "device wait timed out", -6: "out of device memory", -7: "too large for the fixed scratch"}


class Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("a", C.c_double), ("kT", C.c_double), ("wall", C.c_int),
                ("s_min", C.c_double), ("Lx", C.c_double), ("Ly", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("matvecs", C.c_int), ("residual", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return dict(iterations=self.iterations, matvecs=self.matvecs, residual=self.residual, status=self.status)


class Forces(C.Structure):
    _fields_ = [("weight", C.c_double), ("wall_gamma", C.c_double), ("wall_b", C.c_double),
                ("h_floor", C.c_double), ("torque", C.c_double * 3), ("steric_gamma", C.c_double),
                ("steric_b", C.c_double), ("r_floor", C.c_double), ("r_cut", C.c_double)]


class StepParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("delta", C.c_double), ("Lp", C.c_double), ("tol_gmres", C.c_double),
                ("tol_lanczos", C.c_double), ("max_iter_gmres", C.c_int), ("restart", C.c_int),
                ("max_iter_lanczos", C.c_int), ("dtype", C.c_int), ("seed", C.c_uint64), ("step", C.c_uint32),
                ("cold_start", C.c_int)]


# (name, restype, argtypes)
_P, _I64, _I, _D, _U64, _U32 = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_uint64, C.c_uint32
SIGNATURES = [
    ("rpbd_create", _I, [C.POINTER(_P), C.POINTER(Params)]),
    ("rpbd_destroy", _I, [_P]),
    ("rpbd_reserve", _I, [_P, _I64, _I64, _I, _I, _I]),
    ("rpbd_last_error", C.c_char_p, [_P]),
    ("rpbd_status_string", C.c_char_p, [_I]),
    ("rpbd_blobs_from_bodies", _I, [_P, _I64, _I, _P, _P, _P, _P, _P]),
    ("rpbd_mobility_apply", _I, [_P, _I64, _P, _P, _P, _I, _I, _P]),
    ("rpbd_mobility_apply_mixed", _I, [_P, _I64, _P, _P, _P, _I, _I, _P]),
    ("rpbd_mobility_adjoint", _I, [_P, _I64, _P, _P, _P, _P, _P]),
    ("rpbd_mobility_adjoint_f32", _I, [_P, _I64, _P, _P, _P, _P, _P]),
    ("rpbd_mobility_adjoint_multi", _I, [_P, _I64, _P, _P, _P, _I, _P, _I, _P]),
    ("rpbd_mobility_divergence", _I, [_P, _I64, _P, _P, _P]),
    ("rpbd_K_apply", _I, [_P, _I64, _I, _P, _P, _P, _P, _P]),
    ("rpbd_KT_apply", _I, [_P, _I64, _I, _P, _P, _P, _P, _P]),
    ("rpbd_precond_build", _I, [_P, _I64, _I, _P, _P, _P]),
    ("rpbd_precond_apply", _I, [_P, _I, _P, _P, _P]),
    ("rpbd_lanczos_sqrt_apply", _I, [_P, _I64, _P, _P, _P, _D, _I, _I, _I, C.POINTER(Stats), _P]),
    ("rpbd_lanczos_sqrt_apply_multi", _I, [_P, _I64, _P, _I, _P, _P, _D, _I, _I, _I, C.POINTER(Stats), _P]),
    ("rpbd_gmres_rigid_solve_multi", _I, [_P, _I64, _I, _P, _P, _I, _P, _P, _P, _P, _D, _I, _I, _I, _I,
                                          C.POINTER(Stats), _P]),
    ("rpbd_gmres_rigid_solve", _I, [_P, _I64, _I, _P, _P, _P, _P, _P, _P, _D, _I, _I, _I, _I, _I,
                                    C.POINTER(Stats), _P]),
    ("rpbd_rfd_drift", _I, [_P, _I64, _P, _P, _D, _P, _I, _P]),
    ("rpbd_philox_normals", _I, [_P, _U64, _U32, _U32, _I64, _P, _P]),
    ("rpbd_step_ts", _I, [_P, _I64, _I, _P, _P, _P, C.POINTER(Forces), C.POINTER(StepParams),
                          C.POINTER(Stats), _P]),
    ("rpbd_step_emt", _I, [_P, _I64, _I, _P, _P, _P, C.POINTER(Forces), C.POINTER(StepParams),
                           C.POINTER(Stats), _P]),
    ("rpbd_step_emrfd", _I, [_P, _I64, _I, _P, _P, _P, C.POINTER(Forces), C.POINTER(StepParams),
                             C.POINTER(Stats), _P]),
    ("rpbd_step_tt", _I, [_P, _I64, _I, _P, _P, _P, C.POINTER(Forces), C.POINTER(StepParams),
                          C.POINTER(Stats), _P]),
    ("rpbd_blob_forces", _I, [_P, _I64, _I, _P, C.POINTER(Forces), _I, _P, _P]),
    ("rpbd_mobility_apply_batched", _I, [_P, _I, _P, _P, _P, _P, _I, _P]),
    ("rpbd_autotune_batched", _I, [_P, _I, _P, _P, _I, C.POINTER(C.c_double), _P]),
    ("rpbd_lanczos_sqrt_apply_batched", _I, [_P, _I, _P, _P, _P, _P, _P, _P, _D, _I, _I, _I, _P, _P]),
    ("rpbd_mobility_apply_f32_noalloc", _I, [C.POINTER(Params), _I64, _P, _P, _P, _I, _P]),
    ("rpbd_launch_count", C.c_longlong, []),
    ("rpbd_measure_fma_peak", _I, [_P, _I, C.POINTER(C.c_double), _P]),
    ("rpbd_set_option", _I, [_P, _I, _I]),
    ("rpbd_autotune", _I, [_P, _I64, _P, _I, C.POINTER(C.c_double), _P]),
    ("rpbd_profile_enable", _I, [_P, _I]),
    ("rpbd_profile_read", _I, [_P, _I, _I, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                               C.POINTER(C.c_double), _I]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load the library and bind every signature.  Raises if it is missing:
    there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librpbd.so not built ({path}); run paper_1709_02410_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return [s[0] for s in SIGNATURES]
