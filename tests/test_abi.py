"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point include/rpbd.h declares; the binding covers them all."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rpbd.h")).read()
    return sorted(set(re.findall(r"^(?:int|long long|const char\*)\s+(rpbd_\w+)\s*\(", src, re.M)))


def test_header_declares_entry_points():
    names = declared()
    for must in ("rpbd_mobility_apply", "rpbd_mobility_adjoint", "rpbd_lanczos_sqrt_apply",
                 "rpbd_gmres_rigid_solve", "rpbd_rfd_drift", "rpbd_step_ts", "rpbd_step_emt",
                 "rpbd_precond_build"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1709_02410_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_1709_02410_gb300 import _native
    assert sorted(_native.exported_names()) == declared()
    _native.load()      # binds every signature


def test_status_strings_without_gpu():
    from paper_1709_02410_gb300 import _native
    lib = _native.load()
    assert lib.rpbd_status_string(-4) == b"iteration did not converge"
    assert lib.rpbd_status_string(0) == b"ok"
