"""Oracle blob mobility: ctypes front end of oracle_mobility.cpp (FP64).

TEST INFRASTRUCTURE (see oracle/__init__.py).

M_ij = s_i s_j [M_RPY(r~_i - r~_j) + M_wall(r~_i, r~_j)]: free-space RPY
(Sec. 2.1) plus the Faxen-regularised Blake image system for the no-slip wall
at z = 0 (the Rotne-Prager-Blake tensor of Sec. 2.1 / Sec. 4), with the
wall-overlap reading r~ = (x, y, max(z, a)), s = clamp(z/a, s_min, 1).
Positions are SoA [3, n]; vectors [k, 3, n] (or [3, n] for k = 1).
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        d, i64, i = C.c_double, C.c_int64, C.c_int
        P = C.POINTER(C.c_double)
        PI = C.POINTER(C.c_int64)
        _lib.orc_mobility_apply_rows.argtypes = [i64, P, P, P, i, d, d, i, d, d, d, PI, i64]
        _lib.orc_mobility_dense.argtypes = [i64, P, P, d, d, i, d, d, d]
        _lib.orc_mobility_grad_rows.argtypes = [i64, P, P, P, P, d, d, i, d, d, d, PI, i64]
        _lib.orc_mobility_div_rows.argtypes = [i64, P, P, d, d, i, d, d, d, PI, i64]
        _lib.orc_pair_block.argtypes = [P, P, i, d, d, i, d, d, d, P]
        _lib.orc_pair_dblock.argtypes = [P, P, i, d, d, i, d, d, d, P, P]
        _lib.orc_blake_point.argtypes = [P, P, P]
        _lib.orc_num_threads.restype = i
        _lib.orc_set_num_threads.argtypes = [i]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Params:
    """eta, a, wall on/off, overlap floor s_min; Lx, Ly > 0 switch on the
    pseudo-periodic sum of Sec. 4.2 (minimum image + 8 nearest images)."""

    def __init__(self, eta, a, wall=True, s_min=1e-3, Lx=0.0, Ly=0.0):
        self.eta, self.a, self.wall, self.s_min = float(eta), float(a), int(bool(wall)), float(s_min)
        self.Lx, self.Ly = float(Lx), float(Ly)

    def args(self):
        return (self.eta, self.a, self.wall, self.s_min, self.Lx, self.Ly)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int):
    """OpenMP threads of the oracle's loops (timing at a fixed core count)."""
    lib().orc_set_num_threads(int(n))


def apply(r, F, prm: Params, rows=None):
    """U = M(r) F.  r [3, n]; F [3, n] or [k, 3, n].  With rows given, only
    those target rows are computed and U has n_rows columns."""
    r = _c(r)
    n = r.shape[1]
    F = _c(F)
    squeeze = F.ndim == 2
    if squeeze:
        F = F[None]
    k = F.shape[0]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.size, rows.ctypes.data_as(C.POINTER(C.c_int64))
    U = np.zeros((k, 3, nr))
    lib().orc_mobility_apply_rows(n, _p(r), _p(F), _p(U), k, *prm.args(), rp, nr)
    return U[0] if squeeze else U


def dense(r, prm: Params):
    """Dense 3n x 3n matrix, entry (3i+c, 3j+d) = (M_ij)_cd (blob-interleaved)."""
    r = _c(r)
    n = r.shape[1]
    M = np.zeros((3 * n, 3 * n))
    lib().orc_mobility_dense(n, _p(r), _p(M), *prm.args())
    return M


def grad(r, u, F, prm: Params, rows=None):
    """d(u^T M(r) F)/dr_k for all blobs (or the listed ones): [3, n_rows]."""
    r, u, F = _c(r), _c(u), _c(F)
    n = r.shape[1]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.size, rows.ctypes.data_as(C.POINTER(C.c_int64))
    g = np.zeros((3, nr))
    lib().orc_mobility_grad_rows(n, _p(r), _p(u), _p(F), _p(g), *prm.args(), rp, nr)
    return g


def divergence(r, prm: Params, rows=None):
    """(div M)_i = sum_j d_{r_j} . M_ij: [3, n_rows]."""
    r = _c(r)
    n = r.shape[1]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.size, rows.ctypes.data_as(C.POINTER(C.c_int64))
    d = np.zeros((3, nr))
    lib().orc_mobility_div_rows(n, _p(r), _p(d), *prm.args(), rp, nr)
    return d


def pair_block(ri, rj, prm: Params, same=False):
    M = np.zeros(9)
    lib().orc_pair_block(_p(_c(ri)), _p(_c(rj)), int(same), *prm.args(), _p(M))
    return M.reshape(3, 3)


def pair_dblock(ri, rj, prm: Params, same=False):
    """(Dx, Dy) with D[c, d, e] = d(M_ij)_cd / d r_{i|j},e."""
    Dx, Dy = np.zeros(27), np.zeros(27)
    lib().orc_pair_dblock(_p(_c(ri)), _p(_c(rj)), int(same), *prm.args(), _p(Dx), _p(Dy))
    return Dx.reshape(3, 3, 3), Dy.reshape(3, 3, 3)


def blake_point(x, y):
    """8 pi eta times Blake's point-force Green's function (no Faxen terms)."""
    G = np.zeros(9)
    lib().orc_blake_point(_p(_c(x)), _p(_c(y)), _p(G))
    return G.reshape(3, 3)


def soa_to_blob(v):
    """[3, n] -> [3n] blob-interleaved (matches dense())."""
    return np.ascontiguousarray(np.asarray(v).T).reshape(-1)


def blob_to_soa(v):
    return np.ascontiguousarray(np.asarray(v).reshape(-1, 3).T)
