"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (reference body shapes, random body
placements, random vectors); none of the method's arithmetic lives here.  The
CUDA path and the CPU oracle both draw their inputs from it.

Workloads (Sec. 4):
  * boomerangs (Sec. 4.1-4.2): L-shaped rigid bodies of 15 blobs, two straight
    arms of 7 blobs plus the shared cross-point, which is the tracking point.
  * microrollers (Sec. 4.3): spheres resolved by 12 blobs on the vertices of
    an icosahedron.
Body centres are uniform in a square box in x-y; orientations are uniform on
the unit quaternion sphere (normalised 4-D Gaussian).  A body's height above
the wall is a + Exp(mean 1.5 a): by default ("lifted") this is the height of
its lowest blob, so no blob overlaps the wall; with lift=False it is the
height of the tracking point and rotated arms may reach below the wall (the
regime of the wall-overlap regularisation).  Units: um, s, mg.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# physical constants of the workloads (um, s, mg)
ETA = 1.0e-3          # water viscosity, mg / (um s)  (= 1 mPa s)
KT = 0.0041           # k_B T at ~300 K, mg um^2 / s^2
A_BOOMERANG = 0.325   # blob radius for the boomerang workloads, um
A_ROLLER = 0.416      # blob radius for the 12-blob microroller, um
RH_ROLLER = 0.656     # roller hydrodynamic radius, um (Sec. 4.3)


def boomerang_shape(a: float = A_BOOMERANG, spacing: float | None = None) -> np.ndarray:
    """Reference blob offsets [15, 3] of an L-shaped boomerang.

    Blob 0 is the cross-point (the tracking point, at the origin); blobs 1-7
    lie on the +x arm and blobs 8-14 on the +y arm, `spacing` apart
    (default 2.1 a)."""
    d = 2.1 * a if spacing is None else spacing
    s = np.zeros((15, 3))
    for k in range(1, 8):
        s[k] = (k * d, 0.0, 0.0)
        s[7 + k] = (0.0, k * d, 0.0)
    return s


def icosahedron_shape(a: float = A_ROLLER) -> np.ndarray:
    """Reference blob offsets [12, 3]: icosahedron vertices with edge 2a,
    centred on the tracking point (circumradius ~1.902 a)."""
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * g))
            v.append((s1, s2 * g, 0.0))
            v.append((s2 * g, 0.0, s1))
    return a * np.asarray(v)


@dataclass
class Suspension:
    """Rigid bodies of one shape: q [nb, 3] tracking points, theta [nb, 4]
    unit quaternions (s, p), shape [nper, 3] reference offsets."""
    q: np.ndarray
    theta: np.ndarray
    shape: np.ndarray
    a: float
    box: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nb(self) -> int:
        return self.q.shape[0]

    @property
    def nper(self) -> int:
        return self.shape.shape[0]

    @property
    def n(self) -> int:
        return self.nb * self.nper


def random_quaternions(rng: np.random.Generator, nb: int) -> np.ndarray:
    th = rng.standard_normal((nb, 4))
    return th / np.linalg.norm(th, axis=1, keepdims=True)


def _lowest_offset(theta: np.ndarray, shape: np.ndarray) -> np.ndarray:
    """min over blobs of the z-offset of each rotated body (placement only:
    the z row of the rotation of unit quaternion (s, p))."""
    s, p1, p2, p3 = theta.T
    zrow = np.stack([2 * (p1 * p3 - s * p2), 2 * (p2 * p3 + s * p1), s * s - p1 * p1 - p2 * p2 + p3 * p3], 1)
    return (zrow @ shape.T).min(axis=1)


def boomerang_suspension(nb: int, box: float, seed: int, a: float = A_BOOMERANG,
                         spacing: float | None = None, lift: bool = True) -> Suspension:
    """nb boomerangs: centres uniform over [0, box]^2, height a + Exp(1.5 a)."""
    rng = np.random.default_rng(seed)
    q = np.empty((nb, 3))
    q[:, :2] = rng.uniform(0.0, box, size=(nb, 2))
    q[:, 2] = a + rng.exponential(1.5 * a, size=nb)
    th = random_quaternions(rng, nb)
    shape = boomerang_shape(a, spacing)
    if lift:
        q[:, 2] -= _lowest_offset(th, shape)
    return Suspension(q, th, shape, a, box, "boomerang", dict(lift=lift))


def _separate(q: np.ndarray, box: float, dmin: float, rng: np.random.Generator, tries: int = 10000) -> np.ndarray:
    """Placement only: random sequential addition -- each body in turn keeps
    its height and re-draws x, y until its centre is at least dmin (3-D
    distance) from every body already placed (a cell list of side >= dmin)."""
    q = q.copy()
    nc = max(1, int(box // dmin))
    cell = box / nc
    grid = {}
    for i in range(q.shape[0]):
        for _ in range(tries):
            cx, cy = min(int(q[i, 0] // cell), nc - 1), min(int(q[i, 1] // cell), nc - 1)
            clash = False
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for j in grid.get((cx + dx, cy + dy), ()):
                        if np.sum((q[i] - q[j]) ** 2) < dmin * dmin:
                            clash = True
                            break
                    if clash:
                        break
                if clash:
                    break
            if not clash:
                grid.setdefault((cx, cy), []).append(i)
                break
            q[i, :2] = rng.uniform(0.0, box, size=2)
        else:
            raise RuntimeError("could not place the bodies without overlap")
    return q


def roller_suspension(nb: int, phi: float, seed: int, a: float = A_ROLLER,
                      rh: float = RH_ROLLER, lift: bool = True, overlap: bool = True) -> Suspension:
    """nb 12-blob rollers at in-plane packing fraction phi = n pi rh^2;
    height a + Exp(1.5 a) (lowest blob), or rh + Exp(1.5 a) for the centre
    when lift=False.  overlap=False re-draws x, y until no two roller centres
    are closer than 2 rh (hard spheres of the hydrodynamic radius)."""
    box = float(np.sqrt(nb * np.pi * rh * rh / phi))
    rng = np.random.default_rng(seed)
    q = np.empty((nb, 3))
    q[:, :2] = rng.uniform(0.0, box, size=(nb, 2))
    e = rng.exponential(1.5 * a, size=nb)
    th = random_quaternions(rng, nb)
    shape = icosahedron_shape(a)
    q[:, 2] = (a + e - _lowest_offset(th, shape)) if lift else (rh + e)
    if not overlap:
        q = _separate(q, box, 2.0 * rh, rng)
    return Suspension(q, th, shape, a, box, "roller", dict(lift=lift, overlap=overlap))


def gaussian(seed: int, shape, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


# ---- the five workloads -------------------------------------------------

def boomerangs_1920(seed: int = 0) -> Suspension:
    """128 boomerangs x 15 = 1,920 blobs in a 40 x 40 um box (FP64 parity)."""
    return boomerang_suspension(128, 40.0, seed)


def boomerangs_65535(seed: int = 1) -> Suspension:
    """4,369 boomerangs x 15 = 65,535 blobs, box scaled to c0's area density."""
    return boomerang_suspension(4369, 40.0 * np.sqrt(4369 / 128), seed)


def blobs_16384(seed: int = 2) -> Suspension:
    """16,380 blobs as 1,092 boomerangs (adjoint workload), same density."""
    return boomerang_suspension(1092, 40.0 * np.sqrt(1092 / 128), seed)


def rollers_196608(seed: int = 3, nb: int = 16384, overlap: bool = False) -> Suspension:
    """16,384 rollers x 12 = 196,608 blobs at phi = 0.4, placed as hard
    spheres of the hydrodynamic radius (no two centres closer than 2 R_h);
    overlap=True keeps the purely random placement."""
    return roller_suspension(nb, 0.4, seed, overlap=overlap)


def uneven_batch_64(seed: int = 4, n_sys: int = 64):
    """64 boomerang suspensions with body counts log-uniform in [32, 1500]."""
    rng = np.random.default_rng(seed)
    counts = np.floor(np.exp(rng.uniform(np.log(32), np.log(1500), size=n_sys))).astype(int)
    return [boomerang_suspension(int(c), 40.0 * np.sqrt(c / 128), seed * 1000 + s)
            for s, c in enumerate(counts)]
