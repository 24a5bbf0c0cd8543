"""Solver iteration counts against system size (the study of Sec. 2.2,
Fig. BoomResidual): boomerang suspensions of 256, 1024 and 4096 bodies at the
density of the paper's 256 boomerangs in a 45.3 um pseudo-periodic cell.
For each tolerance it reports the iterations of the preconditioned GMRES
saddle solve, the preconditioned Lanczos M^{1/2} W and the unpreconditioned
Lanczos.  With the block preconditioner the counts should not grow with N.

    python -m paper_1709_02410_gb300.iteration_study [--dtype f32|f64]
"""
import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--sizes", default="256,1024,4096")
    ap.add_argument("--tols", default="1e-2,1e-3,1e-4,1e-6")
    a = ap.parse_args()
    import torch
    from . import F32, F64, Handle, synth
    dt = F32 if a.dtype == "f32" else F64
    out = []
    for nb in [int(x) for x in a.sizes.split(",")]:
        Lc = 45.3 * np.sqrt(nb / 256)
        s = synth.boomerang_suspension(nb, Lc, 7)
        h = Handle(synth.ETA, s.a, synth.KT, Lx=Lc, Ly=Lc)
        T = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")
        r = h.blobs_from_bodies(T(s.shape), T(s.q), T(s.theta))
        q = T(s.q)
        W = T(synth.gaussian(8, (3, s.n)))
        FT = T(synth.gaussian(9, (s.nb, 6)) * 1e-2)
        h.precond_build(s.nper, r, q)
        row = {"bodies": nb, "blobs": s.n, "cell_um": Lc}
        for tol in [float(x) for x in a.tols.split(",")]:
            _, _, st = h.gmres_rigid_solve(s.nper, r, q, W, FT, tol=tol, max_iter=400, restart=100, dtype=dt,
                                           build_precond=False)
            _, l1 = h.lanczos_sqrt_apply(r, W, tol=tol, max_iter=80, dtype=dt, use_precond=True)
            _, l2 = h.lanczos_sqrt_apply(r, W, tol=tol, max_iter=80, dtype=dt, use_precond=False)
            row[f"tol={tol:g}"] = {"gmres": st["iterations"], "pc_lanczos": l1["iterations"],
                                   "unpc_lanczos": l2["iterations"]}
        out.append(row)
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
