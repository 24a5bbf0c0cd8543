"""Time one wall-RPY matvec variant on synthetic boomerangs (CUDA events).

    python -m paper_1709_02410_gb300.profile_case --n 65535 --k 16 --dtype f32 --reps 5
    python -m paper_1709_02410_gb300.profile_case --batched --k 1 --reps 5     # 64 uneven suspensions
    python -m paper_1709_02410_gb300.profile_case --adjoint --n 65535 --reps 3 # FP32 adjoint (--k: RHS pairs)

Prints one JSON line: seconds per launch (pack + pair kernel + reduce),
pairs/s and matvecs/s.  Useful on its own and as the target of profilers.
"""
import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65535, help="blobs (rounded down to whole 15-blob bodies)")
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--wall", type=int, default=1)
    ap.add_argument("--sym", type=int, default=1, help="FP32 k <= 4: symmetric kernel (1) or one-direction (0)")
    ap.add_argument("--variant", type=int, default=-1, help="symmetric kernel variant 0..5 (-1: default)")
    ap.add_argument("--batched", action="store_true",
                    help="the uneven batch of 64 boomerang suspensions (one batched launch; --variant: tile variant)")
    ap.add_argument("--adjoint", action="store_true", help="the FP32 adjoint instead of the matvec")
    ap.add_argument("--partials", action="store_true",
                    help="partial sums with the fixed-order reduction (not the fixed-point accumulation)")
    ap.add_argument("--far", action="store_true", help="cancellation-free far field")
    a = ap.parse_args()
    import torch
    from . import F32, F64, Handle, synth
    if a.batched:
        return batched(a)
    if a.adjoint:
        return adjoint(a)
    nb = max(1, a.n // 15)
    s = synth.boomerang_suspension(nb, 40.0 * np.sqrt(nb / 128), 1)
    dev = "cuda:0"
    h = Handle(synth.ETA, s.a, synth.KT, wall=bool(a.wall))
    h.set_symmetric(bool(a.sym))
    h.set_sym_variant(a.variant)
    h.set_sym_partials(a.partials)
    h.set_far_field(a.far)
    T = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    r = h.blobs_from_bodies(T(s.shape), T(s.q), T(s.theta))
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    F = T(synth.gaussian(7, (a.k, 3, s.n)), dt)
    U = torch.empty_like(F)
    h.mobility_apply(r, F, out=U)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        h.mobility_apply(r, F, out=U)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / a.reps
    print(json.dumps({"n": s.n, "k": a.k, "dtype": a.dtype, "sym": a.sym, "variant": a.variant, "partials": a.partials,
                      "far": a.far,
                      "s_per_launch": t, "pairs_per_s": s.n * s.n / t,
                      "matvecs_per_s": a.k / t}))


def batched(a):
    import torch
    from . import Handle, synth
    systems = synth.uneven_batch_64()
    h = Handle(synth.ETA, systems[0].a, synth.KT)
    if a.variant >= 0:
        h.set_batch_variant(a.variant)
    h.set_sym_partials(a.partials)
    dev = "cuda:0"
    T = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    shape = T(systems[0].shape)
    q = T(np.concatenate([s.q for s in systems]))
    th = T(np.concatenate([s.theta for s in systems]))
    r = h.blobs_from_bodies(shape, q, th)
    off = np.concatenate([[0], np.cumsum([s.n for s in systems])]).astype(np.int64)
    F = T(synth.gaussian(7, (a.k, 3, int(off[-1]))), torch.float32)
    U = h.mobility_apply_batched(off, r, F)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        U = h.mobility_apply_batched(off, r, F)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / a.reps
    pairs = float(sum(float(s.n) ** 2 for s in systems))
    print(json.dumps({"batched": len(systems), "blobs": int(off[-1]), "k": a.k, "variant": a.variant,
                      "partials": a.partials,
                      "s_per_launch": t, "pairs_per_s": pairs / t}))


def adjoint(a):
    import torch
    from . import F32, Handle, synth
    nb = max(1, a.n // 15)
    s = synth.boomerang_suspension(nb, 40.0 * np.sqrt(nb / 128), 1)
    h = Handle(synth.ETA, s.a, synth.KT)
    dev = "cuda:0"
    T = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    r = h.blobs_from_bodies(T(s.shape), T(s.q), T(s.theta))
    shp = (3, s.n) if a.k == 1 else (a.k, 3, s.n)   # k right-hand-side pairs, summed
    u, F = T(synth.gaussian(8, shp)), T(synth.gaussian(9, shp))
    g = h.mobility_adjoint(r, u, F, dtype=F32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        g = h.mobility_adjoint(r, u, F, dtype=F32)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / a.reps
    print(json.dumps({"adjoint_f32": True, "n": s.n, "k": a.k, "s_per_launch": t, "pairs_per_s": s.n * s.n / t}))


if __name__ == "__main__":
    main()
