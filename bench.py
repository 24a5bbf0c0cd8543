"""Benchmark of the wall-RPY rigid-multiblob hot path on GB300.

Workload: 4,369 L-shaped boomerangs x 15 blobs = 65,535 blobs above a no-slip
wall (box scaled to the 128-boomerang / 40 x 40 um density), synthetic and
seeded.  One bench step is one pass of the whole hot path over it (every
step starts from the generated configuration, with its own random draws):
  * one Trapezoidal-Slip time step (Algorithm 2): blob geometry, body-block
    preconditioner, GMRES RFD solve, RFD drift D^F / D^S, preconditioned
    Lanczos M^{1/2} W, predictor and corrector GMRES solves -- FP32 pair
    arithmetic, FP64 Krylov vectors;
  * one batched FP32 wall-RPY matvec with k = 16 right-hand sides.
value = pair interactions per second over the timed steps (n^2 per pair-kernel
launch, summed over every launch inside the step), whole job over all ranks.

--impl reference times the CPU oracle (the plain FP64 program the tests check
against) on the host cores on a bounded sample of the same workload.
"""
import argparse
import ctypes as C
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wall-RPY matvec pairs/s + steps/s, FP32 multi-RHS vs FP64 plain, rel err <=1e-5"
UNIT = "pairs/s"
NB, NPER = 4369, 15
N = NB * NPER
K_RHS = 16
# algorithmic flops of one pair block (FMA = 2, rsqrt = 1): 3 for the separation r_i - r_j, 14 for
# the free-space coefficients, 50 for the wall part, 12 to assemble the nine entries
F_GEOM = 79
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels (profiles/pair_kernel_f32_k16_boomerangs_65535.md, profiles/sym_kernel_f32_k*_boomerangs_65535.md);
# None when not captured
NCU_TRAFFIC = {"f32symf_k1": 5897216 + 0, "f32symf_k2": 9592576 + 0, "f32_k16": 39866880 + 470016}
# FMA-pipe activity (sm__pipe_fma_cycles_active) from the same captures
NCU_FMA_PIPE = {"f32symf_k1": 0.778, "f32symf_k2": 0.769, "f32_k16": 0.795}


F_ASSEMBLY = 12             # flops of forming the 9 entries from the block's 5 scalars


def f_pair(k, symmetric=False, factored=False):
    """Algorithmic flops per ordered pair: one block (F_GEOM) and 9 FMA per
    right-hand side; the symmetric kernel forms one block per unordered pair;
    the factored form skips assembling the 9 entries (still 18 flops per
    right-hand side)."""
    g = F_GEOM - (F_ASSEMBLY if factored else 0)
    return (g / 2 if symmetric else g) + 18 * k


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle accuracy / CPU legs")
    ap.add_argument("--no-rollers", action="store_true", help="skip the 196,608-blob roller T-S step")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default kernels (autotuning under a profiler times the profiler)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the steps only: skip the per-row, batched, roller and single-matvec extras")
    return ap.parse_args()


def workload(seed=1):
    from paper_1709_02410_gb300 import synth
    return synth.boomerang_suspension(NB, 40.0 * np.sqrt(NB / 128), seed)


# ---------------------------------------------------------------------------
# clocks during the timed region

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# replicas: whole-job throughput = pairs summed over ranks / slowest rank's time

def aggregate(t_local, work_local, world, dev):
    if world <= 1:
        return t_local, work_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_local], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ww = torch.tensor([work_local], device=dev, dtype=torch.float64)
    dist.all_reduce(ww, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(ww.item())


# ---------------------------------------------------------------------------
# our arm

def run_ours(args, rank, world, local):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import _native, synth
    from paper_1709_02410_gb300._native import Forces, StepParams

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = workload(seed=1 + rank)
    T = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    h = P.Handle(synth.ETA, s.a, synth.KT)
    lib = h.lib
    shape, q0, th0 = T(s.shape), T(s.q), T(s.theta)
    q, th = q0.clone(), th0.clone()
    F16 = T(synth.gaussian(100 + rank, (K_RHS, 3, N), np.float32), torch.float32)
    U16 = torch.empty_like(F16)
    # gravity m_e g per blob (Sec. 4.1: m_e = 1.57e-11 mg, g = 9.81e6 um/s^2), blob-wall Yukawa
    forces = Forces(1.57e-11 * 9.81e6, 0.096, 0.162, 0.1, (0.0, 0.0, 0.0))
    Lp = 14 * 1.05 * s.a          # arm length: 7 spacings of 2.1 a

    # pick the fastest FP32 kernel variant for this suspension (k = 1: the Krylov matvecs;
    # k = 2: the RFD and predictor solves run in lockstep)
    r0 = h.blobs_from_bodies(shape, q0, th0)
    tuned = h.autotune(r0, 1) if not args.no_autotune else (None, None)
    tuned2 = h.autotune(r0, 2) if not args.no_autotune else (None, None)   # the lockstep RFD + predictor solves
    fma32 = h.measure_fma_peak(P.F32)
    fma64 = h.measure_fma_peak(P.F64)
    fma32v = h.measure_fma_peak(3)   # packed FMAs with three distinct varying register operands

    def sp(i):
        return StepParams(0.01, 1e-3, Lp, 1e-6, 1e-4, 300, 100, 80, P.F32, 2024 + rank, i)

    stats_log = []

    def step(i, from_initial=True):
        # every step advances the generated suspension (new normals per step): a trajectory
        # without steric forces drifts toward interpenetrating bodies, which raises the solver
        # iterations from step to step (33 -> 45 GMRES iterations over 25 steps)
        if from_initial:
            q.copy_(q0)
            th.copy_(th0)
        r = h.blobs_from_bodies(shape, q, th)
        st, status = h.step_ts(shape, q, th, forces, sp(i))
        if status != 0:   # a step whose solves did not converge is not a step
            raise RuntimeError(f"T-S step {i}: status {status}, solver statistics {st}")
        stats_log.append(st)
        h.mobility_apply(r, F16, out=U16)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(i)
    barrier()
    lib.rpbd_profile_read(h.h, 1, 1, C.byref(C.c_double()), C.byref(C.c_longlong()), C.byref(C.c_double()), 1)
    lib.rpbd_profile_enable(h.h, 1)
    stats_log.clear()
    clocks = Clocks(local)
    clocks.start()
    launches0 = lib.rpbd_launch_count()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record()
        step(args.warmup + i)
        ev[i][1].record()
    barrier()
    wall = time.perf_counter() - wall0
    launches = lib.rpbd_launch_count() - launches0
    clk = clocks.stop()
    lib.rpbd_profile_enable(h.h, 0)
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(ms_steps) / 1e3
    # per-variant pair-kernel time from the library's own events
    prof = {}
    for dt, name in ((1, "f32"), (0, "f64"), (3, "f32sym"), (4, "f32symf")):
        for k in (1, 2, 4, 8, 16):
            ms, nl, pr = C.c_double(), C.c_longlong(), C.c_double()
            lib.rpbd_profile_read(h.h, dt, k, C.byref(ms), C.byref(nl), C.byref(pr), 0)
            if nl.value:
                prof[f"{name}_k{k}"] = dict(ms=ms.value, launches=nl.value, pairs=pr.value)
    pairs_local = sum(v["pairs"] for v in prof.values())
    rhs_local = sum(v["launches"] * int(name.split("_k")[1]) for name, v in prof.items())

    # whole job: max time over ranks, pairs summed over ranks
    t_max, pairs_total = aggregate(t_local, pairs_local, world, dev)
    value = pairs_total / t_max

    timed_stats = list(stats_log)

    # ---- end-to-end through the public API with host buffers (same steps)
    qh = torch.empty_like(q0, device="cpu").pin_memory()
    thh = torch.empty_like(th0, device="cpu").pin_memory()
    qo = torch.empty_like(qh).pin_memory()
    tho = torch.empty_like(thh).pin_memory()
    Fh = F16.cpu().pin_memory()
    Uh = torch.empty_like(Fh).pin_memory()
    qh.copy_(q0.cpu())
    thh.copy_(th0.cpu())
    lib.rpbd_profile_read(h.h, 1, 1, C.byref(C.c_double()), C.byref(C.c_longlong()), C.byref(C.c_double()), 1)
    lib.rpbd_profile_enable(h.h, 1)
    barrier()
    e0 = time.perf_counter()
    for i in range(args.steps):
        q.copy_(qh, non_blocking=True)
        th.copy_(thh, non_blocking=True)
        F16.copy_(Fh, non_blocking=True)
        step(1000 + i, from_initial=False)
        qo.copy_(q, non_blocking=True)
        tho.copy_(th, non_blocking=True)
        Uh.copy_(U16, non_blocking=True)
        torch.cuda.synchronize()
    barrier()
    e2e_t = time.perf_counter() - e0
    lib.rpbd_profile_enable(h.h, 0)
    e2e_pairs = 0.0
    for dt in (1, 0, 3, 4):
        for k in (1, 2, 4, 8, 16):
            ms, nl, pr = C.c_double(), C.c_longlong(), C.c_double()
            lib.rpbd_profile_read(h.h, dt, k, C.byref(ms), C.byref(nl), C.byref(pr), 0)
            e2e_pairs += pr.value
    lib.rpbd_profile_read(h.h, 1, 1, C.byref(C.c_double()), C.byref(C.c_longlong()), C.byref(C.c_double()), 1)
    h2d = q0.numel() * 8 + th0.numel() * 8 + F16.numel() * 4
    d2h = h2d
    e2e_t, e2e_pairs = aggregate(e2e_t, e2e_pairs, world, dev)

    # ---- separate measurements (outside the timed steps): k = 16 FP32 batch and
    # the plain FP64 single-RHS kernel, each alone, and their accuracy
    r = h.blobs_from_bodies(shape, q0, th0)
    extra = None

    def time_launch(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps / 1e3

    extras = not args.no_extras
    if extras:
        extra, F1, U1 = measure_matvecs(h, r, F16, U16, T, time_launch)
    row_times = measure_rows(h, r, shape, q0, th0, T, time_launch) if (rank == 0 and extras) else None
    batched = measure_batched(h.lib, dev, T) if (rank == 0 and extras) else None
    rollers = measure_rollers(dev, T) if (rank == 0 and extras and not args.no_rollers) else None
    next_rows = measure_next_rows(dev, T, s, shape, q0, th0, forces, Lp) if (rank == 0 and extras) else None
    rfd_div = measure_rfd_vs_divergence(T) if (rank == 0 and extras) else None

    out = None
    if rank == 0:
        # dominant pair-kernel variant of the step -> roofline
        dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
        roof = None
        if dom:
            name, d = dom
            k = int(name.split("_k")[1])
            sym = name.startswith("f32sym")
            fac = name.startswith("f32symf")
            avg = d["ms"] / d["launches"] / 1e3
            flops = d["pairs"] / d["launches"] * f_pair(k, sym, fac)
            ach = flops / avg / 1e12
            roof = {"bound": "alu", "kernel": f"pair_kernel<{name}>", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get(name),
                    "flops_per_pair": f_pair(k, sym, fac), "avg_launch_ms": avg * 1e3,
                    "one_direction_equivalent_tflops":
                        d["pairs"] / d["launches"] * f_pair(k) / avg / 1e12,
                    "share_of_step": d["ms"] / (t_local * 1e3),
                    "measured_fma_peak": fma32, "frac_of_measured_fma_peak": ach / fma32,
                    "ncu_fma_pipe_active": NCU_FMA_PIPE.get(name),
                    "three_varying_operand_fma_rate": fma32v,
                    "peak_note": "peak = 152 SMs x 128 FP32 lanes x 2 x 2.070 GHz (derived); "
                                 "measured_fma_peak = the library's FMA-chain probe on this GPU; "
                                 "three_varying_operand_fma_rate = the same probe when every packed FMA reads "
                                 "three distinct varying registers (the register file's ceiling for such code)"}
        # accuracy vs the FP64 oracle on sampled rows (outside the timed region)
        acc = {}
        if extras and not args.no_oracle:
            from oracle import mobility as om
            from oracle import rigid
            ro = rigid.blob_positions(s.q, s.theta, s.shape)
            prm = om.Params(synth.ETA, s.a)
            rows = np.random.default_rng(5).choice(N, 32, replace=False)
            Fo = F16.cpu().numpy().astype(np.float64)
            Uo = om.apply(ro, Fo, prm, rows=rows)
            Ug = U16.cpu().numpy()[:, :, rows].astype(np.float64)
            acc["f32_k16_rel_err_vs_oracle"] = float(np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo))
            U1o = om.apply(ro, F1.cpu().numpy(), prm, rows=rows)
            acc["f64_k1_rel_err_vs_oracle"] = float(np.linalg.norm(U1.cpu().numpy()[:, rows] - U1o)
                                                    / np.linalg.norm(U1o))
            acc["rows_sampled"] = len(rows)
            # CPU baseline: the oracle as it stands, bounded sample (rows x all sources, k = 16)
            nrows = 4096
            rows_b = np.arange(nrows)
            t0 = time.perf_counter()
            om.apply(ro, Fo, prm, rows=rows_b)
            tc = time.perf_counter() - t0
            cpu = {"value": nrows * N / tc, "unit": UNIT, "cores": om.num_threads(), "kind": "oracle",
                   "sample": f"{nrows} target rows x {N} sources, k = 16, FP64 ({tc:.1f} s)"}
            # the same oracle on one core (smaller row sample)
            ncores = om.num_threads()
            om.set_num_threads(1)
            rows_1 = np.arange(256)
            t0 = time.perf_counter()
            om.apply(ro, Fo, prm, rows=rows_1)
            t1c = time.perf_counter() - t0
            om.set_num_threads(ncores)
            cpu["one_core"] = {"value": len(rows_1) * N / t1c, "unit": UNIT, "cores": 1,
                               "sample": f"{len(rows_1)} target rows x {N} sources, k = 16, FP64 ({t1c:.1f} s)"}
        else:
            cpu = None
        iters = [[x["iterations"] for x in st] for st in timed_stats]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded boomerang suspension, forces N(0,1))",
            "config": bench_config(world),
            "steps_per_s": args.steps / t_max * world,
            "matvecs_per_s": rhs_local * world / t_max,
            "e2e": {"value": e2e_pairs / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "pair_kernels_in_step": prof,
            "solver_iterations_per_step": iters,
            # M applications (right-hand sides) per T-S step, without the k = 16 batch; the
            # paper's count is n_G per saddle solve x 3 + n_L + 2 (two RFD matvecs)
            "m_applies_per_ts_step": {
                "measured": (rhs_local - K_RHS * prof.get("f32_k16", {}).get("launches", 0)) / args.steps,
                "iterations_plus_2": sum(sum(x) + 2 for x in iters) / max(1, len(iters))},
            "autotune_k1": {"choice": tuned[0], "ms_per_launch": tuned[1],
                            "legend": "0: one-direction kernel; 1 + v: symmetric kernel variant v"},
            "autotune_k2": {"choice": tuned2[0], "ms_per_launch": tuned2[1]},
            "measured_fma_peak_tflops": {"f32": fma32, "f64": fma64, "f32_packed_three_varying_operands": fma32v},
            "matvec": extra,
            "rows": row_times,
            "batched_uneven_64": batched,
            "ts_step_rollers_196608": rollers,
            "next_rows": next_rows,
            "rfd_vs_divergence_16380": rfd_div,
            "accuracy": acc,
            "wall_s_timed": wall,
        }
    return out


# ---------------------------------------------------------------------------
# every step of the hot path timed alone on the bench suspension

def measure_matvecs(h, r, F16, U16, T, time_launch):
    """k = 16 FP32 batch, k = 1 FP32 (symmetric and one-direction) and the
    plain FP64 single-RHS kernel, each timed alone."""
    import torch
    from paper_1709_02410_gb300 import synth
    extra = {}
    t16 = time_launch(lambda: h.mobility_apply(r, F16, out=U16), 3)
    F1 = T(synth.gaussian(200, (3, N)))
    U1 = torch.empty_like(F1)
    t64 = time_launch(lambda: h.mobility_apply(r, F1, out=U1), 1)
    F1f = F1.float()
    U1f = torch.empty_like(F1f)
    t32k1 = time_launch(lambda: h.mobility_apply(r, F1f, out=U1f), 3)
    extra["f32_k16"] = dict(s_per_launch=t16, pairs_per_s=N * N / t16, matvecs_per_s=K_RHS / t16,
                            tflops=N * N * f_pair(16) / t16 / 1e12)
    extra["f32_k1_symmetric"] = dict(s_per_launch=t32k1, pairs_per_s=N * N / t32k1,
                                     tflops=N * N * f_pair(1, True, True) / t32k1 / 1e12)
    h.set_symmetric(False)
    t32k1d = time_launch(lambda: h.mobility_apply(r, F1f, out=U1f), 3)
    h.set_symmetric(True)
    extra["f32_k1_one_direction"] = dict(s_per_launch=t32k1d, pairs_per_s=N * N / t32k1d,
                                         tflops=N * N * f_pair(1) / t32k1d / 1e12)
    for kk in (2, 4, 8):
        Fk = T(synth.gaussian(210 + kk, (kk, 3, N)), torch.float32)
        Uk = torch.empty_like(Fk)
        tk = time_launch(lambda: h.mobility_apply(r, Fk, out=Uk), 3)
        sym = kk <= 4
        extra[f"f32_k{kk}"] = dict(s_per_launch=tk, pairs_per_s=N * N / tk, matvecs_per_s=kk / tk,
                                   kernel="symmetric" if sym else "one-direction",
                                   tflops=N * N * f_pair(kk, sym, sym) / tk / 1e12)  # packed: factored form
    # the packed symmetric kernel with per-home-tile partials and the fixed-order reduction
    # (instead of the fixed-point accumulation), and with the cancellation-free far field
    for mode, setter in (("partials", h.set_sym_partials), ("far_field", h.set_far_field)):
        setter(True)
        for kk in (1, 2):
            Fk = F1f if kk == 1 else T(synth.gaussian(212, (2, 3, N)), torch.float32)
            Uk = torch.empty_like(Fk)
            tk = time_launch(lambda: h.mobility_apply(r, Fk, out=Uk), 3)
            extra[f"f32_k{kk}_symmetric_{mode}"] = dict(s_per_launch=tk, pairs_per_s=N * N / tk)
        setter(False)
    extra["f64_k1"] = dict(s_per_launch=t64, pairs_per_s=N * N / t64)
    extra["speedup_f32_k16_vs_f64_k1_per_rhs"] = (t64 * K_RHS) / t16
    extra["speedup_f32_k1_vs_f64_k1"] = t64 / t32k1
    return extra, F1, U1


def measure_rows(h, r, shape, q, th, T, time_launch):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import synth
    n = r.shape[1]
    W = T(synth.gaussian(400, (3, n)))
    u = T(synth.gaussian(401, (3, n)))
    FT = T(synth.gaussian(402, (NB, 6)) * 1e-2)
    out = {}
    out["a1_blob_geometry_s"] = time_launch(lambda: h.blobs_from_bodies(shape, q, th, out=r), 5)
    out["a3_precond_build_s"] = time_launch(lambda: h.precond_build(NPER, r, q), 3)
    st = {}

    def lz():
        st["l"] = h.lanczos_sqrt_apply(r, W, 1e-4, 80, dtype=P.F32)[1]
    out["a4_lanczos_tol1e-4_s"] = time_launch(lz, 2)
    out["a4_lanczos_iterations"] = st["l"]["iterations"]
    # four Brownian increments in lockstep (shared k = 4 matvecs) vs four separate runs
    W4 = [T(synth.gaussian(410 + i, (3, n))) for i in range(4)]

    def lz4():
        st["l4"] = h.lanczos_sqrt_apply_multi(r, W4, tol=1e-4, max_iter=80, dtype=P.F32)
    out["a4_lanczos_x4_lockstep_s"] = time_launch(lz4, 2)
    out["a4_lanczos_x4_iterations"] = [x[1]["iterations"] for x in st["l4"]]

    def gm():
        st["g"] = h.gmres_rigid_solve(NPER, r, q, W, FT, tol=1e-6, max_iter=300, restart=100, dtype=P.F32,
                                      build_precond=False)[2]
    out["a5_gmres_tol1e-6_s"] = time_launch(gm, 2)
    out["a5_gmres_iterations"] = st["g"]["iterations"]
    out["a6_rfd_drift_s"] = time_launch(lambda: h.rfd_drift(r, W, 1e-3, dtype=P.F32), 3)
    out["a7_adjoint_f32_s"] = time_launch(lambda: h.mobility_adjoint(r, u, W, dtype=P.F32), 1)
    out["a7_adjoint_f32_pairs_per_s"] = n * n / out["a7_adjoint_f32_s"]
    # blob forces with the blob-blob Yukawa repulsion of Sec. 4.1 (gamma = 0.096, b = 0.162 um), no cut-off
    fst = P.Forces(1.57e-11 * 9.81e6, 0.096, 0.162, 0.1, (0.0, 0.0, 0.0), 0.096, 0.162, 0.1, 0.0)
    fb = torch.empty_like(r)
    out["f4_steric_forces_f32_s"] = time_launch(lambda: h.blob_forces(r, fst, nper=NPER, dtype=P.F32, out=fb), 3)
    return out


# ---------------------------------------------------------------------------
# the other integrators (f2) on the bench suspension, and the pseudo-periodic
# cell (f1): the bench suspension in a periodic box, and the paper's 256
# boomerangs in a 45.3 um cell

def measure_next_rows(dev, T, s, shape, q0, th0, forces, Lp):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import synth
    from paper_1709_02410_gb300._native import StepParams
    out = {}
    sp = lambda i: StepParams(0.01, 1e-3, Lp, 1e-6, 1e-4, 300, 100, 80, P.F32, 99, i)
    h = P.Handle(synth.ETA, s.a, synth.KT)
    for kind in ("emt", "emrfd", "tt"):
        q, th = q0.clone(), th0.clone()
        fn = getattr(h, "step_" + kind)
        fn(shape, q, th, forces, sp(0))          # warm-up: workspace, plans
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st, status = fn(shape, q, th, forces, sp(1))
        e1.record()
        torch.cuda.synchronize()
        out[f"f2_step_{kind}_s"] = e0.elapsed_time(e1) / 1e3
        out[f"f2_step_{kind}_iterations"] = [x["iterations"] for x in st]
    # f1: periodic images, k = 1 FP32 matvec (9 images per pair) on the bench suspension
    L = 40.0 * np.sqrt(NB / 128)
    hp = P.Handle(synth.ETA, s.a, synth.KT, Lx=L, Ly=L)
    r = hp.blobs_from_bodies(shape, q0, th0)
    F = T(synth.gaussian(500, (1, 3, r.shape[1])), torch.float32)
    U = torch.empty_like(F)
    hp.mobility_apply(r, F, out=U)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        hp.mobility_apply(r, F, out=U)
    e1.record()
    torch.cuda.synchronize()
    tp = e0.elapsed_time(e1) / 2e3
    out["f1_periodic_f32_k1_s"] = tp
    out["f1_periodic_pair_images_per_s"] = 9.0 * r.shape[1] ** 2 / tp
    # f1: T-S step of the paper's periodic boomerang suspension (256 bodies, 45.3 um cell, Sec. 4.2)
    sc = synth.boomerang_suspension(256, 45.3, 7)
    hc = P.Handle(synth.ETA, sc.a, synth.KT, Lx=45.3, Ly=45.3)
    shc, qc, thc = T(sc.shape), T(sc.q), T(sc.theta)
    hc.step_ts(shc, qc, thc, forces, sp(0))
    torch.cuda.synchronize()
    e0.record()
    st, status = hc.step_ts(shc, qc, thc, forces, sp(1))
    e1.record()
    torch.cuda.synchronize()
    out["f1_ts_step_256_boomerangs_periodic_s"] = e0.elapsed_time(e1) / 1e3
    out["f1_ts_step_256_boomerangs_iterations"] = [x["iterations"] for x in st]
    return out


# ---------------------------------------------------------------------------
# The exact divergence of M (FP64 dual-number kernel) against the
# mean of the blob RFD drift over 10^4 random W (Sec. 3), 16,380 blobs

def measure_rfd_vs_divergence(T, samples=10000, chunk=250):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import synth
    s = synth.blobs_16384()
    h = P.Handle(synth.ETA, s.a, synth.KT)
    r = h.blobs_from_bodies(T(s.shape), T(s.q), T(s.theta))
    n = r.shape[1]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    div = h.mobility_divergence(r)
    e1.record()
    torch.cuda.synchronize()
    t_div = e0.elapsed_time(e1) / 1e3
    gen = torch.Generator(device=r.device).manual_seed(2024)
    acc = torch.zeros((3, n), dtype=torch.float64, device=r.device)
    acc2 = torch.zeros_like(acc)
    d = torch.empty((3, n), dtype=torch.float64, device=r.device)
    e0.record()
    for c0 in range(0, samples, chunk):
        Ws = torch.randn((chunk, 3, n), dtype=torch.float64, device=r.device, generator=gen)
        for i in range(chunk):
            h.rfd_drift(r, Ws[i], 1e-3, dtype=P.F32, out=d)
            acc += d
            acc2 += d * d
    e1.record()
    torch.cuda.synchronize()
    t_rfd = e0.elapsed_time(e1) / 1e3
    mean = acc / samples
    se = torch.sqrt(torch.clamp(acc2 / samples - mean * mean, min=0.0) / samples)
    z = (mean - div).abs() / (se + 1e-300)
    return {"n_blobs": n, "samples": samples, "rfd_delta": 1e-3, "rfd_dtype": "f32 pairs",
            "frac_within_3se": float((z < 3).double().mean()), "max_z": float(z.max()),
            "rel_err_mean_vs_div": float(torch.linalg.norm(mean - div) / torch.linalg.norm(div)),
            "rel_se": float(torch.linalg.norm(se) / torch.linalg.norm(div)),
            "divergence_s": t_div, "rfd_s_per_sample": t_rfd / samples}


# ---------------------------------------------------------------------------
# full T-S step on the dense microroller suspension: 16,384 rollers x 12 blobs

def measure_rollers(dev, T, steps=5):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import synth
    from paper_1709_02410_gb300._native import Forces, StepParams
    s = synth.rollers_196608()
    h = P.Handle(synth.ETA, s.a, synth.KT)
    shape, q, th = T(s.shape), T(s.q), T(s.theta)
    # buoyant weight m_e g = 1.24e-14 N = 1.24e-2 mg um/s^2 per roller, shared by its 12 blobs;
    # constant torque 1.0 about +y on every roller; blob-wall Yukawa as for the boomerangs
    forces = Forces(1.24e-2 / 12, 0.096, 0.162, 0.1, (0.0, 1.0, 0.0))
    sp = lambda i: StepParams(0.008, 1e-3, synth.RH_ROLLER, 1e-6, 1e-4, 300, 100, 80, P.F32, 77, i)
    def checked(st, status, i):
        if status != 0:
            raise RuntimeError(f"roller T-S step {i}: status {status}, solver statistics {st}")
        return [x["iterations"] for x in st]

    checked(*h.step_ts(shape, q, th, forces, sp(0)), 0)          # warm-up: workspace, plans
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its = []
    for i in range(steps):
        ev[i][0].record()
        its.append(checked(*h.step_ts(shape, q, th, forces, sp(1 + i)), 1 + i))
        ev[i][1].record()
    torch.cuda.synchronize()
    ts = [a.elapsed_time(b) / 1e3 for a, b in ev]
    t = sum(ts) / steps
    mv = [it[0] + it[1] + it[2] + it[3] + 2 for it in its]
    # one more step at the paper's tolerances (GMRES and Lanczos to 1e-3, Sec. 4.2), to set the
    # matvec count beside the paper's 22 per T-S step
    sp3 = StepParams(0.008, 1e-3, synth.RH_ROLLER, 1e-3, 1e-3, 300, 100, 80, P.F32, 77, 100)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    it3 = checked(*h.step_ts(shape, q, th, forces, sp3), 100)
    e1.record()
    torch.cuda.synchronize()
    # the same suspension placed purely at random (rollers interpenetrating), for comparison
    so = synth.rollers_196608(overlap=True)
    qo, tho = T(so.q), T(so.theta)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    ito = checked(*h.step_ts(shape, qo, tho, forces, sp(200)), 200)
    e3.record()
    torch.cuda.synchronize()
    return {"workload": "rollers_196608: 16384 x 12-blob rollers, phi = 0.4, hard-sphere placement (centres >= 2 R_h)",
            "n_blobs": s.n, "steps": steps,
            "s_per_step": t, "s_per_step_each": ts, "steps_per_s": 1.0 / t,
            "iterations_rfd_lanczos_pred_corr": its, "matvecs_per_step": mv,
            "gmres_tol": 1e-6, "lanczos_tol": 1e-4, "dt": 0.008, "dtype": "f32 pairs, f64 Krylov",
            "status": "every timed step converged (status 0)",
            "paper_tolerances_1e-3": {"iterations_rfd_lanczos_pred_corr": it3,
                                      "matvecs_per_step": sum(it3) + 2, "s_per_step": e0.elapsed_time(e1) / 1e3},
            "random_overlapping_placement": {"iterations_rfd_lanczos_pred_corr": ito, "matvecs_per_step": sum(ito) + 2,
                                             "s_per_step": e2.elapsed_time(e3) / 1e3}}


# ---------------------------------------------------------------------------
# uneven batch: 64 boomerang suspensions, body counts log-uniform in [32, 1500]

def measure_batched(lib, dev, T, tol=1e-4, max_iter=60):
    import torch
    import paper_1709_02410_gb300 as P
    from paper_1709_02410_gb300 import synth
    systems = synth.uneven_batch_64()
    a = systems[0].a
    hb = P.Handle(synth.ETA, a, synth.KT)
    shape = T(systems[0].shape)
    q = T(np.concatenate([s.q for s in systems]))
    th = T(np.concatenate([s.theta for s in systems]))
    r = hb.blobs_from_bodies(shape, q, th)
    counts = [s.n for s in systems]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(off[-1])
    W = T(synth.gaussian(300, (3, n)))
    F = T(synth.gaussian(301, (3, n)))
    hb.precond_build(15, r, q)
    variant, tune_ms = hb.autotune_batched(off, r, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out, U, iters = hb.lanczos_sqrt_apply_batched(off, r, W, tol, max_iter, use_graph=True, F=F)  # capture
    reps = 3
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        out, U, iters = hb.lanczos_sqrt_apply_batched(off, r, W, tol, max_iter, use_graph=True, F=F, out=out, U=U)
    ev1.record()
    torch.cuda.synchronize()
    t_graph = ev0.elapsed_time(ev1) / 1e3 / reps
    # per-system loop of plain launches: one handle per system, its own
    # preconditioner built beforehand, host-driven Lanczos + one matvec
    hs, rs, Ws, Fs = [], [], [], []
    for si, s in enumerate(systems):
        hi = P.Handle(synth.ETA, a, synth.KT)
        ri = r[:, off[si]:off[si + 1]].contiguous()
        hi.precond_build(15, ri, q[sum(c // 15 for c in counts[:si]):sum(c // 15 for c in counts[:si + 1])].contiguous())
        hs.append(hi)
        rs.append(ri)
        Ws.append(W[:, off[si]:off[si + 1]].contiguous())
        Fs.append(F[:, off[si]:off[si + 1]].contiguous())
    def loop():
        it = []
        for hi, ri, wi, fi in zip(hs, rs, Ws, Fs):
            _, st = hi.lanczos_sqrt_apply(ri, wi, tol, max_iter, dtype=P.F32)
            hi.mobility_apply(ri, fi, dtype=P.F32)
            it.append(st["iterations"])
        return it
    loop()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_loop = loop()
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    pairs = float(sum(c * c for c in counts))
    mv = sum(iters) and (max(iters) + 1)
    return {"n_sys": len(systems), "blobs": n, "pairs_per_matvec": pairs, "autotuned_variant": variant,
            "autotune_ms_per_launch": tune_ms, "graph_s": t_graph, "loop_s": t_loop,
            "speedup_graph_vs_loop": t_loop / t_graph, "lanczos_iters_min_max": [min(iters), max(iters)],
            "loop_iters_min_max": [min(it_loop), max(it_loop)],
            "pairs_per_s_graph": pairs * (sum(iters) / len(iters) + 1) / t_graph,
            "tol": tol, "dtype": "f32 pairs, f64 vectors"}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, bounded sample of the same workload

def bench_config(world):
    """the workload both arms report"""
    return {"workload": "boomerangs_65535: 4369 L-bodies x 15 blobs, T-S step + k=16 FP32 batch",
            "n_blobs": N, "n_bodies": NB, "k_rhs": K_RHS, "gmres_tol": 1e-6, "gmres_restart": 100,
            "lanczos_tol": 1e-4, "rfd_delta": 1e-3, "gmres_x0": "corrector starts from the predictor's solution",
            "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import mobility as om
    from oracle import rigid
    from paper_1709_02410_gb300 import synth
    s = workload(1)
    ro = rigid.blob_positions(s.q, s.theta, s.shape)
    prm = om.Params(synth.ETA, s.a)
    F = synth.gaussian(100, (K_RHS, 3, N), np.float32).astype(np.float64)
    # enough rows per step that the call's fixed cost (argument conversion,
    # thread start) stays small next to the pair sums: ~1.5 s per step
    nrows = 512

    def step(i):
        rows = np.arange(i * nrows, (i + 1) * nrows) % N
        om.apply(ro, F, prm, rows=rows)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    t = time.perf_counter() - t0
    v = args.steps * nrows * N / t
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": bench_config(world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": om.num_threads(), "kind": "oracle",
                             "sample": f"each step: {nrows} target rows x {N} sources of the same suspension, "
                                       f"k = 16, FP64 (the oracle's pair interactions per second)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, local)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
