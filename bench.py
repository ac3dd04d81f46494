#!/usr/bin/env python
"""Benchmark: time to a 1e-8 relative residual of the all-at-once RK heat solve.

Workload (one step = one full solve, FP64 FGMRES(20) outer + P_tilde):
  2D 256x256 interior FD grid (M = I), Radau IIA s = 3, 128 steps to T = 1,
  u0 and f seeded Gaussian random fields (squared-exponential, l = 0.1,
  unit variance), f constant in time; n_st = 33,619,968 space-time unknowns.
  The timed solve applies P_tilde in FP32 (Theta_tilde GMRES 3 / 1e-3, 3
  V-cycles); the same problem is also solved once with P_tilde in FP64
  (GMRES 5 / 1e-6) for the mixed-vs-FP64 comparison.

Timing: W warm-up solves, then K solves between CUDA events on the solver's
stream with a barrier and a synchronize on both sides; the working set
(x 269 MB, Krylov basis ~11 GB) is far larger than L2.  `e2e` repeats the
solve through the C ABI with pinned host buffers (copies inside the timed
region).  `roofline` times every launch of the dominant kernel with CUDA
events during one extra solve and divides its algorithmic bytes by that time.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual, mixed vs FP64 precond, same GB300; precond HBM GB/s"
WORKLOAD = "fd2d_n256_radau3_nt128"
# dram__bytes_read.sum + dram__bytes_write.sum of one k_cluster_mg launch (single-item 256x256
# shifted solve, FP32 storage, 512-thread CTAs), from one ncu capture of the current kernel; the
# kernel's inputs are L2-resident, so this is far below its algorithmic bytes
CLUSTER_MG_DRAM_BYTES = 1364


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp16"])
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-preconditioner comparison solve")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--small", action="store_true", help="64x64, nt 16 (quick check; not a bench value)")
    p.add_argument("--workload", default="fd2d_n256_radau3_nt128",
                   choices=["fd2d_n256_radau3_nt128", "fd3d_n96_radau3_nt32", "fd3d_n96_gauss2_nt32", "batched64"],
                   help="extra configurations (the default is the benchmark line)")
    p.add_argument("--precond-case", action="store_true",
                   help="small case for profiler captures: --steps applications of P_tilde (FP32) on the "
                        "256x256 Radau IIA s=3 grid with 16 time steps; prints ms per application")
    return p.parse_args()


def workload(small: bool, name: str = WORKLOAD):
    import synth
    if small:
        return synth.workload_fp32_precond_2d(N=64, nt=16, s=3)
    if name == "fd3d_n96_radau3_nt32":
        return synth.workload_lowprec_3d(method="radau", s=3)
    if name == "fd3d_n96_gauss2_nt32":
        return synth.workload_lowprec_3d(method="gauss", s=2)
    return synth.workload_fp32_precond_2d()


def batched_arm(args):
    """64 uneven 2D problems in one aao_rk_solve_batched call (one stream each)."""
    import torch
    import synth
    from paper_2609_16863_gb300 import Solver, _lib, radau_iia, solve_batched
    dev = torch.device("cuda", 0)
    ws = synth.workload_batched()
    solvers, fs, us, xs = [], [], [], []
    for w in ws:
        st = torch.cuda.Stream(device=dev)
        solvers.append(Solver(w.n, w.T, w.nt, tableau=radau_iia(w.s), prec_P=args.prec, inner_maxit=3,
                              inner_tol=1e-3, tol=w.tol, stream=st.cuda_stream))
        fs.append(torch.from_numpy(w.f).to(dev))
        us.append(torch.from_numpy(w.u0).to(dev))
        xs.append(torch.zeros(solvers[-1].n_st, dtype=torch.float64, device=dev))
    for _ in range(args.warmup):
        solve_batched(solvers, fs, us, xs)
    torch.cuda.synchronize()
    times = []
    lat = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        infos = solve_batched(solvers, fs, us, xs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        lat += [i.t_total_ms for i in infos]
    t = float(np.median(times))
    nst = sum(S.n_st for S in solvers)
    its = [i.outer_its for i in infos]
    line = {"metric": "batched uneven solves to 1e-8: wall time of the batch", "value": t, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": f"f64/{args.prec}",
            "data": "synthetic", "config": {"workload": "batched64", "problems": len(ws), "n_st_total": nst},
            "dofs_its_per_s": sum(S.n_st * i for S, i in zip(solvers, its)) / t,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "outer_its_min_max": [min(its), max(its)], "all_converged": all(i.converged for i in infos)}
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (each rank times its own replica); world == 1: itself."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.close()
        rows = []
        for ln in open(self.tmp.name):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(w, outer_its: int, budget_s: float = 20.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the workload.

    Sample: one all-at-once matvec and inner Theta_tilde solves (the unit of work
    P_tilde repeats 2*nt times per application) at full size, for about
    budget_s seconds; the oracle's time to solution is estimated as
    outer_its * (2 nt t_inner + 2 t_matvec) + t_ortho(outer_its).  `cores` is the
    process CPU time divided by the wall time of the sample.
    """
    from oracle.precond import Preconditioner
    from oracle.solve import build
    op = build(w.n, w.T, w.nt, w.method, w.s)
    P = Preconditioner(op, w.n, inner_maxit=3, inner_tol=1e-3, mg_cycles=3, nu1=2, nu2=2, omega=0.8)
    x = np.random.default_rng(0).standard_normal(op.n_st)
    c0, w0 = time.process_time(), time.perf_counter()
    t0 = time.perf_counter()
    op.matvec(x)
    t_mv = time.perf_counter() - t0
    r = x[op.n_v: op.n_v + w.s * op.nx].copy()
    n_inner = 0
    t0 = time.perf_counter()
    while True:
        P.inner_solve(r)
        n_inner += 1
        if time.perf_counter() - t0 > budget_s * 0.8 or n_inner >= 200:
            break
    t_inner = (time.perf_counter() - t0) / n_inner
    t0 = time.perf_counter()
    basis = [x] * 4
    for v in basis:
        x = x - (v @ x) * v
    t_dot = (time.perf_counter() - t0) / 4
    cores = (time.process_time() - c0) / max(1e-9, time.perf_counter() - w0)
    est = outer_its * (2 * w.nt * t_inner + 2 * t_mv) + t_dot * outer_its * (outer_its + 1) / 2
    return {"value": est, "unit": "s", "cores": round(cores, 2), "kind": "oracle",
            "sample": (f"FP64 oracle (NumPy/SciPy) on the host: 1 full matvec ({t_mv:.2f} s) and {n_inner} inner "
                       f"Theta_tilde solves ({t_inner:.3f} s each) at {'x'.join(map(str, w.n))} s={w.s}; time to "
                       f"solution estimated for "
                       f"{outer_its} outer iterations as its*(2*nt*t_inner+2*t_matvec)+orthogonalisation")}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.small)
    # the FP32-preconditioned solve of this workload takes 8 outer iterations on the GPU;
    # each step is a bounded sample (about 8 s) of the oracle on that count
    steps = []
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(w, outer_its=8, budget_s=8.0)
        steps.append(cb["value"])
    v = float(np.median(steps))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precond": "fp32-equivalent settings, FP64 arithmetic",
                       "outer": "FGMRES(20) tol 1e-8"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precond_case(args):
    """P_tilde^{-1} r on a 256x256, s = 3, 16-step problem: the same kernels as the benchmark's
    Schur sweep and batched Theta_tilde phase, small enough for a full profiler capture."""
    import torch
    import synth
    from paper_2609_16863_gb300 import Solver, radau_iia
    w = synth.workload_fp32_precond_2d(N=256, nt=16, s=3)
    S = Solver(w.n, w.T, w.nt, tableau=radau_iia(3), prec_P=args.prec, inner_maxit=3, inner_tol=1e-3)
    g = torch.Generator(device="cuda:0").manual_seed(5)
    r = torch.randn(S.n_st, dtype=torch.float64, device="cuda:0", generator=g)
    z = torch.zeros_like(r)
    for _ in range(args.warmup):
        S.precond_apply(r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        S.precond_apply(r, z)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "precond_apply fd2d_n256_radau3_nt16", "prec": args.prec,
                      "ms_per_apply": e0.elapsed_time(e1) / max(args.steps, 1)}))
    S.close()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batched64":
        batched_arm(args)
        return
    if args.precond_case:
        precond_case(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2609_16863_gb300 import Solver, _lib, radau_iia

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    lib = _lib.lib()

    def barrier():
        if world > 1:
            dist.barrier()

    w = workload(args.small, args.workload)
    from paper_2609_16863_gb300.tableau import make as make_tableau
    common = dict(tableau=make_tableau(w.method, w.s), tol=w.tol, restart=20, maxit=100, stream=stream.cuda_stream)
    S = Solver(w.n, w.T, w.nt, prec_P=args.prec, inner_maxit=3, inner_tol=1e-3, **common)
    f = torch.from_numpy(w.f).to(dev)
    u0 = torch.from_numpy(w.u0).to(dev)
    x = torch.zeros(S.n_st, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    info = None
    for _ in range(args.warmup):
        _, info = S.solve(f, u0, x)
    clocks = Clocks(local)
    n0 = lib.aao_rk_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        _, info = S.solve(f, u0, x)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    launches = lib.aao_rk_launch_count() - n0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    x_mixed = x.clone()

    # FP64 preconditioner on the same problem (mixed vs FP64 comparison)
    fp64 = None
    if not args.no_fp64:
        S64 = Solver(w.n, w.T, w.nt, prec_P="fp64", inner_maxit=5, inner_tol=1e-6, **common)
        x64 = torch.zeros_like(x)
        S64.solve(f, u0, x64)            # warm-up
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        _, i64 = S64.solve(f, u0, x64)
        a1.record(stream)
        torch.cuda.synchronize()
        t64 = a0.elapsed_time(a1) / 1e3
        diff = float(torch.linalg.norm(x_mixed - x64) / torch.linalg.norm(x64))
        fp64 = {"time_s": t64, "outer_its": i64.outer_its, "inner_its": i64.inner_its_total,
                "rel_res": i64.rel_res, "t_theta_ms": i64.t_theta_ms, "t_schur_ms": i64.t_schur_ms,
                "speedup_mixed_vs_fp64": t64 / (ms / 1e3),
                "rel_diff_mixed_vs_fp64_solution": diff}
        S64.close()
        del x64

    # end to end through the C ABI with pinned host buffers
    fh = torch.from_numpy(w.f).pin_memory()
    uh = torch.from_numpy(w.u0).pin_memory()
    xh = torch.zeros(S.n_st, dtype=torch.float64).pin_memory()
    S.solve(fh, uh, xh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.solve(fh, uh, xh)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps

    # live roofline: CUDA events around every kernel launch of one extra solve (eager
    # launches), per-kernel algorithmic bytes from the launch sites; the dominant
    # kernel is the one with the largest summed event time
    import ctypes as C
    peak, peak_kind = peaks()

    def profiled(fn):
        _lib.check(lib.aao_rk_profile_begin(b"k_"))
        fn()
        nl, pms, pby = C.c_longlong(), C.c_double(), C.c_double()
        _lib.check(lib.aao_rk_profile_end(C.byref(nl), C.byref(pms), C.byref(pby)))
        rows = []
        for ln in lib.aao_rk_profile_report().decode().splitlines():
            name, n, kms, kby = ln.split("\t")
            short = name
            for tok in ("k_vcycle_tail", "k_smooth2", "k_smooth", "k_resid_restrict", "k_residual", "k_restrict",
                        "k_prolong_smooth", "k_prolong_add", "k_coarse_solve", "k_rana_rhs", "k_theta", "k_mgs",
                        "k_norm", "k_scale_store", "k_combine", "k_matvec", "k_givens", "k_hess_solve",
                        "k_schur_update", "k_schur_rhs", "k_schur_g", "k_inner_init", "k_count_its", "k_step_add",
                        "k_step_set", "k_pack_small", "k_outer_init", "k_rhs", "k_load"):
                if tok in name:
                    short = tok + ("<" + name.split("I", 1)[1][:1] + ">" if "I" in name else "")
                    break
            rows.append({"kernel": short, "launches": int(n), "ms": float(kms), "bytes": float(kby)})
        rows.sort(key=lambda r: -r["ms"])
        return rows, pms.value

    def roof_of(r, total_ms):
        ach = r["bytes"] / (r["ms"] * 1e-3) / 1e9 if r["ms"] > 0 else 0.0
        return {"bound": "hbm", "kernel": r["kernel"], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "peak_kind": peak_kind + " (copy bandwidth)",
                "launches_per_solve": r["launches"], "kernel_ms": r["ms"],
                "algorithmic_bytes_per_launch": r["bytes"] / max(1, r["launches"]),
                "share_of_profiled_time": r["ms"] / total_ms if total_ms > 0 else None}

    rows, tot = profiled(lambda: S.solve(f, u0, x))
    roof = roof_of(rows[0], tot)
    roof["measured"] = "CUDA events around each launch during one extra (eager) solve"
    if "k_cluster_mg" in roof["kernel"] and args.prec == "fp32" and args.workload == WORKLOAD and not args.small:
        roof["traffic"] = CLUSTER_MG_DRAM_BYTES
        roof["limit"] = "latency: 25 cluster barriers and dependent step chains per V-cycle on 16 SMs"
    top = [{"kernel": r["kernel"], "launches": r["launches"], "ms": round(r["ms"], 3),
            "GB/s": round(r["bytes"] / (r["ms"] * 1e-3) / 1e9, 1) if r["ms"] > 0 else 0.0} for r in rows[:8]]
    # the batched Theta_tilde phase alone (all nt time blocks at once): HBM-bound kernels
    item = w.s * S.nx
    Rb = torch.randn(w.nt * item, dtype=torch.float64, device=dev)
    Zb = torch.zeros_like(Rb)
    S.inner_solve(w.nt, Rb, Zb)
    rows_t, tot_t = profiled(lambda: S.inner_solve(w.nt, Rb, Zb))
    roof_theta = roof_of(rows_t[0], tot_t)
    roof_theta["measured"] = "CUDA events around each launch of one batched inner solve over all nt blocks"
    del Rb, Zb

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == WORKLOAD:
        cpu = cpu_baseline(w, info.outer_its)

    if rank == 0:
        value = ms / 1e3
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": f"f64/{args.prec}", "data": "synthetic",
                "config": {"workload": args.workload, "grid": list(w.n),
                           "nt": w.nt, "s": w.s, "n_st": S.n_st,
                           "precond": f"P_tilde {args.prec}, inner GMRES 3/1e-3, 3 V(2,2)-cycles",
                           "outer": "FP64 FGMRES(20), tol 1e-8",
                           "l2": "working set larger than L2 (no flush)", "parallelism": "replicas",
                           "small_check_only": bool(args.small)},
                "outer_its": info.outer_its, "inner_its": info.inner_its_total, "rel_res": info.rel_res,
                "t_theta_ms": info.t_theta_ms, "t_schur_ms": info.t_schur_ms,
                "fp64_precond": fp64,
                "dofs_its_per_s": world * S.n_st * info.outer_its / (ms / 1e3),   # all replicas
                "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * (2 * S.nx),
                        "d2h_bytes_per_step": 8 * S.n_st},
                "gpu_launches": launches // max(1, args.steps) * args.steps,
                "roofline": roof, "roofline_theta_phase": roof_theta, "kernels_top": top,
                "cpu_baseline": cpu, "clocks": ck}
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
