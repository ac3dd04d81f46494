#!/usr/bin/env python
"""Benchmark: time to a 1e-8 relative residual of the all-at-once RK heat solve.

Workload (one step = one full solve, FP64 FGMRES(20) outer + P_tilde):
  2D 256x256 interior FD grid (M = I), Radau IIA s = 3, 128 steps to T = 1,
  u0 and f seeded Gaussian random fields (squared-exponential, l = 0.1,
  unit variance), f constant in time; n_st = 33,619,968 space-time unknowns.
  The timed solve applies P_tilde in FP32 (Theta_tilde GMRES 3 / 1e-3, 3
  V-cycles) with S_tilde's recurrence by one two-level MGRIT iteration
  (coarsening factor --mgrit-m; 0 = forward substitution).  The same problem is
  also solved with the forward substitution, and with P_tilde in FP64 at the
  paper's FP64 inner settings (GMRES 5 / 1e-6) and at the FP32 arm's settings
  (3 / 1e-3, as the paper's matched-settings run).

Timing: W warm-up solves, then K solves between CUDA events on the solver's
stream with a barrier and a synchronize on both sides; the working set
(x 269 MB, Krylov basis ~11 GB) is far larger than L2.  `e2e` repeats the
solve through the C ABI with pinned host buffers (copies inside the timed
region).  `roofline` times every launch of the dominant kernel with CUDA
events during one extra solve and divides its algorithmic bytes by that time;
its DRAM traffic comes from the committed ncu summary of that kernel.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# MGRIT's dataflow schedule (shifted solves without a cluster plan, e.g. the FP64 arm) runs up to 16
# worker streams plus the solver's own: give each its hardware queue (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "time-to-1e-8 residual, mixed vs FP64 precond, same GB300; precond HBM GB/s"
WORKLOAD = "fd2d_n256_radau3_nt128"
PROFILES = os.path.join(ROOT, "profiles")


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
                   choices=["fd2d_n256_radau3_nt128", "fd3d_n96_radau3_nt32", "fd3d_n96_gauss2_nt32", "batched64",
                            "adjoint_fd2d_n128_kappa_nt64"],
                   help="extra configurations (the default is the benchmark line)")
    p.add_argument("--precond-case", action="store_true",
                   help="small case for profiler captures: --steps applications of P_tilde (FP32) on the "
                        "256x256 Radau IIA s=3 grid with 16 time steps (MGRIT with --mgrit-m); prints ms per "
                        "application")
    p.add_argument("--theta-case", action="store_true",
                   help="profiler case: --steps batched Theta_tilde solves over all 128 time blocks of the "
                        "benchmark grid (256x256, s=3, P_tilde FP32; vectors of 100 MB, larger than L2)")
    p.add_argument("--batch-case", action="store_true",
                   help="profiler case: batched Theta_tilde solves of 1..32 time blocks of the benchmark grid "
                        "(256x256, s=3, P_tilde --prec): ms per solve and event-timed k_cluster_mg launches per "
                        "batch size (one thread-block cluster per item)")
    p.add_argument("--matvec-case", action="store_true",
                   help="profiler case: --steps FP64 all-at-once matvecs at the benchmark size (269 MB vectors)")
    p.add_argument("--mgrit-m", type=int, default=-1,
                   help="MGRIT coarsening factor for S_tilde's recurrence (0: forward substitution; -1: the "
                        "autotuner times one P_tilde application per candidate and takes the fastest)")
    p.add_argument("--cpu-sample", default=None, choices=["c1", "reduced", "c2"],
                   help=argparse.SUPPRESS)   # one oracle timing, run in a child with a fixed thread count
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
        m_req = 8 if args.mgrit_m < 0 else args.mgrit_m
        m = m_req if 1 < m_req and w.nt // m_req >= 2 else 0
        solvers.append(Solver(w.n, w.T, w.nt, tableau=radau_iia(w.s), prec_P=args.prec, inner_maxit=3,
                              inner_tol=1e-3, tol=w.tol, stream=st.cuda_stream, mgrit_m=m))
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
            "data": "synthetic", "config": {"workload": "batched64", "problems": len(ws), "n_st_total": nst,
                                            "schur": f"MGRIT m = {8 if args.mgrit_m < 0 else args.mgrit_m} "
                                                     f"where nt has two or more intervals",
                                            "execution": "one host thread and stream per problem"},
            "dofs_its_per_s": sum(S.n_st * i for S, i in zip(solvers, its)) / t,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "outer_its_min_max": [min(its), max(its)], "all_converged": all(i.converged for i in infos)}
    print(json.dumps(line), flush=True)


def adjoint_arm(args):
    """Gradient of J = 1/2 ||u(T) - u_target||^2 + 1/2 1e-4 ||f||^2 with respect to f and the nodal
    kappa on the 128x128, Radau IIA s=3, 64-step variable-diffusivity workload through the
    torch.autograd.Function: forward solve keeping states every 8 steps, adjoint solve with
    P_tilde^T, window-by-window recomputation for the kappa gradient.  One step = forward +
    backward."""
    import torch
    import synth
    from paper_2609_16863_gb300 import radau_iia
    from paper_2609_16863_gb300.autograd import heat_solve
    dev = torch.device("cuda", 0)
    w = synth.workload_adjoint_2d()
    m_req = 8 if args.mgrit_m < 0 else args.mgrit_m
    mg_m = m_req if 1 < m_req <= w.nt else 0
    cfg = dict(n=w.n, T=w.T, nt=w.nt, tableau=radau_iia(w.s), prec_P=args.prec, tol=1e-9, maxit=200, ckpt_every=8,
               inner_maxit=3, inner_tol=1e-3, mgrit_m=mg_m)
    lo = w.nt * w.nx
    f0 = torch.from_numpy(w.f).to(dev)
    u0 = torch.from_numpy(w.u0).to(dev)
    k0 = torch.from_numpy(w.kappa).to(dev)
    tg = torch.from_numpy(w.target).to(dev)

    def step():
        fd = f0.clone().requires_grad_(True)
        kd = k0.clone().requires_grad_(True)
        x = heat_solve(fd, u0, kd, **cfg)
        J = 0.5 * ((x[lo: lo + w.nx] - tg) ** 2).sum() + 0.5e-4 * (fd ** 2).sum()
        J.backward()
        return fd.grad, kd.grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        gf, gk = step()
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / args.steps
    line = {"metric": "gradient (forward + adjoint with checkpoints every 8 steps) wall time", "value": t, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": f"f64/{args.prec}",
            "data": "synthetic",
            "config": {"workload": "adjoint_fd2d_n128_kappa_nt64", "n_st": w.nx * (w.nt + 1 + w.s * w.nt),
                       "schur": f"MGRIT m = {mg_m}" if mg_m else "forward substitution",
                       "checkpoints": "every 8 steps", "tol": 1e-9},
            "grad_norms": {"f": float(torch.linalg.norm(gf)), "kappa": float(torch.linalg.norm(gk))}}
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


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS")


class OracleSampler:
    """The FP64 oracle (as it stands: NumPy/SciPy, FGMRES + P_tilde with the forward substitution)
    on the benchmark workload, timed on bounded samples.  The time to solution is estimated as
    outer_its * (2 nt t_inner + 2 t_matvec) + orthogonalisation: P_tilde applies 2 nt inner
    Theta_tilde solves (nt batched, nt in the substitution) and every iteration one matvec plus
    the residual's."""

    def __init__(self, w):
        from oracle.precond import Preconditioner
        from oracle.solve import build
        self.w = w
        self.op = build(w.n, w.T, w.nt, w.method, w.s)
        self.P = Preconditioner(self.op, w.n, inner_maxit=3, inner_tol=1e-3, mg_cycles=3, nu1=2, nu2=2,
                                omega=0.8)
        x = np.random.default_rng(0).standard_normal(self.op.n_st)
        t0 = time.perf_counter()
        self.op.matvec(x)
        self.t_mv = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(4):
            x = x - (x @ x) / (x @ x) * 0.5 * x
        self.t_dot = (time.perf_counter() - t0) / 4
        self.r = x[self.op.n_v: self.op.n_v + w.s * self.op.nx].copy()

    def sample(self, budget_s, outer_its):
        n_inner = 0
        t0 = time.perf_counter()
        while True:
            self.P.inner_solve(self.r)
            n_inner += 1
            if time.perf_counter() - t0 > budget_s or n_inner >= 400:
                break
        wall = time.perf_counter() - t0
        t_inner = wall / n_inner
        est = outer_its * (2 * self.w.nt * t_inner + 2 * self.t_mv) + self.t_dot * outer_its * (outer_its + 1) / 2
        return est, wall, n_inner, t_inner


def oracle_sample(kind: str, outer_its: int):
    """One oracle timing in this process (thread count fixed by the parent through the environment).
    c1: a full solve of the 32x32, Radau IIA s=2, 16-step workload (tol 1e-10, inner 5 / 1e-6);
    reduced: a full solve of the 64x64, Radau IIA s=3, 32-step field workload (tol 1e-8, inner 3 / 1e-3);
    c2: the 256x256, s=3, 128-step workload, estimated from about 8 s of inner solves."""
    import synth
    from oracle.solve import OracleOptions, build, solve
    if kind == "c2":
        t0 = time.perf_counter()
        smp = OracleSampler(synth.workload_fp32_precond_2d())
        est, wall, n, t_inner = smp.sample(8.0, outer_its)
        return {"kind": kind, "estimate_s": est, "sample_wall_s": time.perf_counter() - t0, "inner_solves": n,
                "t_inner_s": t_inner, "t_matvec_s": smp.t_mv}
    if kind == "c1":
        w = synth.workload_small_2d()
        opts = OracleOptions(tol=1e-10, inner_maxit=5, inner_tol=1e-6)
    else:
        w = synth.workload_fp32_precond_2d(N=64, nt=32, s=3)
        opts = OracleOptions(tol=1e-8, inner_maxit=3, inner_tol=1e-3)
    t0 = time.perf_counter()
    op = build(w.n, w.T, w.nt, w.method, w.s)
    r = solve(op, w.n, op.rhs(w.u0, w.f), opts)
    return {"kind": kind, "seconds": time.perf_counter() - t0, "outer_its": r.outer_its, "n_st": op.n_st,
            "rel_res": r.rel_res}


def run_oracle_sample(kind: str, threads: int, outer_its: int):
    env = os.environ.copy()
    for v in THREAD_VARS:
        env[v] = str(threads)
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", kind, "--steps", str(outer_its)],
                       env=env, capture_output=True, text=True, timeout=900)
    if p.returncode != 0:
        raise RuntimeError(f"oracle sample {kind} failed: {p.stderr[-500:]}")
    return json.loads(p.stdout.strip().splitlines()[-1])


def cpu_baseline(outer_its: int):
    """The oracle on the host cores, 1 thread and every core this process may use: full solves of
    the 32x32 workload and of a 64x64 field workload (measured), and the benchmark workload
    estimated from a bounded sample (about 10 s of CPU work per thread count)."""
    cores = len(os.sched_getaffinity(0))
    out = {}
    for kind in ("c1", "reduced", "c2"):
        out[kind] = {"threads_1": run_oracle_sample(kind, 1, outer_its),
                     f"threads_{cores}": run_oracle_sample(kind, cores, outer_its)}
    best = min(out["c2"]["threads_1"]["estimate_s"], out["c2"][f"threads_{cores}"]["estimate_s"])
    return {"value": best, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": (f"FP64 oracle (NumPy/SciPy, forward substitution) on the host, {cores} cores available: "
                       f"value = time to solution of the 256x256 s=3 128-step workload estimated from ~8 s of "
                       f"inner Theta_tilde solves and one matvec as its*(2*nt*t_inner+2*t_matvec)+orthogonalisation "
                       f"for {outer_its} outer iterations (faster of 1 thread / all threads); measured full solves of "
                       f"the 32x32 (c1) and 64x64 (reduced) workloads beside it"),
            "estimated": True, "detail": out}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    w = workload(args.small)
    # the FP32-preconditioned solve of this workload takes 8 outer iterations on the GPU (and in
    # the oracle); every step is a bounded sample of the oracle on that count: ms_per_step is the
    # sample's own wall time, value the time to solution estimated from it
    t_setup = time.perf_counter()
    smp = OracleSampler(w)
    t_setup = time.perf_counter() - t_setup
    for _ in range(args.warmup):
        smp.sample(0.5, 8)
    ests, walls = [], []
    for _ in range(max(1, args.steps)):
        est, wall, n, t_inner = smp.sample(2.0, 8)
        ests.append(est)
        walls.append(wall)
    v = float(np.median(ests))
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(walls)) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precond": "fp32-equivalent settings, FP64 arithmetic",
                       "outer": "FGMRES(20) tol 1e-8", "value_is_estimate": True,
                       "ms_per_step_is": "wall time of each step's bounded sample (about 2 s of inner solves)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": (f"FP64 oracle (NumPy/SciPy) on the host: per step about 2 s of inner "
                                        f"Theta_tilde solves ({t_inner:.3f} s each) at {'x'.join(map(str, w.n))} "
                                        f"s={w.s} plus one "
                                        f"matvec ({smp.t_mv:.2f} s, timed once); time to solution estimated for "
                                        f"8 outer iterations as its*(2*nt*t_inner+2*t_matvec)+orthogonalisation; "
                                        f"oracle set-up {t_setup:.1f} s")},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precond_case(args):
    """P_tilde^{-1} r on a 256x256, s = 3, 16-step problem: the same kernels as the benchmark's
    Schur sweep and batched Theta_tilde phase, small enough for a full profiler capture."""
    import torch
    import synth
    from paper_2609_16863_gb300 import Solver, radau_iia
    w = synth.workload_fp32_precond_2d(N=256, nt=16, s=3)
    m_req = 8 if args.mgrit_m < 0 else args.mgrit_m
    m = m_req if 1 < m_req <= w.nt else 0
    S = Solver(w.n, w.T, w.nt, tableau=radau_iia(3), prec_P=args.prec, inner_maxit=3, inner_tol=1e-3, mgrit_m=m)
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
    print(json.dumps({"case": "precond_apply fd2d_n256_radau3_nt16", "prec": args.prec, "mgrit_m": m,
                      "ms_per_apply": e0.elapsed_time(e1) / max(args.steps, 1)}))
    S.close()


def theta_case(args):
    """Theta_tilde^{-1} over all nt time blocks of the benchmark workload: the HBM-bound batched phase
    (smoother, residual, restriction, prolongation, V-cycle tail, Rana, Theta_hat, MGS) alone."""
    import torch
    from paper_2609_16863_gb300 import Solver, radau_iia
    w = workload(False)
    S = Solver(w.n, w.T, w.nt, tableau=radau_iia(w.s), prec_P=args.prec, inner_maxit=3, inner_tol=1e-3,
               restart=1)
    n = w.nt * w.s * S.nx
    g = torch.Generator(device="cuda:0").manual_seed(6)
    r = torch.randn(n, dtype=torch.float64, device="cuda:0", generator=g)
    z = torch.zeros_like(r)
    for _ in range(args.warmup):
        S.inner_solve(w.nt, r, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        S.inner_solve(w.nt, r, z)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "theta_phase fd2d_n256_radau3_nt128", "prec": args.prec,
                      "ms_per_solve": e0.elapsed_time(e1) / max(args.steps, 1)}))
    S.close()


def batch_case(args):
    """Batched Theta_tilde solves of B = 1..32 time blocks on the benchmark grid: up to 32 items run one
    thread-block cluster per item (16 CTAs for fewer than 8 items, 8 CTAs from 8 on), so the launch
    time of k_cluster_mg against B shows how many clusters are resident at once."""
    import ctypes as C
    import torch
    from paper_2609_16863_gb300 import Solver, radau_iia, _lib
    w = workload(False)
    S = Solver(w.n, w.T, 32, tableau=radau_iia(w.s), prec_P=args.prec, inner_maxit=3, inner_tol=1e-3, restart=1)
    lib = S._lib
    g = torch.Generator(device="cuda:0").manual_seed(6)
    rows = {}
    for B in (1, 2, 4, 7, 8, 12, 14, 16, 24, 32):
        n = B * w.s * S.nx
        r = torch.randn(n, dtype=torch.float64, device="cuda:0", generator=g)
        z = torch.zeros_like(r)
        for _ in range(max(args.warmup, 1)):
            S.inner_solve(B, r, z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(args.steps, 1)):
            S.inner_solve(B, r, z)
        e1.record()
        torch.cuda.synchronize()
        _lib.check(lib.aao_rk_profile_begin(b"k_cluster_mg"))
        S.inner_solve(B, r, z)
        nl, pms, pby = C.c_longlong(), C.c_double(), C.c_double()
        _lib.check(lib.aao_rk_profile_end(C.byref(nl), C.byref(pms), C.byref(pby)))
        rows[B] = {"ms_per_solve": round(e0.elapsed_time(e1) / max(args.steps, 1), 3),
                   "cluster_launches": nl.value, "us_per_cluster_launch": round(1e3 * pms.value / max(1, nl.value), 1)}
    print(json.dumps({"case": "batched theta fd2d_n256_radau3", "prec": args.prec, "batches": rows}))
    S.close()


def matvec_case(args):
    """The FP64 all-at-once matvec y = A x at the benchmark size."""
    import torch
    from paper_2609_16863_gb300 import Solver, radau_iia
    w = workload(False)
    S = Solver(w.n, w.T, w.nt, tableau=radau_iia(w.s), prec_P="fp32", restart=1)
    g = torch.Generator(device="cuda:0").manual_seed(7)
    x = torch.randn(S.n_st, dtype=torch.float64, device="cuda:0", generator=g)
    y = torch.zeros_like(x)
    for _ in range(args.warmup):
        S.matvec(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        S.matvec(x, y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"case": "matvec fd2d_n256_radau3_nt128", "ms_per_matvec": ms,
                      "algorithmic_GBps": 16.0 * S.n_st / (ms * 1e-3) / 1e9}))
    S.close()


def profile_traffic(kernel: str, key: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel` from the
    committed ncu summary profiles/<kernel>.md (a line 'traffic <key>: <bytes>'), else None."""
    path = os.path.join(PROFILES, f"{kernel}.md")
    try:
        for ln in open(path):
            if ln.startswith(f"traffic {key}:"):
                return float(ln.split(":", 1)[1].split()[0])
    except OSError:
        pass
    return None


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(oracle_sample(args.cpu_sample, args.steps)), flush=True)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batched64":
        batched_arm(args)
        return
    if args.workload == "adjoint_fd2d_n128_kappa_nt64":
        adjoint_arm(args)
        return
    if args.precond_case:
        precond_case(args)
        return
    if args.theta_case:
        theta_case(args)
        return
    if args.matvec_case:
        matvec_case(args)
        return
    if args.batch_case:
        batch_case(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2609_16863_gb300 import Solver, _lib

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
    tuned = None
    if args.mgrit_m < 0:
        from paper_2609_16863_gb300.tune import tune_mgrit
        mg_m, tuned = tune_mgrit(w.n, w.T, w.nt, tableau=make_tableau(w.method, w.s), prec_P=args.prec,
                                 inner_maxit=3, inner_tol=1e-3, restart=1)
        tuned = {str(k): round(v, 3) for k, v in tuned.items()}
    else:
        mg_m = args.mgrit_m if 1 < args.mgrit_m <= w.nt else 0
    S = Solver(w.n, w.T, w.nt, prec_P=args.prec, inner_maxit=3, inner_tol=1e-3, mgrit_m=mg_m, **common)
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

    def one_solve(prec, inner_maxit, inner_tol, m):
        """One warm-up and one timed solve of the same problem with another configuration."""
        T = Solver(w.n, w.T, w.nt, prec_P=prec, inner_maxit=inner_maxit, inner_tol=inner_tol, mgrit_m=m, **common)
        xx = torch.zeros_like(x)
        T.solve(f, u0, xx)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        _, ii = T.solve(f, u0, xx)
        a1.record(stream)
        torch.cuda.synchronize()
        t = a0.elapsed_time(a1) / 1e3
        d = float(torch.linalg.norm(x_mixed - xx) / torch.linalg.norm(xx))
        T.close()
        del xx
        return {"time_s": t, "outer_its": ii.outer_its, "inner_its": ii.inner_its_total, "rel_res": ii.rel_res,
                "t_theta_ms": ii.t_theta_ms, "t_schur_ms": ii.t_schur_ms, "mgrit_m": m,
                "inner": [inner_maxit, inner_tol], "rel_diff_timed_solution_vs_this": d}

    # the same problem with the forward substitution in S_tilde, and with an FP64 P_tilde at the
    # paper's FP64 inner settings and at the timed arm's settings (the paper's matched-settings run)
    fp64 = seq = None
    if not args.no_fp64:
        seq = one_solve(args.prec, 3, 1e-3, 0) if mg_m else None
        fp64 = {"paper_fp64_inner_5_1e-6": one_solve("fp64", 5, 1e-6, mg_m),
                "matched_inner_3_1e-3": one_solve("fp64", 3, 1e-3, mg_m)}
        for v in fp64.values():
            v["speedup_timed_vs_this"] = v["time_s"] / (ms / 1e3)

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
            for tok in ("k_strip2dIfLi0", "k_strip2dIfLi1", "k_strip2dIfLi2", "k_strip2dIdLi0", "k_strip2dIdLi1",
                        "k_strip2dIdLi2", "k_cluster_mg", "k_vcycle_tail", "k_smooth2", "k_smooth_rows", "k_smooth", "k_resid_restrict",
                        "k_residual_rows", "k_residual", "k_restrict", "k_prolong_smooth", "k_prolong_add_rows",
                        "k_prolong_add", "k_coarse_solve", "k_rana_rhs", "k_theta", "k_mgs", "k_norm", "k_scale_store",
                        "k_combine", "k_matvec", "k_givens", "k_hess_solve", "k_schur_update_b", "k_schur_update",
                        "k_schur_rhs_b", "k_schur_rhs", "k_schurT", "k_schur_g", "k_mgrit_cpoints", "k_inner_init",
                        "k_count_its", "k_step_add", "k_step_set", "k_outer_init", "k_rhs", "k_load"):
                if tok in name:
                    short = tok
                    break
            ms = re.search(r"k_strip2d_stI([fd])Li(\d)E", name)
            if ms:
                short = (f"k_strip2d_st<{'float' if ms.group(1) == 'f' else 'double'}, "
                         f"{ {'0': 'smooth', '1': 'smooth_zero', '2': 'residual'}[ms.group(2)] }>")
            mv = re.search(r"k_vec16I(\w+?)Li(\d)E", name)
            if mv:
                short = (f"k_vec16<{'bf16' if 'bfloat' in mv.group(1) else 'fp16'}, "
                         f"{ {'0': 'smooth', '1': 'smooth_zero', '2': 'residual'}[mv.group(2)] }>")
            if short.startswith("k_strip2dI") and not ms:
                mode = {"0": "smooth", "1": "smooth_zero", "2": "residual"}[short[-1]]
                short = f"k_strip2d<{'float' if short[10] == 'f' else 'double'}, {mode}>"
            rows.append({"kernel": short, "mangled": name, "launches": int(n), "ms": float(kms), "bytes": float(kby)})
        rows.sort(key=lambda r: -r["ms"])
        return rows, pms.value

    # method-level streaming bytes of one V-cycle of the shifted solve (every vector pass counted
    # once, no cross-step fusion): C_V n_x b_p, C_V = (3 (nu1 + nu2) + 4 + 2^(1-d)) / (1 - 2^-d)
    # = 22 in 2D with nu = 2, plus the first coarse level's 9-point stencil (9 n_x / 4 b_p)
    b_p = {"fp32": 4, "bf16": 2, "fp16": 2}[args.prec]
    cv_bytes = (22.0 + 9.0 / 4.0) * S.nx * b_p

    def roof_of(r, total_ms):
        ach = r["bytes"] / (r["ms"] * 1e-3) / 1e9 if r["ms"] > 0 else 0.0
        per = r["bytes"] / max(1, r["launches"])
        return {"bound": "hbm", "kernel": r["kernel"], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "peak_kind": f"{peak_kind} copy bandwidth, of {peak_kind}",
                "launches_per_solve": r["launches"], "kernel_ms": r["ms"],
                "algorithmic_bytes_per_launch": per,
                "share_of_profiled_time": r["ms"] / total_ms if total_ms > 0 else None}

    rows, tot = profiled(lambda: S.solve(f, u0, x))
    roof = roof_of(rows[0], tot)
    roof["measured"] = "CUDA events around each launch during one extra (eager) solve"
    if roof["kernel"] == "k_cluster_mg":
        # a launch solves `items` shifted systems (3 V-cycles each); its compulsory bytes are b in
        # and x out (2 n_x b_p per item); the method-level model counts every V-cycle pass
        items = roof["algorithmic_bytes_per_launch"] / (2.0 * S.nx * b_p)
        model = 3.0 * cv_bytes * items
        ach_model = model * roof["launches_per_solve"] / (roof["kernel_ms"] * 1e-3) / 1e9
        roof.update({"compulsory": {"achieved": roof["achieved"], "frac": roof["frac"],
                                    "bytes_per_launch": roof["algorithmic_bytes_per_launch"]},
                     "achieved": ach_model, "frac": ach_model / peak, "algorithmic_bytes_per_launch": model,
                     "bytes_model": "method-level: 3 V-cycles x (22 + 9/4) n_x b_p per item",
                     "items_per_launch": items,
                     "limit": "latency: cluster barriers and dependent step chains per V-cycle (16 SMs per item)"})
        roof["traffic"] = profile_traffic("k_cluster_mg_fd2d_n256", f"{args.prec} per item")
        if roof["traffic"] is not None:
            roof["traffic"] *= items
    top = [{"kernel": r["kernel"], "launches": r["launches"], "ms": round(r["ms"], 3),
            "GB/s": round(r["bytes"] / (r["ms"] * 1e-3) / 1e9, 1) if r["ms"] > 0 else 0.0} for r in rows[:10]]
    # the batched Theta_tilde phase alone (all nt time blocks at once): the HBM-bound kernels
    item = w.s * S.nx
    Rb = torch.randn(w.nt * item, dtype=torch.float64, device=dev)
    Zb = torch.zeros_like(Rb)
    S.inner_solve(w.nt, Rb, Zb)
    rows_t, tot_t = profiled(lambda: S.inner_solve(w.nt, Rb, Zb))
    roof_theta = roof_of(rows_t[0], tot_t)
    roof_theta["measured"] = "CUDA events around each launch of one batched inner solve over all nt blocks"
    roof_theta["traffic"] = profile_traffic("theta_phase_fd2d_n256_nt128", f"{args.prec} {rows_t[0]['kernel']}")
    # the dominant kernel of the phase that streams through HBM (the on-chip V-cycle tail excluded)
    stream_rows = [r for r in rows_t if "vcycle_tail" not in r["mangled"] and "cluster" not in r["mangled"]]
    roof_stream = roof_of(stream_rows[0], tot_t) if stream_rows else None
    if roof_stream:
        roof_stream["measured"] = roof_theta["measured"]
        roof_stream["traffic"] = profile_traffic("theta_phase_fd2d_n256_nt128",
                                                 f"{args.prec} {stream_rows[0]['kernel']}")
    top_theta = [{"kernel": r["kernel"], "launches": r["launches"], "ms": round(r["ms"], 3),
                  "algorithmic_GB/s": round(r["bytes"] / (r["ms"] * 1e-3) / 1e9, 1) if r["ms"] > 0 else 0.0,
                  "frac": round(r["bytes"] / (r["ms"] * 1e-3) / 1e9 / peak, 3) if r["ms"] > 0 else 0.0}
                 for r in rows_t[:10]]
    del Rb, Zb

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.workload == WORKLOAD:
        cpu = cpu_baseline(info.outer_its)

    if rank == 0:
        value = ms / 1e3
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": f"f64/{args.prec}", "data": "synthetic",
                "config": {"workload": args.workload, "grid": list(w.n),
                           "nt": w.nt, "s": w.s, "n_st": S.n_st,
                           "precond": f"P_tilde {args.prec}, inner GMRES 3/1e-3, 3 V(2,2)-cycles",
                           "schur": (f"two-level MGRIT, m = {mg_m}, F-relaxation, one iteration" if mg_m
                                     else "forward substitution"),
                           "schur_autotune_ms_per_precond_apply": tuned,
                           "outer": "FP64 FGMRES(20), tol 1e-8",
                           "l2": "working set larger than L2 (no flush)", "parallelism": "replicas",
                           "small_check_only": bool(args.small)},
                "outer_its": info.outer_its, "inner_its": info.inner_its_total, "rel_res": info.rel_res,
                "t_theta_ms": info.t_theta_ms, "t_schur_ms": info.t_schur_ms,
                "substitution_precond": seq, "fp64_precond": fp64,
                "dofs_its_per_s": world * S.n_st * info.outer_its / (ms / 1e3),   # all replicas
                "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * (2 * S.nx),
                        "d2h_bytes_per_step": 8 * S.n_st},
                "gpu_launches": launches // max(1, args.steps) * args.steps,
                "roofline": roof, "roofline_theta_phase": roof_theta, "roofline_theta_streaming": roof_stream,
                "kernels_top": top,
                "kernels_theta_phase": top_theta, "cpu_baseline": cpu, "clocks": ck}
        print(json.dumps(line), flush=True)
    S.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
