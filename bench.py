#!/usr/bin/env python
"""Benchmark of the PCG-ATKM hot path on the 256x256x64 workload.

Workload: box [-16,16]^2 x [-1.5,1.5], grid 256x256x64, gamma = (1, 1.2, 30),
beta = 1000, lambda = 400, n = (sin 30deg, 0, cos 30deg), Omega = 0.9,
initial guess (d).  One step = one PCG iteration of Algorithm 1 on this
workload: H phi with the energy sums, residual, preconditioner, PR+ direction,
H p, the curvature ATKM, retraction and the trial-energy ATKM (plus one per
halving) -- every hot-path row, entirely on the device.  W warm-up iterations
start the solve from psi_0; the K timed iterations resume it (the same
solve), bracketed by barrier + synchronize and timed with CUDA events.

value = ATKM evaluations per second sustained by the full PCG step (the ATKM
calls the K iterations made / their time); the line also carries the time per
iteration, the stand-alone ATKM rate (FP64 and FP32), the roofline of the
dominant kernel (timed live with CUDA events inside the timed iterations),
an end-to-end number through the public API with host buffers, and the CPU
oracle on a bounded sample (one oracle PCG iteration of the same workload).
Time to 1e-8 is not a bench step here: this vortex-lattice state needs
O(10^4) iterations to reach that residual.

  python bench.py [--gpus N --steps K --warmup W] [--precision f64|mixed]
  python bench.py --impl reference ...   # the CPU oracle on the same metric

For N > 1 (torchrun) every rank runs its own replica (the solver does not
shard; replicas only) and the value is the sum over ranks of ATKM evaluations
divided by the max over ranks of the time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG time-to-1e-8 residual & ATKM evals/s at 256x256x64; HBM % of peak"
UNIT = "ATKM evals/s"
WORKLOAD = "cfg3_256x256x64"
TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "f64"], default="f64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-form", action="store_true", help="skip the FP32-bulk arm")
    ap.add_argument("--no-time-to-tol", action="store_true", help="skip the multigrid solve to 1e-8")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile-case", choices=["atkm_f32", "atkm_f64", "atkm_df32", "pcg_f64", "pcg_mixed",
                                               "profiling_overhead", "polish_df32"],
                    help="run a small fixed amount of work on the bench grid for an ncu capture, or one of the "
                         "timings quoted in the design notes, and exit")
    return ap.parse_args()


# --------------------------------------------------------------- CPU oracle
def cpu_sample(iters: int = 1) -> dict:
    """Times the CPU oracle (as it stands, one thread) on a bounded sample of
    the workload: plan (untimed), one stand-alone ATKM evaluation, and `iters`
    PCG iterations from psi_0 (the start-up ATKM + energy is timed separately
    and subtracted).  Returns ATKM evaluations per second of the PCG step."""
    import numpy as np
    import atkm_workloads as W
    import oracle as O
    w = W.CONFIGS[WORKLOAD]
    plan = O.Plan(w.N, w.L, w.n)
    prm = O.Params(w.gamma, w.beta, w.lam, w.Omega)
    psi = W.initial_guess(w)
    t0 = time.perf_counter()
    plan.dipolar_potential(np.abs(psi) ** 2)
    t_atkm = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.pcg_ground_state(plan, prm, psi, O.PcgOptions(max_iter=0))
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = O.pcg_ground_state(plan, prm, psi, O.PcgOptions(max_iter=iters))
    t_run = time.perf_counter() - t0
    t_iters = max(t_run - t_init, 1e-9)
    evals = sum(2 + e.get("halvings", 0) for e in res.log[:iters])
    return dict(atkm_s=t_atkm, iter_s=t_iters / iters, iters=iters, evals=evals, value=evals / t_iters, threads=1)


def run_cpu_sample_subprocess() -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample"], capture_output=True, text=True,
                       env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    if int(parts[0]) != self.idx:
                        continue
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            return local_rank
    return local_rank


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# FP64 FMA throughput of this machine's GB300 (FMA-chain microbenchmark, 2 flops
# per FMA, 1216 CTAs x 256 threads x 8 independent chains): 1255 GFLOP/s.
FP64_PEAK_GFLOPS = 1255.0


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# passes that can be the dominant kernel, from one ncu capture of the current
# kernels on this workload (the profile file gives the command).  A kernel not
# listed here reports traffic null.
NCU_TRAFFIC = {
    "atkm_z_f64": {"bytes": 374209280.0, "profile": "profiles/atkm_z_f64_256x256x64.md"},
    "H_z_f32": {"bytes": 172407808.0,
                "profile": "profiles/pcg_mixed_kernels_256x256x64.md (the H phi launch with energy sums)"},
}


# ------------------------------------------------------------------ ours
def atkm_evals(stats) -> int:
    """ATKM evaluations in a profiling record: one x-forward pass each."""
    return sum(k["launches"] for k in stats if k["name"].startswith("atkm_x_fwd"))


def aggregate_ranks(ms: float, evals: float, device: str = "cpu"):
    """Whole-job figures of the replica runs: the slowest rank's time and the
    ATKM evaluations of all ranks (the value is their ratio)."""
    import torch
    import torch.distributed as td
    tm = torch.tensor([ms], dtype=torch.float64, device=device)
    te = torch.tensor([evals], dtype=torch.float64, device=device)
    td.all_reduce(tm, op=td.ReduceOp.MAX)
    td.all_reduce(te, op=td.ReduceOp.SUM)
    return float(tm.item()), float(te.item())


def roofline(stats, peaks):
    dom = max(stats, key=lambda s: s["ms_total"]) if stats else None
    # vector kernels (FP64 vectors, HBM-bound) carry no flops: always "hbm"
    if dom is None or dom["ms_total"] <= 0:
        return None
    per_launch_ms = dom["ms_total"] / dom["launches"]
    if dom["name"].endswith("_f32") or dom["name"].startswith("vec_"):
        achieved = dom["bytes_total"] / (dom["ms_total"] * 1e-3) / 1e9
        return {"kernel": dom["name"], "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": NCU_TRAFFIC.get(dom["name"], {}).get("bytes"),
                "traffic_source": NCU_TRAFFIC.get(dom["name"], {}).get("profile"),
                "algorithmic_bytes_per_launch": dom["bytes_total"] / dom["launches"],
                "launch_ms": round(per_launch_ms, 4), "launches": dom["launches"]}
    achieved = dom["flops_total"] / (dom["ms_total"] * 1e-3) / 1e9
    return {"kernel": dom["name"], "bound": "alu", "achieved": round(achieved, 1), "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
            "peak_source": "measured FP64 FMA microbenchmark on this pool's GB300",
            "traffic": NCU_TRAFFIC.get(dom["name"], {}).get("bytes"),
            "traffic_source": NCU_TRAFFIC.get(dom["name"], {}).get("profile"),
            "algorithmic_flops_per_launch": dom["flops_total"] / dom["launches"],
            "algorithmic_bytes_per_launch": dom["bytes_total"] / dom["launches"],
            "hbm_GBs": round(dom["bytes_total"] / (dom["ms_total"] * 1e-3) / 1e9, 1),
            "launch_ms": round(per_launch_ms, 4), "launches": dom["launches"]}


def timed_steps(B, plan, prm, psi0, precision, warmup, steps, barrier, clk=None):
    """W warm-up PCG iterations from psi_0, then K timed iterations resuming
    the same solve, profiled per pass with CUDA events on the plan stream."""
    import torch
    psi = psi0.clone()
    kw = dict(tol_residual=TOL, precision=precision, switch_tol=1e-5)
    plan.pcg_ground_state(prm, psi, max_iter=warmup, **kw)
    barrier()
    if clk:
        clk.start()
    launches0 = B.launch_count()
    plan.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    res = plan.pcg_ground_state(prm, psi, max_iter=steps, resume=True, **kw)
    ev1.record()
    barrier()
    clocks = clk.stop() if clk else None
    launches = B.launch_count() - launches0
    stats = plan.kernel_stats()
    plan.set_profiling(False)
    return dict(ms=ev0.elapsed_time(ev1), evals=atkm_evals(stats), res=res, stats=stats, clocks=clocks,
                launches=launches, steps=res["iters"] - warmup, psi=psi)


def kernel_table(stats, n=12):
    top = sorted(stats, key=lambda k: -k["ms_total"])[:n]
    return [{"name": k["name"], "launches": k["launches"], "ms": round(k["ms_total"], 3),
             "GB/s": round(k["bytes_total"] / (k["ms_total"] * 1e-3) / 1e9, 1) if k["ms_total"] else None,
             "GFLOP/s": round(k["flops_total"] / (k["ms_total"] * 1e-3) / 1e9, 1) if k["ms_total"] else None}
            for k in top]


def rel2(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def time_to_tol(B, w):
    """PCG-ATKM-MG (Algorithm 2; levels N/4, N/2, N) in the double-word split
    form from guess (d) on the coarsest grid to residual 1e-8 (residual formed
    from the double-word H phi, about 1e-14 relative), wall time around the
    call; plus the FP32- and double-word-vs-FP64 ATKM errors at the final
    state."""
    import torch
    import atkm_workloads as W
    from paper_2603_05194_gb300 import multigrid as MG

    def guess(p, N):
        return W.initial_guess(W.with_grid(p, N))

    res, sec, psi, grids = MG.solve_mg(w, guess, levels=3, tol=TOL, max_iter=20000,
                                       precision=B.PRECISION_DF32_SPLIT)
    plan = B.Plan(w.N, w.L, w.n, f32=True, df32=True)
    try:
        phi64 = plan.dipolar_potential_from_psi(psi)
        phi32 = plan.dipolar_potential_from_psi(psi, f32=True)
        phidw = plan.dipolar_potential_from_psi(psi, df32=True)
        prm = B.make_params(w.gamma, w.beta, w.lam, w.Omega)
        e64 = plan.energy_parts(prm, psi, phi64)
        e32 = plan.energy_parts(prm, psi, phi32)
        err = {"Phi_rel_l2_f32_vs_f64": rel2(phi32, phi64), "Phi_rel_l2_df32_vs_f64": rel2(phidw, phi64),
               "E_rel_f32_vs_f64": abs(e32["E"] - e64["E"]) / abs(e64["E"]),
               "mu_rel_f32_vs_f64": abs(e32["mu"] - e64["mu"]) / abs(e64["mu"])}
    finally:
        plan.close()
    out = MG.summary(res, sec, grids)
    out.update(method="PCG-ATKM-MG, 3 levels, double-word split form (FP32 bulk; polish with H phi and the "
                      "trial-energy ATKM in double-FP32, reductions and retraction in FP64, P r / H p / "
                      "step-model ATKM in FP32)", tol=TOL,
               precision_errors_at_final_state=err)
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import atkm_workloads as W
    from paper_2603_05194_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td
    w = W.CONFIGS[WORKLOAD]
    precision = B.PRECISION_F32_F64 if args.precision == "mixed" else B.PRECISION_F64
    plan = B.Plan(w.N, w.L, w.n, f32=True, df32=True)
    prm = B.make_params(w.gamma, w.beta, w.lam, w.Omega)
    psi0_host = torch.from_numpy(W.initial_guess(w)).pin_memory()
    psi0 = psi0_host.cuda()

    def barrier():
        if dist:
            td.barrier()
        torch.cuda.synchronize()

    # ---- the headline arm: W warm-up + K timed PCG iterations
    main = timed_steps(B, plan, prm, psi0, precision, args.warmup, args.steps, barrier,
                       ClockSampler(gpu_index_for(local_rank)))
    ms_max, evals_all = aggregate_ranks(main["ms"], float(main["evals"]), "cuda") if dist else \
        (main["ms"], float(main["evals"]))

    # ---- the precision form on the same workload (FP32 bulk, FP64 reductions)
    pform = None
    if precision == B.PRECISION_F64 and not args.no_precision_form:
        mx = timed_steps(B, plan, prm, psi0, B.PRECISION_F32_F64, args.warmup, args.steps, barrier)
        mms, mev = aggregate_ranks(mx["ms"], float(mx["evals"]), "cuda") if dist else (mx["ms"], float(mx["evals"]))
        pform = {"value": round(mev / (mms * 1e-3), 2), "unit": UNIT,
                 "ms_per_step": round(mms / max(mx["steps"], 1), 3), "steps": mx["steps"],
                 "roofline": roofline(mx["stats"], measured_peaks()), "kernels": kernel_table(mx["stats"]),
                 "gpu_launches": mx["launches"], "residual_after_steps": mx["res"]["residual"],
                 "f32_iterations": mx["res"]["f32_iters"]}

    # ---- stand-alone ATKM evaluations per second (FP64 and FP32 arithmetic)
    Phi = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    standalone = {}
    for key, kw in (("f64", {}), ("df32", {"df32": True}), ("f32", {"f32": True})):
        for _ in range(3):
            plan.dipolar_potential_from_psi(psi0, out=Phi, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 50
        e0.record()
        for _ in range(n):
            plan.dipolar_potential_from_psi(psi0, out=Phi, **kw)
        e1.record()
        torch.cuda.synchronize()
        standalone[key] = round(n / (e0.elapsed_time(e1) * 1e-3), 1)

    # ---- end to end through the public API with host buffers: H2D of psi_0,
    # W + K iterations from it, D2H of the state
    barrier()
    psi = torch.empty_like(psi0)
    host_out = torch.empty_like(psi0_host).pin_memory()
    kw = dict(tol_residual=TOL, precision=precision, switch_tol=1e-5)
    plan.set_profiling(True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    psi.copy_(psi0_host, non_blocking=True)
    plan.pcg_ground_state(prm, psi, max_iter=args.warmup + args.steps, **kw)
    host_out.copy_(psi, non_blocking=True)
    f1.record()
    barrier()
    e2e_stats = plan.kernel_stats()
    plan.set_profiling(False)
    e2e_ms = f0.elapsed_time(f1)
    e2e_evals = atkm_evals(e2e_stats)
    nbytes = psi0_host.numel() * psi0_host.element_size()
    plan.close()

    # ---- time to the residual tolerance (single process only: replicas would
    # only repeat it)
    ttt = None
    if not args.no_time_to_tol and world == 1:
        ttt = time_to_tol(B, w)
    return dict(ms=ms_max, evals=evals_all, steps=main["steps"], res=main["res"], standalone=standalone,
                e2e_value=e2e_evals * world / (e2e_ms * 1e-3), nbytes=nbytes,
                roof=roofline(main["stats"], measured_peaks()), stats=main["stats"], clocks=main["clocks"],
                launches=main["launches"], pform=pform, ttt=ttt)


def timing_case(case: str):
    """Timings quoted in the design notes, one JSON line each.
    profiling_overhead: 30 FP64 PCG iterations (after 3) without and with the
    per-pass CUDA events, twice.  polish_df32: 1500 iterations of the
    double-word split form from psi_0 (the FP32 phase, then the polish), then
    200 polish iterations without and with the events, with the per-pass
    times per iteration."""
    import torch
    import atkm_workloads as W
    from paper_2603_05194_gb300 import binding as B
    w = W.CONFIGS[WORKLOAD]
    prm = B.make_params(w.gamma, w.beta, w.lam, w.Omega)
    psi0 = torch.from_numpy(W.initial_guess(w)).cuda()

    def timed(plan, psi, n, prof, kw):
        plan.set_profiling(prof)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = plan.pcg_ground_state(prm, psi, max_iter=n, resume=True, **kw)
        e1.record()
        torch.cuda.synchronize()
        stats = plan.kernel_stats() if prof else []
        plan.set_profiling(False)
        return r, e0.elapsed_time(e1), stats

    if case == "profiling_overhead":
        plan = B.Plan(w.N, w.L, w.n)
        kw = dict(tol_residual=TOL, precision=B.PRECISION_F64, switch_tol=1e-5)
        try:
            for prof in (False, True, False, True):
                psi = psi0.clone()
                plan.pcg_ground_state(prm, psi, max_iter=3, **kw)
                torch.cuda.synchronize()
                r, ms, _ = timed(plan, psi, 30, prof, kw)
                n = r["iters"] - 3
                print(json.dumps({"case": case, "profiling": prof, "iters": n, "ms_per_iter": ms / max(n, 1)}))
        finally:
            plan.close()
        return
    plan = B.Plan(w.N, w.L, w.n, f32=True, df32=True)
    kw = dict(tol_residual=TOL, precision=B.PRECISION_DF32_SPLIT, switch_tol=1e-5)
    try:
        psi = psi0.clone()
        r = plan.pcg_ground_state(prm, psi, max_iter=1500, **kw)
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "warm_iters": r["iters"], "f32_iters": r["f32_iters"],
                          "residual": r["residual"]}))
        for prof in (False, True):
            it0 = r["iters"]
            r, ms, stats = timed(plan, psi, 200, prof, kw)
            n = max(r["iters"] - it0, 1)
            out = {"case": case, "profiling": prof, "iters": n, "ms_per_iter": ms / n}
            if prof:
                out["kernel_ms_per_iter"] = sum(k["ms_total"] for k in stats) / n
                out["passes_ms_per_iter"] = [(k["name"], round(k["ms_total"] / n, 4))
                                             for k in sorted(stats, key=lambda k: -k["ms_total"])]
            print(json.dumps(out))
    finally:
        plan.close()


def profile_case(case: str):
    """Small fixed workloads on the bench grid for ncu captures (about 1 GB of
    device memory): two ATKM evaluations, or three PCG iterations."""
    if case in ("profiling_overhead", "polish_df32"):
        timing_case(case)
        return
    import torch
    import atkm_workloads as W
    from paper_2603_05194_gb300 import binding as B
    w = W.CONFIGS[WORKLOAD]
    plan = B.Plan(w.N, w.L, w.n, f32=True, df32=True)
    psi = torch.from_numpy(W.initial_guess(w)).cuda()
    if case.startswith("atkm"):
        for _ in range(2):
            Phi = plan.dipolar_potential_from_psi(psi, f32=(case == "atkm_f32"), df32=(case == "atkm_df32"))
        torch.cuda.synchronize()
        print(case, "max|Phi|", float(Phi.abs().max()))
    else:
        prm = B.make_params(w.gamma, w.beta, w.lam, w.Omega)
        prec = B.PRECISION_F64 if case == "pcg_f64" else B.PRECISION_F32_F64
        r = plan.pcg_ground_state(prm, psi, max_iter=3, precision=prec)
        torch.cuda.synchronize()
        print(case, r["status_name"], r["iters"], r["E"])


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample()))
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # The CPU oracle on the same metric, rank 0 only; other ranks exit without work.
        if rank != 0:
            return
        samples = [run_cpu_sample_subprocess() for _ in range(args.warmup + args.steps)]
        timed = samples[args.warmup:] if len(samples) > args.warmup else samples
        value = statistics.median(s["value"] for s in timed)
        it_s = statistics.median(s["iter_s"] for s in timed)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": it_s * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": [256, 256, 64], "step": "one PCG iteration (all rows)",
                           "precision": "f64"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": "each step: one oracle PCG iteration of the workload from psi_0 "
                                           "(numpy/scipy FP64, one thread), start-up excluded",
                                 "standalone_atkm_evals_per_s": 1.0 / statistics.median(s["atkm_s"] for s in timed)},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            s = run_cpu_sample_subprocess()
            cpu = {"value": round(s["value"], 4), "unit": UNIT, "cores": s["threads"], "kind": "oracle",
                   "sample": f"one oracle PCG iteration of the same workload from psi_0 ({s['iter_s']:.1f} s, "
                             f"{s['evals']} ATKM evals; numpy/scipy FP64, one thread); stand-alone oracle ATKM "
                             f"{s['atkm_s']:.2f} s"}
        except Exception as exc:  # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"[:300]}
    if rank == 0:
        res = out["res"]
        value = out["evals"] / (out["ms"] * 1e-3)
        ktable = kernel_table(out["stats"], 24)
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": out["steps"],
            "warmup": args.warmup, "ms_per_step": round(out["ms"] / max(out["steps"], 1), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "f64" else "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [256, 256, 64], "step": "one PCG iteration (all rows)",
                       "precision": args.precision, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (padded ATKM spectrum 268-537 MB per pass)",
                       "atkm_evals_in_steps": int(out["evals"]), "iteration_after_steps": res["iters"],
                       "residual_after_steps": res["residual"], "E_after_steps": res["E"],
                       "halvings": res["halvings"]},
            "standalone_atkm_evals_per_s": out["standalone"],
            "roofline": out["roof"], "kernels": ktable, "clocks": out["clocks"],
            "gpu_launches": out["launches"],
            "e2e": {"value": round(out["e2e_value"], 2), "unit": UNIT,
                    "h2d_bytes_per_step": round(out["nbytes"] / (args.warmup + args.steps)),
                    "d2h_bytes_per_step": round(out["nbytes"] / (args.warmup + args.steps)),
                    "note": "pcg_ground_state from pinned host psi_0: one H2D of psi_0, warmup+steps iterations, "
                            "one D2H of the state, all inside the timed region (bytes per step = bytes / iterations)"},
            "cpu_baseline": cpu,
            "precision_form": out["pform"],
            "time_to_1e-8": out["ttt"],
        }
        print(json.dumps(line))
    if dist:
        td.destroy_process_group()


if __name__ == "__main__":
    main()
