"""Batched sweep of independent ground-state problems on uneven grids.

Every instance is its own Algorithm 1 run (own plan, own multiplier K, own
state); pcg_ground_state_batched builds all of them into one CUDA graph and
launches it once.  The plans are autotuned (atkm_plan_autotune: the FFT
engine and tile of every non-power-of-two line length picked by timing).
This module times that call against the same instances solved one after
another (and against untuned plans), and runs the sweep to the residual
tolerance (in one launch, double-word split form), optionally against each
instance solved alone in binary64.  It only orders calls and keeps the
books.
"""
from __future__ import annotations

import argparse
import collections
import json
import time

import torch

from . import binding as B


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def _summary(res, seconds):
    st = collections.Counter(r["status_name"] for r in res)
    return dict(seconds=seconds, statuses=dict(st), iters=[r["iters"] for r in res],
                residual=[r["residual"] for r in res], E=[r["E"] for r in res],
                device_loop=all(r.get("device_loop", False) for r in res))


def _agreement(res, ref):
    both = [(a, b) for a, b in zip(res, ref) if a["status"] == B.ATKM_OK and b["status"] == B.ATKM_OK]
    dE = [(a["E"] - b["E"]) / abs(b["E"]) for a, b in both]
    return dict(both_converged=len(both), same_energy=sum(abs(d) <= 1e-9 for d in dE),
                lower_energy=sum(d < -1e-9 for d in dE), higher_energy=sum(d > 1e-9 for d in dE),
                max_abs_rel_dE_same=max([abs(d) for d in dE if abs(d) <= 1e-9], default=0.0))


def to_tolerance(problems, psi0_fn, max_iter=12000, tol=1e-8, log=print, autotune=True):
    """The sweep to the residual tolerance three ways on the same autotuned
    plans: every instance alone in binary64, one after another (the plain
    method); all instances in one graph launch in binary64 (the batching
    alone: the same arithmetic, so the same trajectories and energies); and
    all in one launch in the double-word split form (FP32 bulk phase)."""
    plans = [B.Plan(p.N, p.L, p.n, f32=True, df32=True, autotune=autotune) for p in problems]
    prms = [B.make_params(p.gamma, p.beta, p.lam, p.Omega) for p in problems]

    def psis():
        return [torch.from_numpy(psi0_fn(p)).cuda() for p in problems]

    out = dict(instances=len(problems), grids=[list(p.N) for p in problems], tol=tol, max_iter=max_iter,
               autotune=autotune)
    if autotune:
        tun = [t for pl in plans for t in pl.tuning()]
        out["tuning"] = dict(entries=len(tun), changed=sum(1 for t in tun if t["ms_best"] < t["ms_default"]),
                             mixed_radix=sum(1 for t in tun if t["engine"] == 1),
                             narrowed_tiles=sum(1 for t in tun if t["engine"] == 2 and t["tile_shift"] > 0),
                             ms_default=sum(t["ms_default"] for t in tun), ms_best=sum(t["ms_best"] for t in tun))
    try:
        for prec in (B.PRECISION_F64, B.PRECISION_DF32_SPLIT):  # capture every instance's graphs once
            B.pcg_ground_state_batched(plans, prms, psis(), max_iter=3, precision=prec)
        ps = psis()
        ref, tr = _timed(lambda: [pl.pcg_ground_state(pr, p, max_iter=max_iter, tol_residual=tol,
                                                      precision=B.PRECISION_F64)
                                  for pl, pr, p in zip(plans, prms, ps)])
        out["f64_one_by_one"] = _summary(ref, tr)
        log(f"binary64, one by one: {tr:.1f} s, {out['f64_one_by_one']['statuses']}")
        for name, prec in (("f64_batched", B.PRECISION_F64), ("df32_split_batched", B.PRECISION_DF32_SPLIT)):
            ps = psis()
            res, t = _timed(lambda: B.pcg_ground_state_batched(plans, prms, ps, max_iter=max_iter, tol_residual=tol,
                                                               precision=prec))
            out[name] = _summary(res, t)
            out[name]["speedup_vs_f64_one_by_one"] = tr / t
            out[name]["energy_vs_f64_one_by_one"] = _agreement(res, ref)
            log(f"{name}: {t:.1f} s ({tr / t:.2f}x), {out[name]['statuses']}, "
                f"energies {out[name]['energy_vs_f64_one_by_one']}")
    finally:
        for pl in plans:
            pl.close()
    return out


def run(problems, psi0_fn, iters=40, full_iters=3000, tol=1e-8, precisions=(B.PRECISION_F32_F64, B.PRECISION_F64),
        log=print, reference=False, autotune=True):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plans = [B.Plan(p.N, p.L, p.n, f32=True, df32=True, autotune=autotune) for p in problems]
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    prms = [B.make_params(p.gamma, p.beta, p.lam, p.Omega) for p in problems]

    def psis():
        return [torch.from_numpy(psi0_fn(p)).cuda() for p in problems]

    out = dict(instances=len(problems), grids=[list(p.N) for p in problems], fixed_iters=iters, autotune=autotune,
               plan_create_s=tune_s)
    if autotune:
        tun = [t for pl in plans for t in pl.tuning()]
        out["tuning"] = dict(entries=len(tun), changed=sum(1 for t in tun if t["ms_best"] < t["ms_default"]),
                             mixed_radix=sum(1 for t in tun if t["engine"] == 1),
                             narrowed_tiles=sum(1 for t in tun if t["engine"] == 2 and t["tile_shift"] > 0),
                             ms_default=sum(t["ms_default"] for t in tun), ms_best=sum(t["ms_best"] for t in tun))
        log(f"autotuned {len(plans)} plans in {tune_s:.1f} s (plan creation included): {out['tuning']}")
    untuned = [B.Plan(p.N, p.L, p.n, f32=True, df32=True) for p in problems] if autotune else None
    try:
        for prec in precisions:
            name = "mixed" if prec == B.PRECISION_F32_F64 else "f64"
            arms = [("", plans)] + ([("untuned_", untuned)] if untuned else [])
            for label, pls in arms:
                ps = psis()
                B.pcg_ground_state_batched(pls, prms, ps, max_iter=3, precision=prec)  # capture graphs
                ps = psis()
                _, tb = _timed(lambda: B.pcg_ground_state_batched(pls, prms, ps, max_iter=iters, tol_residual=0.0,
                                                                  precision=prec))
                out[f"{name}_{label}batched_s"] = tb
            ps = psis()
            _, ts = _timed(lambda: [pl.pcg_ground_state(pr, p, max_iter=iters, tol_residual=0.0, precision=prec)
                                    for pl, pr, p in zip(plans, prms, ps)])
            tb = out[f"{name}_batched_s"]
            out[f"{name}_sequential_s"] = ts
            out[f"{name}_instance_iters_per_s_batched"] = len(problems) * iters / tb
            log(f"{name}: {iters} iterations x {len(problems)} instances: batched {tb:.3f} s, "
                f"one by one {ts:.3f} s ({ts / tb:.2f}x)" +
                (f", batched on untuned plans {out[f'{name}_untuned_batched_s']:.3f} s" if untuned else ""))
        if full_iters > 0:
            # the sweep to the tolerance: all instances in one graph launch
            # (double-word split form) against each instance alone in binary64
            ps = psis()
            res, t = _timed(lambda: B.pcg_ground_state_batched(plans, prms, ps, max_iter=full_iters, tol_residual=tol,
                                                               precision=B.PRECISION_DF32_SPLIT))
            st = collections.Counter(r["status_name"] for r in res)
            out["full"] = dict(tol=tol, max_iter=full_iters, seconds=t, statuses=dict(st),
                               iters=[r["iters"] for r in res], residual=[r["residual"] for r in res],
                               E=[r["E"] for r in res], device_loop=all(r["device_loop"] for r in res))
            log(f"sweep to {tol:g} (one launch, double-word split form, at most {full_iters} iterations): "
                f"{t:.1f} s, {dict(st)}")
            if reference:
                ps = psis()
                ref, tr = _timed(lambda: [pl.pcg_ground_state(pr, p, max_iter=full_iters, tol_residual=tol,
                                                              precision=B.PRECISION_F64)
                                          for pl, pr, p in zip(plans, prms, ps)])
                sr = collections.Counter(r["status_name"] for r in ref)
                both = [(a, b) for a, b in zip(res, ref) if a["status"] == B.ATKM_OK and b["status"] == B.ATKM_OK]
                dE = [(a["E"] - b["E"]) / abs(b["E"]) for a, b in both]
                out["reference_f64_one_by_one"] = dict(
                    seconds=tr, statuses=dict(sr), iters=[r["iters"] for r in ref], E=[r["E"] for r in ref],
                    both_converged=len(both), same_energy=sum(abs(d) <= 1e-9 for d in dE),
                    lower_energy_batched=sum(d < -1e-9 for d in dE), higher_energy_batched=sum(d > 1e-9 for d in dE),
                    speedup=tr / t)
                log(f"reference, one by one in binary64: {tr:.1f} s, {dict(sr)}; batched/reference energies: "
                    f"{out['reference_f64_one_by_one']['same_energy']} same, "
                    f"{out['reference_f64_one_by_one']['lower_energy_batched']} lower, "
                    f"{out['reference_f64_one_by_one']['higher_energy_batched']} higher of {len(both)}")
    finally:
        for pl in plans + (untuned or []):
            pl.close()
    return out


def main(argv=None):
    import atkm_workloads as W
    ap = argparse.ArgumentParser(description="batched uneven-grid sweep vs one-by-one solves")
    ap.add_argument("--count", type=int, default=48)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--full-iters", type=int, default=3000, help="0 skips the run to the tolerance")
    ap.add_argument("--reference", action="store_true", help="also solve each instance alone in binary64")
    ap.add_argument("--no-autotune", action="store_true", help="plans with the fixed engine rule")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    B.load_library()
    res = run(W.sweep_instances(a.count), W.initial_guess, a.iters, a.full_iters, reference=a.reference,
              autotune=not a.no_autotune)
    js = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(js + "\n")
    print(json.dumps({k: v for k, v in res.items() if k not in ("grids", "full", "reference_f64_one_by_one")}))
    if "full" in res:
        f = res["full"]
        print(json.dumps({"full": {k: f[k] for k in ("tol", "max_iter", "seconds", "statuses", "device_loop")}}))


if __name__ == "__main__":
    main()
