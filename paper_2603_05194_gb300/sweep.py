"""Batched sweep of independent ground-state problems on uneven grids.

Every instance is its own Algorithm 1 run (own plan, own multiplier K, own
state); pcg_ground_state_batched runs them concurrently, each on its own
stream with graph-captured iterations, and the host processes each instance as
soon as its last phase has finished.  This module times that call against the
same instances solved one after another, and runs the sweep to the residual
tolerance.  It only orders calls and keeps the books.
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


def run(problems, psi0_fn, iters=40, full_iters=3000, tol=1e-8, precisions=(B.PRECISION_F32_F64, B.PRECISION_F64),
        log=print):
    plans = [B.Plan(p.N, p.L, p.n, f32=True, df32=True) for p in problems]
    prms = [B.make_params(p.gamma, p.beta, p.lam, p.Omega) for p in problems]

    def psis():
        return [torch.from_numpy(psi0_fn(p)).cuda() for p in problems]

    out = dict(instances=len(problems), grids=[list(p.N) for p in problems], fixed_iters=iters)
    try:
        for prec in precisions:
            name = "mixed" if prec == B.PRECISION_F32_F64 else "f64"
            ps = psis()
            B.pcg_ground_state_batched(plans, prms, ps, max_iter=3, precision=prec)  # capture graphs
            ps = psis()
            _, tb = _timed(lambda: B.pcg_ground_state_batched(plans, prms, ps, max_iter=iters, tol_residual=0.0,
                                                              precision=prec))
            ps = psis()
            _, ts = _timed(lambda: [pl.pcg_ground_state(pr, p, max_iter=iters, tol_residual=0.0, precision=prec)
                                    for pl, pr, p in zip(plans, prms, ps)])
            out[f"{name}_batched_s"] = tb
            out[f"{name}_sequential_s"] = ts
            out[f"{name}_instance_iters_per_s_batched"] = len(problems) * iters / tb
            log(f"{name}: {iters} iterations x {len(problems)} instances: batched {tb:.3f} s, "
                f"one by one {ts:.3f} s ({ts / tb:.2f}x)")
        if full_iters > 0:
            ps = psis()
            res, t = _timed(lambda: B.pcg_ground_state_batched(plans, prms, ps, max_iter=full_iters, tol_residual=tol,
                                                               precision=B.PRECISION_DF32_SPLIT))
            st = collections.Counter(r["status_name"] for r in res)
            out["full"] = dict(tol=tol, max_iter=full_iters, seconds=t, statuses=dict(st),
                               iters=[r["iters"] for r in res], residual=[r["residual"] for r in res],
                               E=[r["E"] for r in res])
            log(f"sweep to {tol:g} (double-word split form, at most {full_iters} iterations): {t:.1f} s, {dict(st)}")
    finally:
        for pl in plans:
            pl.close()
    return out


def main(argv=None):
    import atkm_workloads as W
    ap = argparse.ArgumentParser(description="batched uneven-grid sweep vs one-by-one solves")
    ap.add_argument("--count", type=int, default=48)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--full-iters", type=int, default=3000, help="0 skips the run to the tolerance")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    B.load_library()
    res = run(W.sweep_instances(a.count), W.initial_guess, a.iters, a.full_iters)
    js = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(js + "\n")
    print(json.dumps({k: v for k, v in res.items() if k not in ("grids", "full")}))


if __name__ == "__main__":
    main()
