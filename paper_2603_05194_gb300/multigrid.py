"""Time to the residual tolerance with the cascadic multigrid driver.

PCG-ATKM-MG (Algorithm 2) solves on N/4, N/2 and N points per axis, each
level seeded by the Fourier interpolant of the previous level's ground state;
the paper runs every experiment this way.  This module sets up the levels of
a problem, runs pcg_ground_state_mg, and for comparison Algorithm 1 on the
finest grid alone from the same formula guess.  It only orders calls.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import binding as B


def level_grids(N, levels=3):
    """N_a / 2^(levels-1-i) per axis, coarsest first (each must stay even)."""
    out = []
    for i in range(levels):
        f = 2 ** (levels - 1 - i)
        g = tuple(int(n) // f for n in N)
        if any(n % f or v % 2 for n, v in zip(N, g)):
            raise ValueError(f"grid {tuple(N)} does not coarsen {levels - 1} times to even sizes")
        out.append(g)
    return out


def solve_mg(problem, psi0_fn, levels=3, tol=1e-8, max_iter=20000, precision=B.PRECISION_F32_F64):
    """Runs Algorithm 2 on the problem; psi0_fn(problem, N) gives the initial
    guess on the coarsest grid.  Returns (per-level results, seconds, finest psi)."""
    grids = level_grids(problem.N, levels)
    f32 = precision != B.PRECISION_F64
    df32 = precision == B.PRECISION_DF32_SPLIT
    plans = [B.Plan(N, problem.L, problem.n, f32=f32, df32=df32) for N in grids]
    try:
        psis = [torch.from_numpy(psi0_fn(problem, grids[0])).cuda()] + \
               [torch.empty(p.shape, dtype=torch.complex128, device="cuda") for p in plans[1:]]
        prm = B.make_params(problem.gamma, problem.beta, problem.lam, problem.Omega)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = B.pcg_ground_state_mg(plans, prm, psis, tol_residual=tol, max_iter=max_iter, precision=precision)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0, psis[-1], grids
    finally:
        for p in plans:
            p.close()


def solve_single(problem, psi0_fn, tol=1e-8, max_iter=20000, precision=B.PRECISION_F32_F64):
    plan = B.Plan(problem.N, problem.L, problem.n, f32=(precision != B.PRECISION_F64),
                  df32=(precision == B.PRECISION_DF32_SPLIT))
    try:
        psi = torch.from_numpy(psi0_fn(problem, problem.N)).cuda()
        prm = B.make_params(problem.gamma, problem.beta, problem.lam, problem.Omega)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = plan.pcg_ground_state(prm, psi, tol_residual=tol, max_iter=max_iter, precision=precision)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0
    finally:
        plan.close()


def summary(res, seconds, grids):
    return dict(seconds=seconds, status=res[-1]["status_name"], E=res[-1]["E"], mu=res[-1]["mu"],
                residual=res[-1]["residual"],
                levels=[dict(grid=list(g), iters=r["iters"], f32_iters=r["f32_iters"], status=r["status_name"],
                             residual=r["residual"], E=r["E"]) for g, r in zip(grids, res)])


def main(argv=None):
    import atkm_workloads as W
    ap = argparse.ArgumentParser(description="time to the residual tolerance: PCG-ATKM-MG vs single-level PCG")
    ap.add_argument("--workload", default="cfg3_256x256x64", choices=sorted(W.CONFIGS))
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=20000, help="per level")
    ap.add_argument("--precision", choices=["dwsplit", "split", "mixed", "f64"], default="split")
    ap.add_argument("--single", action="store_true", help="also run the finest grid alone from the same guess")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    B.load_library()
    w = W.CONFIGS[a.workload]
    prec = {"dwsplit": B.PRECISION_DF32_SPLIT, "split": B.PRECISION_F32_SPLIT, "mixed": B.PRECISION_F32_F64,
            "f64": B.PRECISION_F64}[a.precision]

    def guess(p, N):
        return W.initial_guess(W.with_grid(p, N))

    res, sec, _, grids = solve_mg(w, guess, a.levels, a.tol, a.max_iter, prec)
    out = dict(workload=a.workload, precision=a.precision, tol=a.tol, max_iter_per_level=a.max_iter,
               mg=summary(res, sec, grids))
    print(json.dumps(out["mg"]))
    if a.single:
        r, s = solve_single(w, guess, a.tol, a.max_iter, prec)
        out["single"] = dict(seconds=s, status=r["status_name"], iters=r["iters"], f32_iters=r["f32_iters"],
                             E=r["E"], residual=r["residual"])
        print(json.dumps(out["single"]))
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(json.dumps(out) + "\n")


if __name__ == "__main__":
    main()
