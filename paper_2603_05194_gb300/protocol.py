"""The paper's ground-state protocol: Algorithm 1 from each of the ten
initial guesses of §3 and the lowest energy kept as the ground state, with the
stop rule ||phi_{n+1} - phi_n||_inf <= 1e-10 (Eq. (stop_maxnorm)).

The ten solves are independent, so they run as one batched call
(pcg_ground_state_batched; each instance needs a plan of its own, all for the
same grid and box).  This module only orders the calls and compares the
energies; the guesses themselves are inputs (see atkm_workloads.paper_guesses).
"""
from __future__ import annotations

import time

import torch

from . import binding as B


def lowest_energy_state(N, L, n, params: B.Params, guesses: dict, tol_residual=0.0, tol_linf=1e-10,
                        max_iter=20000, precision=B.PRECISION_F64):
    """Solves from every guess (name -> host complex128 array of shape
    (N_z, N_y, N_x)) in one batched call.  Returns (name of the lowest-energy
    finished solve, {name: result dict}, {name: final device state}, seconds).
    Solves that end in an error status are not candidates."""
    names = list(guesses)
    f32 = precision != B.PRECISION_F64
    plans = [B.Plan(N, L, n, f32=f32, df32=(precision == B.PRECISION_DF32_SPLIT)) for _ in names]
    try:
        psis = [torch.from_numpy(guesses[k]).cuda() for k in names]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = B.pcg_ground_state_batched(plans, [params] * len(names), psis, tol_residual=tol_residual,
                                         tol_linf=tol_linf, max_iter=max_iter, precision=precision)
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
    finally:
        for p in plans:
            p.close()
    results = dict(zip(names, res))
    ok = [k for k in names if results[k]["status_name"] in ("OK", "NOT_CONVERGED", "STAGNATED")]
    if not ok:
        raise RuntimeError("no solve of the protocol finished")
    best = min(ok, key=lambda k: results[k]["E"])
    return best, results, dict(zip(names, psis)), seconds
