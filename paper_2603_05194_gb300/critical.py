"""Critical rotation frequency Omega_c on the batched solver (§3, Examples
3.4 and 3.5).

A vortex appears in the ground state once Omega exceeds Omega_c.  For each
Omega of a sweep, two states are solved in one batched call
(pcg_ground_state_batched): one from the vortex-free Gaussian (guess (a) of
§3) and one from the single-vortex guess (b) = (x + iy) times it.  Each
converged state is classified by its angular momentum <L_z> = -E_rot/Omega
(about 0 without a vortex, about 1 with one centred vortex).  With E_0(Omega)
the lowest energy among the vortex-free states and E_1(Omega) among the
one-vortex states, Omega_c is the root of dE(Omega) = E_1 - E_0, taken from a
least-squares line through the Omegas where both exist (in an axially
symmetric setup E_0 does not depend on Omega and E_1 falls with slope
-<L_z>, so dE is a straight line).  Energy components and the virial residual
are reported per state.  This module only sets up the instances and reads
the results.

  python -m paper_2603_05194_gb300.critical --example 3.5 --case I ...
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B


def _mesh(N, L):
    axes = [-L[a] + (2.0 * L[a] / N[a]) * np.arange(N[a]) for a in range(3)]
    return axes[0][None, None, :], axes[1][None, :, None], axes[2][:, None, None]


def _normalised(f, N, L):
    h3 = np.prod([2.0 * L[a] / N[a] for a in range(3)])
    f = np.broadcast_to(f, (N[2], N[1], N[0])).astype(np.complex128)
    return f / math.sqrt(h3 * float(np.sum(np.abs(f) ** 2)))


def guess_vortex_free(N, L):
    """Guess (a) of §3: the unit-width Gaussian."""
    x, y, z = _mesh(N, L)
    return _normalised(np.exp(-(x * x + y * y + z * z) / 2.0), N, L)


def guess_one_vortex(N, L):
    """Guess (b) of §3: (x + i y) times the unit-width Gaussian."""
    x, y, z = _mesh(N, L)
    return _normalised((x + 1j * y) * np.exp(-(x * x + y * y + z * z) / 2.0), N, L)


def energies_vs_omega(gamma, beta, lam, n, omegas, N, L, tol=1e-8, max_iter=6000, precision=B.PRECISION_F64):
    """One batched solve of both guesses at every Omega; one row per Omega."""
    plans, prms, psis, tags = [], [], [], []
    for Om in omegas:
        for tag, fn in (("a", guess_vortex_free), ("b", guess_one_vortex)):
            plans.append(B.Plan(N, L, n, f32=precision != B.PRECISION_F64, df32=precision == B.PRECISION_DF32_SPLIT))
            prms.append(B.make_params(gamma, beta, lam, Om))
            psis.append(torch.from_numpy(fn(N, L)).cuda())
            tags.append((Om, tag))
    try:
        outs = B.pcg_ground_state_batched(plans, prms, psis, tol_residual=tol, max_iter=max_iter, precision=precision)
    finally:
        for p in plans:
            p.close()
    rows = {}
    for (Om, tag), o in zip(tags, outs):
        Lz = -o["E_rot"] / Om if Om != 0 else 0.0
        rows.setdefault(Om, {})[tag] = dict(status=o["status_name"], iters=o["iters"], E=o["E"], mu=o["mu"], Lz=Lz,
                                            E_kin=o["E_kin"], E_pot=o["E_pot"], E_int=o["E_int"], E_dip=o["E_dip"],
                                            E_rot=o["E_rot"], virial=o["virial"], residual=o["residual"])
    return [dict(Omega=Om, **rows[Om]) for Om in omegas]


def critical_omega(rows) -> dict:
    """Omega_c from the rows of energies_vs_omega (see the module docstring)."""
    pts = []
    for r in rows:
        states = [r[t] for t in ("a", "b") if r[t]["status"] == "OK"]
        free = [s["E"] for s in states if abs(s["Lz"]) < 0.5]
        one = [s["E"] for s in states if 0.5 <= s["Lz"] < 1.5]
        if free and one:
            pts.append((r["Omega"], min(one) - min(free)))
    out = {"points": [[o, d] for o, d in pts]}
    if len(pts) < 2:
        out["Omega_c"] = None
        return out
    om = np.array([p[0] for p in pts])
    dE = np.array([p[1] for p in pts])
    slope, icpt = np.polyfit(om, dE, 1)
    out.update(Omega_c=float(-icpt / slope) if slope != 0 else None, slope=float(slope),
               fit_residual=float(np.max(np.abs(icpt + slope * om - dE))))
    return out


def omega_c(gamma, beta, lam, n, N, L, omegas=None, **kw) -> dict:
    omegas = list(omegas) if omegas is not None else [0.15 + 0.1 * i for i in range(8)]
    rows = energies_vs_omega(gamma, beta, lam, n, omegas, N, L, **kw)
    res = critical_omega(rows)
    res["rows"] = rows
    return res


# Setups of Examples 3.4 and 3.5 (box [-10,10]^3 unless stated; the paper
# runs 128^3, and 256^3 on [-16,16]^3 for Example 3.4 Cases I-II).
def example_setups(example: str, case: str):
    """(label, gamma, beta, lambda, n, L) tuples of one case of an example."""
    box = (10.0, 10.0, 10.0)
    z, x = (0.0, 0.0, 1.0), (1.0, 0.0, 0.0)
    if example == "3.4":
        if case == "I":
            return [(f"gamma_y={gy}", (1.0, gy, 1.0), 2000.0, 0.0, z, (16.0, 16.0, 16.0)) for gy in (1.0, 1.1, 1.2, 1.3)]
        if case == "II":
            return [(f"gamma_z={gz}", (1.0, 1.0, gz), 2000.0, 0.0, z, (16.0, 16.0, 16.0)) for gz in (1.0, 2.0, 4.0)]
        return [(f"beta={b}", (1.0, 1.0, 1.0), b, 0.0, z, box) for b in (100.0, 200.0, 400.0, 800.0)]
    if case in ("I", "II"):
        nn = z if case == "I" else x
        return [(f"beta={b},lambda={l}", (1.0, 1.0, 1.0), b, l, nn, box)
                for b in (200.0, 300.0, 400.0) for l in (-100.0, 0.0, 100.0)]
    out = []
    for l in (-100.0, 100.0):
        for th in (0.0, 45.0, 90.0):
            t = math.radians(th)
            out.append((f"lambda={l},theta={th}", (1.0, 1.0, 1.0), 400.0, l, (math.sin(t), 0.0, math.cos(t)), box))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="critical rotation frequency on the batched solver (Examples 3.4-3.5)")
    ap.add_argument("--example", choices=["3.4", "3.5"], default="3.5")
    ap.add_argument("--case", choices=["I", "II", "III"], default="I")
    ap.add_argument("--n", type=int, default=64, help="grid points per axis")
    ap.add_argument("--omegas", default="0.15,0.25,0.35,0.45,0.55,0.65,0.75,0.85")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    B.load_library()
    omegas = [float(v) for v in a.omegas.split(",")]
    N = (a.n, a.n, a.n)
    results = []
    for label, gamma, beta, lam, nn, L in example_setups(a.example, a.case):
        t0 = time.perf_counter()
        r = omega_c(gamma, beta, lam, nn, N, L, omegas, tol=a.tol)
        r.update(label=label, seconds=round(time.perf_counter() - t0, 2), grid=list(N), box=list(L))
        print(json.dumps({k: v for k, v in r.items() if k != "rows"}))
        results.append(r)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(dict(example=a.example, case=a.case, results=results), fh)


if __name__ == "__main__":
    main()
