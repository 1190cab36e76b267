"""The CUDA solver against the energies the paper prints for the U-shape
vortex line of Example 3.2 (Table 2; tests/golden/table2_example32.txt): a
cigar trap (gamma_z = 0.05) in a 1:1:10 box with attractive dipoles.

The paper keeps the lowest energy over its initial guesses.  Here:
  * 256^3: the cascadic multigrid driver (64^3, 128^3, 256^3; binary64, stop
    at residual 1e-9) from guess (d) ends at E = 2.2762103901793, the printed
    2.276210390179 to all 12 decimals (194, 165 and 81 iterations, about 4 s);
    checked to 1e-12 absolute.  (Other guesses end higher: (b) at
    2.276210396898, (a) and the Thomas-Fermi guess at 2.286022170034.  The
    split precision form from guess (d) wanders on the coarsest level -- its
    FP32 direction and step-model operators slow the polish there to 5e4
    iterations -- and ends at 2.2762103968981, the state of guess (b).)
  * 128^3: the paper's under-resolved S-shape state (its |I| ~ 9e-6), reached
    here from guess (b): E agrees to 1.4e-10 absolute; checked to 5e-10, and
    |I| to 1e-2 relative.
The 128^3 state is reached in the split precision form.
"""
import math
import os

import numpy as np
import pytest
import torch

import atkm_workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_example32.txt")
GAMMA, L, BETA, LAM, NAX, OM = (1.0, 1.0, 0.05), (10.0, 10.0, 100.0), 1000.0, -300.0, (0.0, 0.0, 1.0), 0.75


def table2():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        n, e, vi, r = line.split()
        rows[int(n)] = (float(e), float(vi), float(r))
    return rows


def _guess_b(N):
    """(x + i y) times the unit-width Gaussian, normalised (guess (b))."""
    x, y, z = W.mesh(N, L)
    f = (x + 1j * y) * np.exp(-(x * x + y * y + z * z) / 2) * np.ones((N[2], N[1], N[0]))
    h3 = np.prod([2 * L[a] / N[a] for a in range(3)])
    return f / math.sqrt(h3 * np.sum(np.abs(f) ** 2))


def _mg(lib, levels, psi0, max_iter, precision):
    grids = [(m, m, m) for m in levels]
    plans = [lib.Plan(N, L, NAX, f32=precision != lib.PRECISION_F64) for N in grids]
    psis = [torch.from_numpy(np.ascontiguousarray(psi0)).cuda()] + \
           [torch.empty(p.shape, dtype=torch.complex128, device="cuda") for p in plans[1:]]
    res = lib.pcg_ground_state_mg(plans, lib.make_params(GAMMA, BETA, LAM, OM), psis, tol_residual=1e-9,
                                  max_iter=max_iter, precision=precision)
    for p in plans:
        p.close()
    return res


def test_table2_u_shape_energy_256(lib):
    E_paper, _, _ = table2()[256]
    res = _mg(lib, (64, 128, 256), W.guess_phi_d((64, 64, 64), L, GAMMA, OM), 30000, lib.PRECISION_F64)
    fine = res[-1]
    assert fine["status_name"] == "OK" and fine["residual"] <= 1e-9
    assert abs(fine["E"] - E_paper) <= 1e-12, fine["E"]
    assert abs(fine["virial"]) <= 1e-10


def test_table2_s_shape_energy_128(lib):
    E_paper, I_paper, _ = table2()[128]
    res = _mg(lib, (64, 128), _guess_b((64, 64, 64)), 30000, lib.PRECISION_F32_SPLIT)
    r = res[-1]
    assert r["status_name"] == "OK"
    assert abs(r["E"] - E_paper) <= 5e-10, r["E"]
    assert abs(abs(r["virial"]) - I_paper) <= 1e-2 * I_paper, r["virial"]
