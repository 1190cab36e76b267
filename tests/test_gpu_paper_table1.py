"""The CUDA solver against values the paper prints: Example 3.1, Table 1
(tests/golden/table1_example31.txt).  For each row the cascadic multigrid
driver (Algorithm 2) solves on 32^3, 64^3, 128^3 and 256^3 (residual 1e-10,
FP64 stop test), and E2(N) = ||phi_N - kappa phi_256|| / ||phi_256|| on the
N-grid points (kappa removes the global phase) stands in for the paper's
error against its 512^3 solution (the paper's own E2 at 256^3 is 1e-11 or
below, so the reference changes nothing at the printed digits).

Observed agreement with the printed E2: 1e-3 - 3e-3 relative at 32^3 and
1e-5 - 5e-4 at 64^3 and 128^3 (the vortex rows at Omega = 0.8 included); |I| 2.6e-4 - 5.5e-3 (the largest at 128^3
in Case II, where |I| ~ 4e-6), and 2.2e-2 for Case II Omega = 0.8 at 128^3.
|I| = |2 E_kin - 2 E_pot + 3 E_int + 3 E_dip| is a cancellation: where it is
about 1e-6 of S = 2|E_kin| + 2|E_pot| + 3|E_int| + 3|E_dip|, a relative
difference d between two evaluations of the energy terms moves it by up to
d S.  The |I| of that entry does not depend on the stop rule (the same to 7
digits at residual 1e-8 ... 1e-12); its gap to the printed value, 1.3e-7, is
3.5e-9 of S, the size of a relative difference of 3e-8 in E_dip alone, and
the paper does not state the accuracy of its truncated-kernel coefficients
(ours are within 1e-13 of two independent quadratures).  So |I| is checked to
max(1e-2 |I_paper|, 1e-8 S).
Tolerances: E2 2e-3 at 64^3 and 128^3, 1e-2 at 32^3; |I| as above; on
resolved grids (Case I, 128^3 and 256^3) |I| is at round-off level in both
(paper 1.7e-11 and 1.3e-12), checked as <= 1e-10.  Not checked: the vortex
rows at 32^3 (which under-resolved state the solve lands in depends on the
guess; the paper's Case I entry there is not the lowest-energy state).
"""
import numpy as np
import pytest
import torch

import atkm_workloads as W

from tests.test_oracle_paper_table1 import setup, table1

pytestmark = pytest.mark.gpu

GRIDS = (32, 64, 128, 256)


def _gaussian_a(N, L):
    x, y, z = W.mesh(N, L)
    return np.exp(-(x * x + y * y + z * z) / 2).astype(np.complex128) * np.ones((N[2], N[1], N[0]))


@pytest.mark.parametrize("case,Om", [("I", 0.2), ("I", 0.6), ("I", 0.8), ("II", 0.2), ("II", 0.4), ("II", 0.8)])
def test_table1_errors_and_virial(lib, case, Om):
    gamma, L = setup(case)
    grids = [(n, n, n) for n in GRIDS]
    plans = [lib.Plan(N, L, (0.0, 0.0, 1.0), f32=True) for N in grids]
    prm = lib.make_params(gamma, 100.0, 80.0, Om)
    # guess (a): the lowest-energy 32^3 state of Case II at Omega = 0.4 (see
    # the oracle test); the same state as guess (d) everywhere else
    psis = [torch.from_numpy(_gaussian_a(grids[0], L)).cuda()] + \
           [torch.empty(p.shape, dtype=torch.complex128, device="cuda") for p in plans[1:]]
    res = lib.pcg_ground_state_mg(plans, prm, psis, tol_residual=1e-10, max_iter=4000,
                                  precision=lib.PRECISION_F32_SPLIT)
    assert [r["status_name"] for r in res] == ["OK"] * 4
    ref = psis[-1].cpu().numpy()
    paper = table1()
    vortex = Om == 0.8
    for n, r, p in zip(GRIDS, res, psis):
        e2_paper, vir_paper = paper[(case, Om, n)]
        if vortex and n == 32:
            continue  # the under-resolved 32^3 vortex states depend on the guess
        if n < 256:
            s = 256 // n
            ex = ref[::s, ::s, ::s]
            ph = p.cpu().numpy()
            kappa = np.vdot(ex, ph) / np.vdot(ex, ex)
            e2 = np.linalg.norm(ph - kappa * ex) / np.linalg.norm(ex)
            tol = 1e-2 if n == 32 else 2e-3
            assert abs(e2 - e2_paper) <= tol * e2_paper, (n, e2, e2_paper)
        vir = abs(r["virial"])
        S = 2 * abs(r["E_kin"]) + 2 * abs(r["E_pot"]) + 3 * abs(r["E_int"]) + 3 * abs(r["E_dip"])
        if vir_paper > 1e-9:
            assert abs(vir - vir_paper) <= max(1e-2 * vir_paper, 1e-8 * S), (n, vir, vir_paper, S)
        else:
            assert vir <= 1e-10, (n, vir)
