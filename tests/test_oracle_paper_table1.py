"""Pins of the oracle against values the paper prints: the virial-identity
residual |I| of the discrete ground state in Example 3.1 (Table 1;
tests/golden/table1_example31.txt).  |I| on an under-resolved grid is a
discretisation-error measure, so it checks the whole discrete operator
(spectral kinetic and rotation terms, trap, contact term, ATKM with the
truncated kernel) and the converged state together.

Observed agreement: 2.6e-4 relative at 32^3 (Case I, three Omegas), 2.2e-3
at 64^3 (5.5e-8 absolute) and 2.3e-3 for Case II at 32^3; the remaining
difference is systematic and not explained (the paper does not state how
accurately it evaluates the truncated-kernel coefficients).  Tolerances:
5e-4 (Case I, 32^3) and 5e-3 (the others); a dropped term or a wrong
factor moves |I| by O(1)."""
import math
import os

import numpy as np
import pytest

import atkm_workloads as W
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_example31.txt")


def table1():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        case, om, n, e2, vi = line.split()
        rows[(case, float(om), int(n))] = (float(e2), float(vi))
    return rows


def setup(case):
    if case == "I":
        return (1.0, 1.0, 1.0), (16.0, 16.0, 16.0)
    return (1.0, 2.0, 10.0), (16.0, 16.0, 10.0)


def ground_state(case, Om, N, guess="d"):
    gamma, L = setup(case)
    NN = (N, N, N)
    plan = O.Plan(NN, L, (0.0, 0.0, 1.0))
    prm = O.Params(gamma, 100.0, 80.0, Om)
    if guess == "d":
        psi0 = W.guess_phi_d(NN, L, gamma, Om)
    else:  # (a): the normalised Gaussian of unit width
        x, y, z = W.mesh(NN, L)
        psi0 = np.exp(-(x * x + y * y + z * z) / 2).astype(np.complex128) * np.ones((N, N, N))
    r = O.pcg_ground_state(plan, prm, psi0, O.PcgOptions(tol_residual=1e-10, max_iter=3000))
    assert r.status == O.OK
    return r


@pytest.mark.parametrize("Om", [0.2, 0.4, 0.6])
def test_case1_virial_residual_32(Om):
    ref = table1()[("I", Om, 32)][1]
    got = abs(ground_state("I", Om, 32).parts["virial"])
    assert abs(got - ref) <= 5e-4 * ref, (got, ref)


def test_case1_virial_residual_64():
    ref = table1()[("I", 0.2, 64)][1]
    got = abs(ground_state("I", 0.2, 64).parts["virial"])
    assert abs(got - ref) <= 5e-3 * ref, (got, ref)


@pytest.mark.parametrize("Om", [0.2, 0.4])
def test_case2_virial_residual_32_lowest_energy(Om):
    """Case II at 32^3 has several stationary states; like the paper, take the
    lowest energy over initial guesses ((a) and (d) here)."""
    ref = table1()[("II", Om, 32)][1]
    best = min((ground_state("II", Om, 32, g) for g in ("a", "d")), key=lambda r: r.parts["E"])
    got = abs(best.parts["virial"])
    assert abs(got - ref) <= 5e-3 * ref, (got, ref)
