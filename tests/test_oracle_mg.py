"""Pins of the oracle's cascadic multigrid driver (Algorithm 2): the coarse
levels only change the starting point, so the finest level must reach the
same ground state as a single-level solve, in fewer fine-grid iterations."""
import numpy as np

import atkm_workloads as W
import oracle as O


def test_mg_reaches_the_single_level_ground_state_faster():
    L, gamma, n = (8.0, 8.0, 2.0), (1.0, 1.0, 4.0), (0.0, 0.0, 1.0)
    prm = O.Params(gamma, 50.0, 15.0, 0.4)
    grids = [(8, 8, 4), (16, 16, 8), (32, 32, 16)]
    plans = [O.Plan(N, L, n) for N in grids]
    opts = O.PcgOptions(tol_residual=1e-9, max_iter=400)
    mg = O.pcg_ground_state_mg(plans, prm, W.guess_phi_d(grids[0], L, gamma, 0.4), opts)
    single = O.pcg_ground_state(plans[-1], prm, W.guess_phi_d(grids[-1], L, gamma, 0.4), opts)
    assert all(r.status == O.OK for r in mg) and single.status == O.OK
    E = [r.parts["E"] for r in (mg[-1], single)]
    assert abs(E[0] - E[1]) <= 1e-10 * abs(E[1])
    # the same state up to a global phase
    g = plans[-1].grid
    ov = abs(O.inner(mg[-1].phi, single.phi, g) + 1j * O.inner(mg[-1].phi, 1j * single.phi, g))
    assert abs(ov - 1.0) < 1e-8
    assert mg[-1].iters < single.iters


def test_mg_levels_of_the_harmonic_oscillator():
    """beta = lambda = Omega = 0: E = (gx+gy+gz)/2 on the resolved finest
    level (h = 0.3), within the discretisation error on the coarse one."""
    L, gamma, n = (6.0, 6.0, 4.5), (1.0, 1.5, 2.0), (0.0, 0.0, 1.0)
    prm = O.Params(gamma, 0.0, 0.0, 0.0)
    plans = [O.Plan(N, L, n) for N in [(20, 20, 16), (40, 40, 30)]]
    opts = O.PcgOptions(tol_residual=1e-10, max_iter=300)
    mg = O.pcg_ground_state_mg(plans, prm, W.guess_phi_d((20, 20, 16), L, gamma, 0.0), opts)
    assert all(r.status == O.OK for r in mg)
    assert abs(mg[0].parts["E"] - 0.5 * sum(gamma)) < 1e-2
    assert abs(mg[1].parts["E"] - 0.5 * sum(gamma)) < 1e-10
