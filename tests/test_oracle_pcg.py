"""Pins of the oracle's Algorithm 1 (PCG-ATKM): closed-form ground states,
invariants along the iteration, and planted mistakes that the pins catch."""
import math

import numpy as np
import pytest

import atkm_workloads as W
import oracle as O
import oracle.atkm_oracle as OM  # the module whose globals the oracle uses


def test_harmonic_oscillator_ground_state():
    """beta = lambda = Omega = 0: E = mu = (gamma_x + gamma_y + gamma_z)/2."""
    N, L = (32, 32, 32), (8.0, 8.0, 4.0)
    plan = O.Plan(N, L, (0, 0, 1))
    prm = O.Params((1.0, 1.0, 4.0), 0.0, 0.0, 0.0)
    phi0 = W.random_smooth_field(N, L, (0.8, 0.9, 3.0), seed=7)
    res = O.pcg_ground_state(plan, prm, phi0, O.PcgOptions(tol_residual=1e-10, max_iter=500))
    assert res.status == O.OK
    assert abs(res.parts["E"] - 3.0) < 1e-10
    assert abs(res.mu - 3.0) < 1e-10


@pytest.fixture(scope="module")
def cfg1_run():
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = O.Plan(w.N, w.L, w.n)
    prm = O.Params(w.gamma, w.beta, w.lam, w.Omega)
    res = O.pcg_ground_state(plan, prm, W.initial_guess(w), O.PcgOptions(max_iter=400))
    return plan, prm, res


def test_cfg1_converges(cfg1_run):
    plan, prm, res = cfg1_run
    assert res.status == O.OK
    assert res.residual <= 1e-8
    assert abs(O.norm(res.phi, plan.grid) - 1.0) < 1e-14


def test_cfg1_energy_monotone(cfg1_run):
    _, _, res = cfg1_run
    Es = [e["E"] for e in res.log]
    for a, b in zip(Es, Es[1:]):
        assert b <= a + 32 * O.EPS * abs(a)


def test_cfg1_mu_energy_identity_and_virial_parts(cfg1_run):
    plan, prm, res = cfg1_run
    p = res.parts
    assert abs(res.mu - (p["E"] + p["E_int"] + p["E_dip"])) < 1e-13 * abs(res.mu)
    assert abs(sum(p[k] for k in ("E_kin", "E_pot", "E_int", "E_dip", "E_rot")) - p["E"]) < 1e-14 * p["E"]


def test_converged_state_solves_euler_lagrange(cfg1_run):
    plan, prm, res = cfg1_run
    g = plan.grid
    Hphi = O.apply_H(plan, prm, res.phi, res.phi, res.Phi)
    assert O.norm(Hphi - res.mu * res.phi, g) <= 1.0000001e-8


def test_energy_independent_of_Omega_below_critical():
    """Isotropic xy trap, Omega below the critical value: the ground state is
    vortex-free and E does not depend on Omega (§3, Example 3.7)."""
    N, L = (24, 24, 12), (6.0, 6.0, 2.0)
    plan = O.Plan(N, L, (0, 0, 1))
    Es = []
    for Om in (0.0, 0.1, 0.2):
        prm = O.Params((1.0, 1.0, 4.0), 10.0, 3.0, Om)
        phi0 = W.guess_phi_d(N, L, (1.0, 1.0, 4.0), 0.0)
        res = O.pcg_ground_state(plan, prm, phi0, O.PcgOptions(tol_residual=1e-10, max_iter=500))
        assert res.status == O.OK
        Es.append(res.parts["E"])
    assert max(Es) - min(Es) < 1e-11


def test_virial_identity_resolved():
    """At a stationary state on a resolved grid, I = 2Ekin - 2Epot + 3Eint + 3Edip ~ 0."""
    N, L = (32, 32, 32), (7.0, 7.0, 7.0)
    plan = O.Plan(N, L, (0, 0, 1))
    prm = O.Params((1.0, 1.0, 1.0), 20.0, 8.0, 0.3)
    phi0 = W.guess_phi_d(N, L, (1.0, 1.0, 1.0), 0.3)
    res = O.pcg_ground_state(plan, prm, phi0, O.PcgOptions(tol_residual=1e-10, max_iter=500))
    assert res.status == O.OK
    assert abs(res.parts["virial"]) < 1e-6


def test_max_iter_gives_not_converged():
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = O.Plan(w.N, w.L, w.n)
    prm = O.Params(w.gamma, w.beta, w.lam, w.Omega)
    res = O.pcg_ground_state(plan, prm, W.initial_guess(w), O.PcgOptions(max_iter=2))
    assert res.status == O.NOT_CONVERGED and res.iters == 2


# --------------------------------------------------------- planted mistakes
# Each test plants one plausible mistake in the oracle (on the CPU, through
# monkeypatch) and checks that one of the pins above then fails.
def test_planted_sign_error_in_Lz_is_caught(monkeypatch):
    def bad_Lz(f, g):
        return 1j * (g.x * O.d_dy(f, g) - g.y * O.d_dx(f, g))
    monkeypatch.setattr(OM, "L_z", bad_Lz)
    N, L = (64, 64, 16), (8.0, 8.0, 2.0)
    g = O.Grid(N, L)
    f = (g.x + 1j * g.y) * W.gaussian_G(N, L, (1.0, 1.0, 4.0))
    assert np.max(np.abs(OM.L_z(f, g) - f)) > 0.1 * np.max(np.abs(f))


def test_planted_missing_delta_term_is_caught():
    """Dropping the -rho of Eq. (DDI2Cou3D) breaks the zero-trace identity."""
    N, L = (24, 24, 12), (6.0, 6.0, 1.5)
    U0 = O.truncated_coulomb_fourier(N, L)
    rho = np.real(W.random_smooth_field(N, L, (1.3, 1.0, 9.0), seed=3, complex_valued=False)) ** 2
    tot = 0
    for e in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        K = O.dipolar_multiplier(N, L, e, U0) + 1.0   # planted: no -1
        tot = tot + O.truncated_convolution(rho, K)
    assert np.max(np.abs(tot)) > 0.1 * np.max(rho)


def test_planted_transposed_axes_in_multiplier_is_caught():
    """Swapping the x and z box lengths in U0 breaks the closed form at k=0
    for an anisotropic box only if the swap changes the box -- use a box that
    is not symmetric and check against the Gaussian closed form."""
    N, L = (64, 64, 64), (8.0, 8.0, 1.6)
    sigma = (1.0, 1.0, 0.2)
    n = (0.0, 0.0, 1.0)
    good = O.dipolar_multiplier(N, L, n)
    bad_U0 = np.transpose(O.truncated_coulomb_fourier(N, L), (2, 1, 0))  # planted
    bad = O.dipolar_multiplier(N, L, n, bad_U0)
    rho = W.gaussian_density(N, L, sigma)
    a = O.truncated_convolution(rho, good)
    b = O.truncated_convolution(rho, bad)
    assert np.max(np.abs(a - b)) > 1e-3 * np.max(np.abs(a))


def test_planted_wrong_preconditioner_exponent_breaks_spd_plane_wave(monkeypatch):
    plan = O.Plan((16, 12, 8), (4.0, 3.0, 1.5), (0, 0, 1))
    g = plan.grid
    prm0 = O.Params((0.0, 0.0, 0.0), 0.0, 0.0, 0.0)
    phi = np.ones(g.shape, dtype=np.complex128)
    Phi = np.zeros(g.shape)
    orig = O.spectral_apply

    def bad(f, mult):
        return orig(f, mult ** 2)   # planted: squared P_Delta
    monkeypatch.setattr(OM, "spectral_apply", bad)
    nux = math.pi * 2 / g.L[0]
    f = np.broadcast_to(np.exp(1j * nux * (g.x + g.L[0])), g.shape).astype(np.complex128)
    a = 1.7
    Pf = OM.apply_precond(plan, prm0, f, phi, Phi, a)
    assert np.max(np.abs(Pf - f / (a * (a + 0.5 * nux ** 2)))) > 1e-3
