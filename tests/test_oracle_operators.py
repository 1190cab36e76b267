"""Pins of the oracle's spectral operators, energy and preconditioner (§2.1, §2.3)."""
import math

import numpy as np
import pytest

import atkm_workloads as W
import oracle as O


def test_spectral_derivatives_exact_on_trig_polynomials():
    N, L = (12, 10, 8), (2.0, 1.5, 1.0)
    g = O.Grid(N, L)
    # band-limited: |k| < N/2 on each axis, phase e^{i nu (x + L)}
    kx, ky, kz = 3, -2, 1
    nux, nuy, nuz = math.pi * kx / L[0], math.pi * ky / L[1], math.pi * kz / L[2]
    f = np.exp(1j * (nux * (g.x + L[0]) + nuy * (g.y + L[1]) + nuz * (g.z + L[2])))
    f = np.broadcast_to(f, g.shape).copy()
    assert np.max(np.abs(O.d_dx(f, g) - 1j * nux * f)) < 1e-12
    assert np.max(np.abs(O.d_dy(f, g) - 1j * nuy * f)) < 1e-12
    assert np.max(np.abs(O.laplacian(f, g) + (nux ** 2 + nuy ** 2 + nuz ** 2) * f)) < 1e-11
    # real cosine in x: d_x cos = -nu sin
    c = np.broadcast_to(np.cos(nux * (g.x + L[0])), g.shape).astype(np.complex128)
    assert np.max(np.abs(O.d_dx(c, g) + nux * np.sin(nux * (g.x + L[0])))) < 1e-12


def test_Lz_of_vortex_gaussian_is_itself():
    """L_z[(x+iy) G] = (x+iy) G for a Gaussian isotropic in the xy plane."""
    N, L = (64, 64, 16), (8.0, 8.0, 2.0)
    g = O.Grid(N, L)
    G = W.gaussian_G(N, L, (1.0, 1.0, 4.0))
    f = (g.x + 1j * g.y) * G
    assert np.max(np.abs(O.L_z(f, g) - f)) < 1e-10 * np.max(np.abs(f))
    # and L_z G = 0 (no angular momentum)
    assert np.max(np.abs(O.L_z(G.astype(np.complex128), g))) < 1e-10


def _setup(N=(16, 12, 8), L=(4.0, 3.0, 1.5), n=(0.6, 0.0, 0.8)):
    plan = O.Plan(N, L, n)
    prm = O.Params((1.0, 1.3, 6.0), 40.0, -12.0, 0.55)
    phi = W.random_smooth_field(N, L, (1.0, 1.3, 6.0), seed=21)
    phi = phi / O.norm(phi, plan.grid)
    Phi = plan.dipolar_potential(np.abs(phi) ** 2)
    return plan, prm, phi, Phi


def test_H_is_hermitian():
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    u = W.random_field(g.shape, 31)
    v = W.random_field(g.shape, 32)
    a = O.inner(O.apply_H(plan, prm, u, phi, Phi), v, g)
    b = O.inner(u, O.apply_H(plan, prm, v, phi, Phi), g)
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_energy_invariant_under_global_phase():
    plan, prm, phi, Phi = _setup()
    e1 = O.energy(plan, prm, phi, Phi)
    e2 = O.energy(plan, prm, np.exp(0.7j) * phi, Phi)
    assert abs(e1 - e2) < 1e-13 * abs(e1)


def test_mu_energy_identity():
    """mu = <H phi, phi> = E + int beta/2 |phi|^4 + lambda/2 Phi |phi|^2 (§1)."""
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    mu = O.inner(O.apply_H(plan, prm, phi, phi, Phi), phi, g)
    p = O.energy_parts(plan, prm, phi, Phi)
    assert abs(mu - (p["E"] + p["E_int"] + p["E_dip"])) < 1e-13 * abs(mu)


def test_energy_gradient_matches_finite_difference():
    """grad E = 2 H_phi phi (§2.3): directional derivative by central differences."""
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    d = W.random_smooth_field(plan.grid.N, plan.grid.L, (1.2, 1.0, 5.0), seed=41)
    eps = 1e-5

    def E(f):
        return O.energy(plan, prm, f, plan.dipolar_potential(np.abs(f) ** 2))

    fd = (E(phi + eps * d) - E(phi - eps * d)) / (2 * eps)
    an = 2 * O.inner(O.apply_H(plan, prm, phi, phi, Phi), d, g)
    assert abs(fd - an) < 1e-7 * abs(an)


def test_quadratic_model_second_variation():
    """d^2/dt^2 E(phi + t p) at 0 = 2(<H p, p> + <g, p>), g = 2 phi (beta rho' + lambda U_dip*rho'),
    rho' = Re(conj(phi) p): pins the reading of the kernel in Eq. (Energy_Expend)."""
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    p = W.random_smooth_field(g.N, g.L, (1.2, 1.0, 5.0), seed=42)

    def E(f):
        return O.energy(plan, prm, f, plan.dipolar_potential(np.abs(f) ** 2))

    eps = 1e-3
    fd2 = (E(phi + eps * p) - 2 * E(phi) + E(phi - eps * p)) / eps ** 2
    rho1 = np.real(np.conj(phi) * p)
    gn = 2 * phi * (prm.beta * rho1 + prm.lam * plan.dipolar_potential(rho1))
    an = 2 * (O.inner(O.apply_H(plan, prm, p, phi, Phi), p, g) + O.inner(gn, p, g))
    assert abs(fd2 - an) < 1e-6 * abs(an)


def test_projection_is_tangent_and_idempotent():
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    f = W.random_field(g.shape, 51)
    Jf = O.project(f, phi, g)
    assert abs(O.inner(Jf, phi, g)) < 1e-14 * O.norm(f, g)
    assert np.max(np.abs(O.project(Jf, phi, g) - Jf)) < 1e-14 * np.max(np.abs(f))


def test_preconditioner_spd_and_plane_wave():
    plan, prm, phi, Phi = _setup()
    g = plan.grid
    alpha = O.precond_shift(plan, prm, phi, Phi)
    assert alpha > 0
    u = W.random_field(g.shape, 61)
    v = W.random_field(g.shape, 62)
    Pu = O.apply_precond(plan, prm, u, phi, Phi, alpha)
    Pv = O.apply_precond(plan, prm, v, phi, Phi, alpha)
    assert abs(O.inner(Pu, v, g) - O.inner(u, Pv, g)) < 1e-13 * O.norm(Pu, g) * O.norm(v, g)
    assert O.inner(Pu, u, g) > 0
    # with V = 0 and no interactions P_V = 1/alpha: P e^{i nu x} = e^{i nu x} / (alpha (alpha + nu^2/2))
    prm0 = O.Params((0.0, 0.0, 0.0), 0.0, 0.0, 0.0)
    nux = math.pi * 2 / g.L[0]
    f = np.broadcast_to(np.exp(1j * nux * (g.x + g.L[0])), g.shape).astype(np.complex128)
    a = 1.7
    Pf = O.apply_precond(plan, prm0, f, phi, Phi, a)
    assert np.max(np.abs(Pf - f / (a * (a + 0.5 * nux ** 2)))) < 1e-13


def test_preconditioner_shift_definition():
    """alpha = E_kin + E_pot + 2 E_int + |2 E_dip| in terms of the energy parts."""
    plan, prm, phi, Phi = _setup()
    p = O.energy_parts(plan, prm, phi, Phi)
    alpha = O.precond_shift(plan, prm, phi, Phi)
    assert abs(alpha - (p["E_kin"] + p["E_pot"] + 2 * p["E_int"] + abs(2 * p["E_dip"]))) < 1e-13 * alpha
