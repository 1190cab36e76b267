"""Pins of the C++ oracle (oracle/cpp/atkm_oracle.cpp), each independent of
its own code:
  * its FFT against the brute-force DFT (an O(n^2) matrix with exactly
    reduced arguments) on every {2,3,5}-smooth length 2 ... 384 and on a few
    lengths with larger prime factors, both signs; Parseval; the inverse of
    the forward transform; delta and plane-wave inputs; the 3D transform
    against numpy's FFT (a library routine the C++ oracle does not use);
  * its Faddeeva function against mpmath at 40 digits, and on the axes
    against closed forms (e^{-x^2} + 2i D(x)/sqrt(pi) with Dawson's D;
    erfcx on the imaginary axis);
  * U0 at k = 0 against the 8-corner closed form and at k != 0 against the
    face-decomposition quadrature (both from tests/test_oracle_kernel.py);
  * the dipolar potential of an isotropic Gaussian against its exact value;
  * the harmonic oscillator ground state E = mu = (gx + gy + gz)/2;
  * the whole method against the numpy oracle (a second, independent
    restatement with pocketfft and scipy's Faddeeva function): U0, K, Phi,
    H, the energy terms, alpha, P r, spectral interpolation, and full
    Algorithm 1 runs with the same decisions;
  * the thread count changes no bit of any result.
"""
import math

import numpy as np
import pytest
from scipy.special import dawsn, erfcx

import atkm_workloads as W
import oracle as O
import oracle.cpp_oracle as OC
from tests.test_oracle_kernel import box_inverse_distance_integral, face_decomposition_U0, iso_gaussian_dipolar


def smooth_lengths(limit):
    out = []
    for n in range(2, limit + 1):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


def brute_dft(x, sign):
    n = x.size
    j = np.arange(n)
    return np.exp(sign * 2j * math.pi * (np.outer(j, j) % n) / n) @ x


@pytest.mark.parametrize("n", smooth_lengths(384) + [7, 11, 13, 14, 21, 49, 77, 98])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = brute_dft(x, sign)
        got = OC.dft1(x, sign)
        assert np.max(np.abs(got - ref)) <= 4e-15 * np.max(np.abs(ref)), (n, sign)


@pytest.mark.parametrize("n", [2, 6, 30, 96, 120, 243, 256, 384])
def test_fft_parseval_inverse_delta_plane_wave(n):
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = OC.dft1(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) <= 1e-13 * np.sum(np.abs(x) ** 2)
    assert np.max(np.abs(OC.dft1(X, 1) / n - x)) <= 1e-14 * np.max(np.abs(x))
    d = np.zeros(n, dtype=np.complex128)
    d[0] = 1.0
    assert np.max(np.abs(OC.dft1(d, -1) - 1.0)) == 0.0
    k0 = n // 3
    wave = np.exp(2j * math.pi * k0 * np.arange(n) / n)
    spec = OC.dft1(wave, -1)
    expect = np.zeros(n)
    expect[k0] = n
    assert np.max(np.abs(spec - expect)) <= 1e-12 * n


@pytest.mark.parametrize("shape", [(4, 6, 10), (9, 8, 15), (16, 12, 20)])
def test_fft3_matches_numpy(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    f = OC.fft3(a, -1)
    assert np.max(np.abs(f - np.fft.fftn(a) / a.size)) <= 1e-15 * np.max(np.abs(a))
    assert np.max(np.abs(OC.fft3(f, 1) - a)) <= 1e-14 * np.max(np.abs(a))


def test_faddeeva_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    pts = []
    for x in (-60, -12.5, -9.2, -8.01, -7.99, -3.3, -0.7, 0.0, 0.4, 2.2, 5.3, 7.9, 8.1, 15, 40):
        for y in (1e-12, 1e-6, 1e-3, 0.05, 0.26, 0.9, 2.0, 5.0, 7.9, 8.2, 30.0):
            pts.append(complex(x, y))
    z = np.array(pts)
    got = OC.faddeeva(z)
    for zz, g in zip(pts, got):
        ex = complex(mp.exp(-mp.mpc(zz) ** 2) * mp.erfc(-1j * mp.mpc(zz)))
        assert abs(g - ex) <= 2e-15 * abs(ex), (zz, g, ex)


def test_faddeeva_on_the_axes():
    x = np.linspace(-7.5, 7.5, 301)
    got = OC.faddeeva(x + 1e-300j)  # limit onto the real axis from above
    assert np.max(np.abs(got.real - np.exp(-x * x))) <= 2e-15
    assert np.max(np.abs(got.imag - 2 * dawsn(x) / math.sqrt(math.pi))) <= 2e-15
    y = np.linspace(0.01, 50, 200)
    got = OC.faddeeva(1j * y)
    assert np.max(np.abs(got.real - erfcx(y)) / erfcx(y)) <= 2e-15
    assert np.max(np.abs(got.imag) / erfcx(y)) <= 1e-16  # zero up to rounding


@pytest.mark.parametrize("N,L", [((8, 8, 4), (1.0, 1.0, 0.5)), ((32, 32, 16), (8.0, 8.0, 2.0)),
                                 ((12, 10, 6), (3.0, 2.5, 0.4)), ((256, 256, 64), (16.0, 16.0, 1.5))])
def test_U0_at_zero_frequency_closed_form(N, L):
    U0 = OC.Plan(N, L, (0, 0, 1), threads=4).U0()
    ref = box_inverse_distance_integral(*[2 * v for v in L]) / (4 * math.pi)
    assert abs(U0[0, 0, 0] - ref) <= 2e-14 * ref


def test_U0_nonzero_frequencies_vs_face_decomposition():
    N, L = (6, 8, 4), (1.0, 0.75, 0.35)
    U0 = OC.Plan(N, L, (0, 0, 1)).U0()
    a = [2 * v for v in L]
    worst = 0.0
    for k in [(1, 0, 0), (0, 2, 0), (0, 0, 1), (1, 2, 1), (3, 1, 2), (6, 8, 4), (2, 5, 3)]:
        nu = [math.pi * k[i] / a[i] for i in range(3)]
        worst = max(worst, abs(U0[k[2], k[1], k[0]] - face_decomposition_U0(nu, a)) / U0[0, 0, 0])
    assert worst < 1e-12


@pytest.mark.parametrize("n", [(0.0, 0.0, 1.0), (math.sin(math.radians(30)), 0.0, math.cos(math.radians(30)))])
def test_dipolar_potential_of_isotropic_gaussian(n):
    N, L = (64, 64, 64), (8.0, 8.0, 8.0)
    rho, _, Phi = iso_gaussian_dipolar(N, L, n)
    got = OC.Plan(N, L, n, threads=8).dipolar_potential(rho)
    assert np.max(np.abs(got - Phi)) <= 1e-12 * np.max(np.abs(Phi))


def test_harmonic_oscillator_ground_state():
    N, L = (32, 32, 32), (8.0, 8.0, 4.0)
    plan = OC.Plan(N, L, (0, 0, 1), threads=8)
    prm = O.Params((1.0, 1.0, 4.0), 0.0, 0.0, 0.0)
    psi0 = W.random_smooth_field(N, L, (0.8, 0.9, 3.0), seed=7)
    r = plan.pcg_ground_state(prm, psi0, OC.PcgOptions(tol_residual=1e-10, max_iter=500))
    assert r.status == OC.OK
    assert abs(r.parts["E"] - 3.0) < 1e-10 and abs(r.mu - 3.0) < 1e-10


CASES = [
    ((32, 32, 16), (8.0, 8.0, 2.0), (0.0, 0.0, 1.0)),
    ((24, 20, 12), (5.0, 4.0, 1.2), (0.6, 0.0, 0.8)),
    ((40, 36, 10), (6.0, 5.5, 1.0), (0.5, 0.5, math.sqrt(0.5))),
    ((6, 4, 2), (1.0, 0.8, 0.5), (1.0, 0.0, 0.0)),
]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("N,L,n", CASES)
def test_operators_match_numpy_oracle(N, L, n):
    cp = OC.Plan(N, L, n, threads=4)
    op = O.Plan(N, L, n)
    assert np.max(np.abs(cp.U0() - op.U0)) <= 1e-13 * np.max(np.abs(op.U0))
    assert np.max(np.abs(cp.K() - op.K)) <= 1e-12
    prm = O.Params((1.0, 1.3, 6.0), 40.0, -12.0, 0.55)
    psi = W.random_smooth_field(N, L, (1.0, 1.1, 5.0), seed=3)
    rho = np.abs(psi) ** 2
    Phi = op.dipolar_potential(rho)
    assert rel(cp.dipolar_potential(rho), Phi) <= 1e-13
    white = W.random_field(op.grid.shape, 11, complex_valued=False)
    assert rel(cp.dipolar_potential(white), op.dipolar_potential(white)) <= 1e-13
    f = W.random_field(op.grid.shape, 4)
    assert rel(cp.apply_H(prm, f, psi, Phi), O.apply_H(op, prm, f, psi, Phi)) <= 1e-13
    e1, e2 = cp.energy_parts(prm, psi, Phi), O.energy_parts(op, prm, psi, Phi)
    for k in e2:
        assert abs(e1[k] - e2[k]) <= 1e-13 * (abs(e2["E"]) + abs(e2["E_kin"])), k
    a1, a2 = cp.precond_shift(prm, psi, Phi), O.precond_shift(op, prm, psi, Phi)
    assert abs(a1 - a2) <= 1e-13 * a2
    assert rel(cp.apply_precond(prm, f, psi, Phi, a2), O.apply_precond(op, prm, f, psi, Phi, a2)) <= 1e-13


def test_spectral_upsample_matches_numpy_oracle():
    c = W.random_field((6, 8, 10), 21)
    for Nf in ((10, 8, 6), (20, 16, 12), (30, 24, 18)):
        assert np.max(np.abs(OC.spectral_upsample(c, Nf) - O.spectral_upsample(c, Nf))) <= 1e-13


@pytest.mark.parametrize("name,max_iter", [("cfg1_32x32x16", 400)])
def test_pcg_run_matches_numpy_oracle(name, max_iter):
    w = W.CONFIGS[name]
    prm = O.Params(w.gamma, w.beta, w.lam, w.Omega)
    psi0 = W.initial_guess(w)
    r1 = OC.Plan(w.N, w.L, w.n, threads=4).pcg_ground_state(prm, psi0, OC.PcgOptions(max_iter=max_iter))
    r2 = O.pcg_ground_state(O.Plan(w.N, w.L, w.n), prm, psi0, O.PcgOptions(max_iter=max_iter))
    assert r1.status == r2.status == O.OK and r1.iters == r2.iters
    assert abs(r1.parts["E"] - r2.parts["E"]) <= 1e-12 * abs(r2.parts["E"])
    assert abs(r1.mu - r2.mu) <= 1e-12 * abs(r2.mu)
    for a, b in zip(r1.log, r2.log):
        assert abs(a["E"] - b["E"]) <= 1e-12 * abs(b["E"])
        if "halvings" in b:
            assert a["halvings"] == b["halvings"] and a["reset"] == b["reset"] and a["accepted"] == b["accepted"]


def test_tilted_anisotropic_pcg_matches_numpy_oracle():
    N, L, n = (24, 20, 12), (5.0, 4.0, 1.2), (0.6, 0.0, 0.8)
    prm = O.Params((1.0, 1.3, 6.0), 40.0, -12.0, 0.3)
    psi0 = W.guess_phi_d(N, L, prm.gamma, prm.Omega)
    opts = dict(tol_residual=1e-9, max_iter=600)
    r1 = OC.Plan(N, L, n).pcg_ground_state(prm, psi0, OC.PcgOptions(**opts))
    r2 = O.pcg_ground_state(O.Plan(N, L, n), prm, psi0, O.PcgOptions(**opts))
    assert r1.status == r2.status == O.OK and r1.iters == r2.iters
    assert abs(r1.parts["E"] - r2.parts["E"]) <= 1e-12 * abs(r2.parts["E"])
    assert rel(r1.phi, r2.phi) <= 1e-9


def test_thread_count_changes_no_bit():
    N, L, n = (24, 20, 12), (5.0, 4.0, 1.2), (0.6, 0.0, 0.8)
    prm = O.Params((1.0, 1.3, 6.0), 40.0, -12.0, 0.3)
    psi0 = W.guess_phi_d(N, L, prm.gamma, prm.Omega)
    outs = []
    for th in (1, 3, 8):
        plan = OC.Plan(N, L, n, threads=th)
        r = plan.pcg_ground_state(prm, psi0, OC.PcgOptions(max_iter=15))
        outs.append((plan.U0(), plan.dipolar_potential(np.abs(psi0) ** 2), r.phi, [e["E"] for e in r.log]))
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(np.asarray(a), np.asarray(b))


def test_plan_rejects_bad_arguments():
    with pytest.raises(ValueError):
        OC.Plan((31, 32, 16), (8, 8, 2), (0, 0, 1))
    with pytest.raises(ValueError):
        OC.Plan((32, 32, 16), (8, 8, 2), (0, 0, 1.001))
