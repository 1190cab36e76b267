"""The seeded synthetic inputs (atkm_workloads): the counter-based generator
against its published outputs, the sweep and learned-guess draws against the
recipes they state, and the paper's initial guesses of §3 against properties
fixed by their definitions (unit discrete norm, conjugate pairs, the
Thomas-Fermi profile's mass and support)."""
import math

import numpy as np
import pytest

import atkm_workloads as W


def _norm2(f, N, L):
    h3 = np.prod([2.0 * L[a] / N[a] for a in range(3)])
    return float(np.sum(np.abs(f) ** 2) * h3)


def test_splitmix64_published_outputs():
    # The first outputs of SplitMix64 (Steele, Lea and Flood; Vigna's
    # splitmix64.c) from the state 1234567.
    g = W.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]
    g = W.SplitMix64(1234567)
    assert g.uniform() == (6457827717110365317 >> 11) / 2.0 ** 53


def test_vortex_positions_in_disc_and_seeded():
    p = W.vortex_positions(500, 4.0, 1)
    r = np.hypot(*np.array(p).T)
    assert len(p) == 500 and r.max() <= 4.0
    # area-uniform: the fraction inside radius 2 is 1/4
    assert abs(np.mean(r < 2.0) - 0.25) < 0.06
    assert W.vortex_positions(8, 4.0, 1) == W.vortex_positions(8, 4.0, 1)
    assert W.vortex_positions(8, 4.0, 1) != W.vortex_positions(8, 4.0, 2)


def test_sweep_instances_follow_their_recipe():
    inst = W.sweep_instances()
    assert len(inst) == 48
    for w in inst:
        e = w.N[0]
        assert w.N == (e, e, e // 4) and e in (64, 72, 80, 96, 120, 128, 144, 160, 192)
        assert 0.5 <= w.Omega <= 0.95
        assert w.gamma[:2] == (1.0, 1.0) and w.gamma[2] in (10.0, 20.0, 40.0)
        assert w.beta == 200.0 and w.lam / w.beta in (0.2, 0.4)
        assert w.n == (0.0, 0.0, 1.0)
        assert w.L[:2] == (16.0, 16.0) and w.L[2] == pytest.approx(math.sqrt(64.0 / w.gamma[2]))
    assert len({w.N for w in inst}) > 4  # uneven grids


def test_guess_draws_follow_their_recipe():
    draws = W.guess_draws(200)
    for w in draws:
        assert w.N == W.GUESS_COARSE_N
        assert 0.3 <= w.Omega <= 0.95 and 5.0 <= w.gamma[2] <= 50.0 and 100.0 <= w.beta <= 1000.0
        assert 0.0 <= w.lam / w.beta <= 0.45
        th = math.atan2(w.n[0], w.n[2])
        assert 0.0 <= th <= math.radians(60.0) + 1e-15 and w.n[1] == 0.0
        assert math.hypot(w.n[0], w.n[2]) == pytest.approx(1.0)
        assert w.L[2] == pytest.approx(math.sqrt(64.0 / w.gamma[2]))
    fine = W.with_grid(draws[0], W.GUESS_FINE_N)
    assert fine.L == draws[0].L and fine.N == W.GUESS_FINE_N


@pytest.mark.parametrize("name", sorted(W.CONFIGS))
def test_initial_guesses_have_unit_norm(name):
    w = W.CONFIGS[name]
    psi = W.initial_guess(w)
    assert psi.shape == w.shape and psi.dtype == np.complex128
    assert _norm2(psi, w.N, w.L) == pytest.approx(1.0, abs=1e-12)


def test_paper_guesses_definitions():
    N, L, gamma, beta, Om = (32, 32, 32), (8.0, 4.0, 1.0), (1.0, 2.0, 10.0), 100.0, 0.4
    g = W.paper_guesses(N, L, gamma, beta, Om)
    assert tuple(g) == W.PAPER_GUESS_NAMES
    for k, f in g.items():
        assert f.shape == (N[2], N[1], N[0])
        assert _norm2(f, N, L) == pytest.approx(1.0, abs=1e-12), k
    for k in ("b", "c", "d", "e"):
        assert np.array_equal(g[k + "bar"], np.conj(g[k]))
    # (d) is proportional to (1 - Omega) a + Omega b
    d = (1 - Om) * g["a"] + Om * g["b"]
    c = np.vdot(d, g["d"]) / np.vdot(d, d)
    assert np.abs(g["d"] - c * d).max() <= 1e-12 * np.abs(g["d"]).max()


def test_thomas_fermi_guess_mass_and_support():
    # mu_TF is the chemical potential at which the Thomas-Fermi profile of the
    # trap V = (gamma_x^2 x^2 + gamma_y^2 y^2 + gamma_z^2 z^2)/2 carries unit
    # mass: int (mu_TF - V)_+ / beta = 1.  So the normalised guess (f) has
    # |f(0)|^2 = mu_TF / beta up to the grid's quadrature error, and it
    # vanishes where V >= mu_TF, e.g. beyond sqrt(2 mu_TF) / gamma_a on axis a.
    gamma, beta = (1.0, 2.0, 10.0), 100.0
    mu = 0.5 * (15.0 * beta * gamma[0] * gamma[1] * gamma[2] / (4.0 * math.pi)) ** 0.4
    N, L = (64, 64, 64), (8.0, 4.0, 1.0)
    f = W.paper_guesses(N, L, gamma, beta, 0.5)["f"]
    c = (N[2] // 2, N[1] // 2, N[0] // 2)  # the grid point at the origin
    x, y, z = (W.axis_coords(N[a], L[a]) for a in range(3))
    assert x[c[2]] == 0.0 and y[c[1]] == 0.0 and z[c[0]] == 0.0
    assert abs(f[c]) ** 2 * beta / mu == pytest.approx(1.0, abs=1e-3)
    for a, coord in enumerate((x, y, z)):
        R = math.sqrt(2.0 * mu) / gamma[a]
        inside = np.flatnonzero(np.abs(coord) < 0.98 * R)
        outside = np.flatnonzero(np.abs(coord) > 1.02 * R)
        idx = list(c)
        for j, want_zero in ((inside, False), (outside, True)):
            for i in j:
                idx[2 - a] = i
                assert (f[tuple(idx)] == 0.0) == want_zero, (a, i)
