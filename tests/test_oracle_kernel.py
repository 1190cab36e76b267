"""Pins of the oracle's truncated-kernel coefficients and ATKM apply (§2.2).

Each test checks the oracle against something other than itself: a closed
form, an independent quadrature, an exact identity of the continuous problem,
or a brute-force sum.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.special import erf, roots_legendre
from scipy import integrate

import atkm_workloads as W
import oracle as O


# ---------------------------------------------------------------- closed forms
def _corner_F(x, y, z):
    """Antiderivative of 1/|y| over [0,x]x[0,y]x[0,z] (zero-face limits taken)."""
    r = math.sqrt(x * x + y * y + z * z)
    t = 0.0
    if y * z:
        t += y * z * math.log(x + r)
    if x * z:
        t += x * z * math.log(y + r)
    if x * y:
        t += x * y * math.log(z + r)
    if x:
        t -= 0.5 * x * x * math.atan(y * z / (x * r))
    if y:
        t -= 0.5 * y * y * math.atan(x * z / (y * r))
    if z:
        t -= 0.5 * z * z * math.atan(x * y / (z * r))
    return t


def box_inverse_distance_integral(a, b, c):
    """int_{[-a,a]x[-b,b]x[-c,c]} dy/|y| = 8 * (8-corner inclusion-exclusion of F)."""
    tot = 0.0
    for cx, cy, cz in itertools.product((0, 1), repeat=3):
        sgn = (-1) ** (3 - cx - cy - cz)
        tot += sgn * _corner_F(a * cx, b * cy, c * cz)
    return 8.0 * tot


def test_corner_formula_unit_cube():
    # int over [0,1]^3 of 1/|y|: the classical value 1.1900386819897766...
    # (3 ln((1+sqrt3)/sqrt2) - pi/4, a known closed form).
    s = box_inverse_distance_integral(1, 1, 1) / 8.0
    ref = 3 * math.log((1 + math.sqrt(3)) / math.sqrt(2)) - math.pi / 4
    assert abs(s - ref) < 1e-14


@pytest.mark.parametrize("N,L", [((8, 8, 4), (1.0, 1.0, 0.5)), ((32, 32, 16), (8.0, 8.0, 2.0)),
                                 ((12, 10, 6), (3.0, 2.5, 0.4)), ((256, 256, 64), (16.0, 16.0, 1.5))])
def test_U0_at_zero_frequency_closed_form(N, L):
    U0 = O.truncated_coulomb_fourier(N, L)
    a = [2 * v for v in L]
    ref = box_inverse_distance_integral(*a) / (4 * math.pi)
    assert abs(U0[0, 0, 0] - ref) <= 2e-14 * ref


def _G(aa, R):
    """int_0^R r e^{-i aa r} dr."""
    x = aa * R
    out = np.empty(np.shape(x), dtype=np.complex128)
    small = np.abs(x) < 1e-3
    xs = x[small]
    Rs = R[small]
    out[small] = Rs ** 2 * (0.5 - 1j * xs / 3 - xs ** 2 / 8 + 1j * xs ** 3 / 30 + xs ** 4 / 144)
    xl = x[~small]
    al = aa[~small]
    out[~small] = (np.exp(-1j * xl) * (1 + 1j * xl) - 1) / al ** 2
    return out


def face_decomposition_U0(nu, a, nodes=80):
    """Independent route to U0(nu) = int_box e^{-i nu.y}/(4 pi |y|) dy: the box
    is a union of cones from the origin over its six faces; along each ray the
    radial integral is int_0^R r e^{-i (nu.q) r} dr in closed form, leaving a
    smooth 2D Gauss-Legendre quadrature over each face."""
    xg, wg = roots_legendre(nodes)
    total = 0.0 + 0.0j
    for axis in range(3):
        o1, o2 = [i for i in range(3) if i != axis]
        u = a[o1] * xg
        v = a[o2] * xg
        U, V = np.meshgrid(u, v, indexing="ij")
        Wt = np.outer(wg, wg) * a[o1] * a[o2]
        for sgn in (1.0, -1.0):
            q = np.zeros((3,) + U.shape)
            q[axis] = sgn * a[axis]
            q[o1] = U
            q[o2] = V
            R = np.sqrt((q ** 2).sum(0))
            qhat = q / R
            aa = nu[0] * qhat[0] + nu[1] * qhat[1] + nu[2] * qhat[2]
            total += np.sum(Wt * a[axis] / R ** 3 * _G(aa, R))
    return total.real / (4 * math.pi)


def test_U0_nonzero_frequencies_vs_face_decomposition():
    N, L = (6, 8, 4), (1.0, 0.75, 0.35)
    U0 = O.truncated_coulomb_fourier(N, L)
    a = [2 * v for v in L]
    worst = 0.0
    for k in [(1, 0, 0), (0, 2, 0), (0, 0, 1), (1, 2, 1), (3, 1, 2), (6, 8, 4), (2, 5, 3)]:
        nu = [math.pi * k[i] / a[i] for i in range(3)]
        ref = face_decomposition_U0(nu, a)
        got = U0[k[2], k[1], k[0]]
        worst = max(worst, abs(got - ref) / U0[0, 0, 0])
    assert worst < 1e-12


def test_U0_quadrature_converged_in_step():
    N, L = (16, 12, 8), (4.0, 3.0, 0.6)
    A = O.truncated_coulomb_fourier(N, L, h_tau=0.1)
    B = O.truncated_coulomb_fourier(N, L, h_tau=0.05)
    assert np.max(np.abs(A - B)) <= 1e-15 * np.max(np.abs(A))


# ----------------------------------------------- Gaussian densities (closed form)
def _iso_potential_series(r, sigma):
    """phi_C(r) = erf(r/(sqrt2 sigma)) / (4 pi r) and the radial pieces needed
    for d_nn: returns (phi_C, phi_C'/r, phi_C''), by the Maclaurin series in r
    (used for r < 1) and by the closed form elsewhere."""
    c = 1.0 / (math.sqrt(2.0) * sigma)
    pref = 1.0 / (4 * math.pi) * 2.0 / math.sqrt(math.pi)
    r = np.asarray(r, dtype=np.float64)
    f0 = np.zeros_like(r)
    f1 = np.zeros_like(r)
    f2 = np.zeros_like(r)
    small = r < 1.0
    rs = r[small]
    for m in range(0, 30):
        am = pref * (-1) ** m * c ** (2 * m + 1) / (math.factorial(m) * (2 * m + 1))
        f0[small] += am * rs ** (2 * m)
        if m >= 1:
            f1[small] += 2 * m * am * rs ** (2 * m - 2)
            f2[small] += 2 * m * (2 * m - 1) * am * rs ** (2 * m - 2)
    rl = r[~small]
    fe = erf(c * rl)
    fp = 2 * c / math.sqrt(math.pi) * np.exp(-(c * rl) ** 2)
    fpp = -2 * c * c * rl * fp
    f0[~small] = fe / (4 * math.pi * rl)
    d1 = (fp * rl - fe) / (4 * math.pi * rl ** 2)
    f1[~small] = d1 / rl
    f2[~small] = fpp / (4 * math.pi * rl) - 2 * (fp * rl - fe) / (4 * math.pi * rl ** 3)
    return f0, f1, f2


def iso_gaussian_dipolar(N, L, n, sigma=1.0):
    """Exact Phi = -rho - 3 d_nn (U * rho) for an isotropic Gaussian rho."""
    x, y, z = W.mesh(N, L)
    r = np.sqrt(x * x + y * y + z * z)
    rho = W.gaussian_density(N, L, (sigma,) * 3)
    f0, f1, f2 = _iso_potential_series(r, sigma)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos2 = np.where(r > 0, ((n[0] * x + n[1] * y + n[2] * z) / np.where(r > 0, r, 1)) ** 2, 0.0)
    dnn = f2 * cos2 + f1 * (1 - cos2)
    # at r = 0 both radial pieces tend to the same limit, so d_nn = f2(0)
    return rho, f0, -rho - 3 * dnn


@pytest.fixture(scope="module")
def iso64():
    N, L = (64, 64, 64), (8.0, 8.0, 8.0)
    U0 = O.truncated_coulomb_fourier(N, L)
    return N, L, U0


def test_coulomb_isotropic_gaussian(iso64):
    N, L, U0 = iso64
    rho, phiC, _ = iso_gaussian_dipolar(N, L, (0, 0, 1))
    got = O.truncated_convolution(rho, O.coulomb_multiplier_full(N, L, U0))
    assert np.max(np.abs(got - phiC)) <= 1e-12 * np.max(np.abs(phiC))


@pytest.mark.parametrize("n", [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0),
                               (math.sin(math.radians(30)), 0.0, math.cos(math.radians(30))),
                               (0.5, 0.5, math.sqrt(0.5))])
def test_dipolar_isotropic_gaussian(iso64, n):
    N, L, U0 = iso64
    rho, _, Phi = iso_gaussian_dipolar(N, L, n)
    K = O.dipolar_multiplier(N, L, n, U0)
    got = O.truncated_convolution(rho, K)
    assert np.max(np.abs(got - Phi)) <= 1e-12 * np.max(np.abs(Phi))


def _aniso_gaussian_dipolar_point(xv, sigma, n):
    """Exact Coulomb and d_nn-Coulomb potential of an anisotropic Gaussian at
    one point, by 1D quadrature of the Gaussian-transform representation."""
    pref = 1.0 / (4 * math.pi) * 2.0 / math.sqrt(math.pi)

    def terms(s):
        aa = [s * s / (1 + 2 * s * s * sg * sg) for sg in sigma]
        amp = 1.0
        for sg in sigma:
            amp /= math.sqrt(1 + 2 * s * s * sg * sg)
        e = amp * math.exp(-sum(aa[i] * xv[i] ** 2 for i in range(3)))
        lin = sum(n[i] * aa[i] * xv[i] for i in range(3))
        fac = 4 * lin * lin - 2 * sum(n[i] ** 2 * aa[i] for i in range(3))
        return e, e * fac

    c = integrate.quad(lambda s: terms(s)[0], 0, np.inf, epsabs=1e-16, epsrel=1e-14, limit=400)[0]
    d = integrate.quad(lambda s: terms(s)[1], 0, np.inf, epsabs=1e-16, epsrel=1e-14, limit=400)[0]
    return pref * c, pref * d


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_dipolar_anisotropic_gaussian_points():
    N, L = (64, 64, 64), (8.0, 8.0, 1.6)
    sigma = (1.0, 1.0, 0.2)
    n = (math.sin(math.radians(30)), 0.0, math.cos(math.radians(30)))
    K = O.dipolar_multiplier(N, L, n)
    rho = W.gaussian_density(N, L, sigma)
    Phi = O.truncated_convolution(rho, K)
    scale = np.max(np.abs(Phi))
    xs = [W.axis_coords(N[i], L[i]) for i in range(3)]
    g = W.SplitMix64(11)
    worst = 0.0
    for _ in range(12):
        j = [int(g.uniform() * N[i]) for i in range(3)]
        xv = [xs[i][j[i]] for i in range(3)]
        _, dnn = _aniso_gaussian_dipolar_point(xv, sigma, n)
        r = rho[j[2], j[1], j[0]]
        ref = -r - 3 * dnn
        worst = max(worst, abs(Phi[j[2], j[1], j[0]] - ref) / scale)
    assert worst < 1e-11


# ----------------------------------------------------------------- identities
def test_trace_of_dipolar_kernel_vanishes():
    """sum over n in {e_x, e_y, e_z} of U_dip = 0 (Eq. (DDI-3D)): the three
    potentials of a smooth density supported in the box sum to zero."""
    N, L = (32, 32, 16), (6.0, 6.0, 1.5)
    U0 = O.truncated_coulomb_fourier(N, L)
    rho = np.real(W.random_smooth_field(N, L, (1.3, 1.0, 9.0), seed=3, complex_valued=False)) ** 2
    tot = sum(O.truncated_convolution(rho, O.dipolar_multiplier(N, L, e, U0))
              for e in [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
    single = O.truncated_convolution(rho, O.dipolar_multiplier(N, L, (0, 0, 1), U0))
    assert np.max(np.abs(tot)) <= 1e-11 * np.max(np.abs(single))


def test_dipolar_operator_symmetric():
    N, L = (16, 12, 8), (4.0, 3.0, 1.0)
    n = (0.6, 0.0, 0.8)
    plan = O.Plan(N, L, n)
    g = plan.grid
    r1 = W.random_field(g.shape, 5, complex_valued=False)
    r2 = W.random_field(g.shape, 6, complex_valued=False)
    a = O.inner(plan.dipolar_potential(r1), r2, g)
    b = O.inner(r1, plan.dipolar_potential(r2), g)
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))


def test_truncated_convolution_matches_direct_circular_sum():
    """FFT route = brute-force sum_j g(i - j) rho_j with g the padded kernel
    (inverse DFT of K), for i, j on the original grid: pins padding and crop."""
    N, L = (6, 4, 4), (1.0, 0.8, 0.5)
    n = (0.6, 0.0, 0.8)
    K = O.dipolar_multiplier(N, L, n)
    gker = np.fft.ifftn(K)
    rho = W.random_field((N[2], N[1], N[0]), 9, complex_valued=False)
    M = (2 * N[2], 2 * N[1], 2 * N[0])
    direct = np.zeros((N[2], N[1], N[0]), dtype=np.complex128)
    for iz, iy, ix in itertools.product(range(N[2]), range(N[1]), range(N[0])):
        acc = 0j
        for jz, jy, jx in itertools.product(range(N[2]), range(N[1]), range(N[0])):
            acc += gker[(iz - jz) % M[0], (iy - jy) % M[1], (ix - jx) % M[2]] * rho[jz, jy, jx]
        direct[iz, iy, ix] = acc
    got = O.truncated_convolution(rho, K)
    assert np.max(np.abs(got - direct.real)) <= 1e-13 * np.max(np.abs(direct))


def test_plan_rejects_non_unit_axis():
    with pytest.raises(ValueError):
        O.Plan((8, 8, 4), (1, 1, 1), (0, 0, 1.01))
