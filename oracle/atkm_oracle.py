"""CPU oracle of PCG-ATKM (Tang, Wang, Zhang, Zhang): TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of the paper's method in numpy/scipy.  It is
used only by tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg
of ``bench.py``; the product path never calls it.  It shares no code with the
CUDA path: the only common module is ``atkm_workloads`` (seeded inputs).

Library primitives used as single steps: ``numpy.fft.fftn/ifftn`` (the DFT of
§2.1, Eq. (FourphiCo)), ``scipy.special.wofz`` (Faddeeva function) and
``scipy.special.erf``.  There is no blocking, fusion or reordering beyond the
definitions below.

Arrays have shape (N_z, N_y, N_x) (x fastest).  Complex wave functions are
complex128, densities and potentials float64.

Readings of the paper where it is silent or garbled (each is also listed in
the design notes):
  * truncated-kernel coefficients: the unshifted, real, even
    U0(nu) = int_{D_2L} e^{-i nu.y} / (4 pi |y|) dy (Eq. (FUk) without the
    basis phase (-1)^{k_x+k_y+k_z}); rho occupies padded indices [0, N) and the
    result is cropped to [0, N);
  * the ATKM output is real-part'ed (equivalently, the multiplier is
    symmetrised on the padded Nyquist planes);
  * the kernel in g_n of Eq. (Energy_Expend) is U_dip (the dipolar multiplier);
  * the stop rule is ||r_n|| <= tol with r_n = H phi_n - mu phi_n in the
    discrete L2 norm of Eq. (innerPro); ||phi_{n+1}-phi_n||_inf is logged and
    can be used instead (Eq. (stop_maxnorm));
  * "halve until the energy decreases" accepts E+ <= E + 32 eps |E| and stops
    after at most ``max_halvings`` halvings (then the lowest trial is taken and
    the next direction is forced to steepest descent); three consecutive
    exhausted halvings end the run as stagnated;
  * after each retraction phi is divided by its norm;
  * when Step 4 resets p to J(-P r), that reset p is the p_n kept for n+1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf, wofz

EPS = np.finfo(np.float64).eps

# Status codes (same meaning as the C interface; the values are restated, not shared).
OK = 0
NOT_CONVERGED = 5
STAGNATED = 6
ERR_NAN = 7


# ---------------------------------------------------------------------------
# §2.1 Spatial discretisation
# ---------------------------------------------------------------------------
class Grid:
    """Uniform grid on prod_a [-L_a, L_a] (§2.1): h_a = 2 L_a / N_a,
    x_j = -L_a + j h_a, Fourier frequencies nu_k = pi k / L_a with
    k in [-N_a/2, N_a/2 - 1] (stored in FFT order)."""

    def __init__(self, N, L):
        self.N = tuple(int(v) for v in N)
        self.L = tuple(float(v) for v in L)
        for Na in self.N:
            if Na <= 0 or Na % 2:
                raise ValueError("grid sizes must be even and positive")
        self.h = tuple(2.0 * La / Na for La, Na in zip(self.L, self.N))
        self.hvol = self.h[0] * self.h[1] * self.h[2]
        self.shape = (self.N[2], self.N[1], self.N[0])
        xs = [-La + h * np.arange(Na) for La, Na, h in zip(self.L, self.N, self.h)]
        self.x = xs[0][None, None, :]
        self.y = xs[1][None, :, None]
        self.z = xs[2][:, None, None]
        nus = [np.pi * fft_index(Na) / La for La, Na in zip(self.L, self.N)]
        self.nu_x = nus[0][None, None, :]
        self.nu_y = nus[1][None, :, None]
        self.nu_z = nus[2][:, None, None]
        self.nu2 = self.nu_x ** 2 + self.nu_y ** 2 + self.nu_z ** 2


def fft_index(M: int) -> np.ndarray:
    """Integer frequencies k of a length-M DFT in FFT order: 0..M/2-1, -M/2..-1."""
    m = np.arange(M)
    return np.where(m < M // 2, m, m - M).astype(np.float64)


def inner(U, V, g: Grid) -> float:
    """<U, V> = Re(h_x h_y h_z sum_j U_j conj(V_j))  (Eq. (innerPro))."""
    return float(np.real(g.hvol * np.sum(U * np.conj(V))))


def norm(U, g: Grid) -> float:
    """||U|| = <U, U>^(1/2)  (Eq. (innerPro))."""
    return math.sqrt(inner(U, U, g))


def spectral_apply(f, mult):
    """Sum_k mult_k fhat_k W_k at the grid points (Eq. (Fourphi)-(Laplacian))."""
    return np.fft.ifftn(mult * np.fft.fftn(f))


def d_dx(f, g: Grid):
    """[[d_x]] f: multiplier i nu_x (Eq. (Laplacian)); Nyquist kept literally."""
    return spectral_apply(f, 1j * g.nu_x)


def d_dy(f, g: Grid):
    return spectral_apply(f, 1j * g.nu_y)


def laplacian(f, g: Grid):
    """[[Delta]] f: multiplier -(nu_x^2 + nu_y^2 + nu_z^2) (Eq. (Laplacian))."""
    return spectral_apply(f, -g.nu2)


def L_z(f, g: Grid):
    """[[L_z]] f = -i (x [[d_y]] f - y [[d_x]] f)  (Eq. (Laplacian))."""
    return -1j * (g.x * d_dy(f, g) - g.y * d_dx(f, g))


def trap(g: Grid, gamma):
    """V = (gamma_x^2 x^2 + gamma_y^2 y^2 + gamma_z^2 z^2) / 2  (Eq. (Vpoten))."""
    return 0.5 * (gamma[0] ** 2 * g.x ** 2 + gamma[1] ** 2 * g.y ** 2 + gamma[2] ** 2 * g.z ** 2)


# ---------------------------------------------------------------------------
# §2.2 Anisotropic truncated kernel method
# ---------------------------------------------------------------------------
def _axis_gauss_cos_integral(nu, a, s, k):
    """I(s; nu) = int_{-a}^{a} exp(-s^2 y^2) cos(nu y) dy for nu = pi k / a.

    Closed form (√pi/s) e^{-nu^2/4s^2} Re erf(s a + i nu/(2s)), written with the
    Faddeeva function w(z) = e^{-z^2} erfc(-iz) so nothing overflows:
        I = (√pi/s) Re[ e^{-nu^2/(4 s^2)} - e^{-s^2 a^2} e^{-i nu a} w(-nu/(2s) + i s a) ],
    with e^{-i nu a} = (-1)^k exactly; for k = 0 it is (√pi/s) erf(s a).
    ``nu`` and ``k`` have shape (K, 1), ``s`` shape (1, Q)."""
    out = np.empty(np.broadcast(nu, s).shape)
    zero = (k == 0)[:, 0]
    sq = math.sqrt(math.pi)
    out[zero, :] = (sq / s) * erf(s * a)
    if np.any(~zero):
        nz = nu[~zero]
        sign = np.where(k[~zero] % 2 == 0, 1.0, -1.0)
        z = -nz / (2.0 * s) + 1j * (s * a)
        with np.errstate(under="ignore", over="ignore"):
            val = np.exp(-nz ** 2 / (4.0 * s * s)) - np.exp(-(s * a) ** 2) * sign * np.real(wofz(z))
        out[~zero, :] = (sq / s) * val
    return out


def truncated_coulomb_fourier(N, L, h_tau: float = 0.1):
    """U0 on the nonnegative octant of the twofold-padded frequency grid.

    Eq. (FUk) (reading: unshifted basis) for the Coulomb kernel
    U(y) = 1/(4 pi |y|) on the padded box D_2L = prod [-2L_a, 2L_a]:
        U0(nu) = int_{D_2L} U(y) e^{-i nu.y} dy,  nu_a = pi k_a / (2 L_a),
    for |k_a| = 0..N_a (the padded grid has 2N_a points per axis).

    Route: 1/|y| = (2/√pi) int_0^inf e^{-s^2|y|^2} ds makes the box integral
    separable, U0 = (1/(2 pi^{3/2})) int_0^inf prod_a I_a(s) ds, with I_a the
    Gaussian-cosine integral above.  The s-integral is taken with the
    trapezoidal rule on the whole line in tau = ln s (integrand analytic in a
    strip and exponentially decaying at both ends, so the rule converges
    geometrically in 1/h_tau).  Returns an array of shape
    (N_z+1, N_y+1, N_x+1) indexed by (|k_z|, |k_y|, |k_x|)."""
    a = [2.0 * La for La in L]
    prod2a = (2 * a[0]) * (2 * a[1]) * (2 * a[2])
    tau_lo = math.log(1e-20 / prod2a)
    tau_hi = 0.5 * math.log(math.pi ** 1.5 * 1e20)
    nq = int(math.ceil((tau_hi - tau_lo) / h_tau)) + 1
    tau = tau_lo + h_tau * np.arange(nq)
    s = np.exp(tau)[None, :]
    tables = []
    for Na, aa in zip(N, a):
        k = np.arange(Na + 1, dtype=np.int64)[:, None]
        nu = np.pi * k.astype(np.float64) / aa
        tables.append(_axis_gauss_cos_integral(nu, aa, s, k))
    Tx, Ty, Tz = tables
    w = h_tau * s[0]  # d s = s d tau
    U0 = np.empty((N[2] + 1, N[1] + 1, N[0] + 1))
    for kz in range(N[2] + 1):
        U0[kz] = (Ty * (w * Tz[kz])[None, :]) @ Tx.T
    return U0 / (2.0 * math.pi ** 1.5)


def dipolar_multiplier(N, L, n, U0=None):
    """K(k) = -1 + 3 (n.nu_k)^2 U0(nu_k) on the full padded grid (FFT order).

    From Eq. (DDI2Cou3D): Phi = -rho - 3 U * (d_nn rho), and the spectral
    d_nn has multiplier -(n.nu)^2.  Shape (2N_z, 2N_y, 2N_x)."""
    if U0 is None:
        U0 = truncated_coulomb_fourier(N, L)
    M = [2 * Na for Na in N]
    kx, ky, kz = (fft_index(Ma) for Ma in M)
    nux = (np.pi * kx / (2.0 * L[0]))[None, None, :]
    nuy = (np.pi * ky / (2.0 * L[1]))[None, :, None]
    nuz = (np.pi * kz / (2.0 * L[2]))[:, None, None]
    ix = np.abs(kx).astype(np.int64)
    iy = np.abs(ky).astype(np.int64)
    iz = np.abs(kz).astype(np.int64)
    U0full = U0[np.ix_(iz, iy, ix)]
    ndotnu = n[0] * nux + n[1] * nuy + n[2] * nuz
    return -1.0 + 3.0 * ndotnu ** 2 * U0full


def coulomb_multiplier_full(N, L, U0=None):
    """U0 on the full padded grid (FFT order): the truncated Coulomb convolution."""
    if U0 is None:
        U0 = truncated_coulomb_fourier(N, L)
    M = [2 * Na for Na in N]
    ix, iy, iz = (np.abs(fft_index(Ma)).astype(np.int64) for Ma in M)
    return U0[np.ix_(iz, iy, ix)]


def truncated_convolution(rho, mult):
    """Three-step ATKM apply (§2.2): zero-pad rho to the twofold grid
    (indices [0, N) hold rho), FFT (Eq. (fouriercoeff)), multiply pointwise,
    inverse FFT (Eq. (U_TrunFour)), real part, crop to [0, N)."""
    Nz, Ny, Nx = rho.shape
    pad = np.zeros((2 * Nz, 2 * Ny, 2 * Nx), dtype=np.complex128)
    pad[:Nz, :Ny, :Nx] = rho
    out = np.fft.ifftn(mult * np.fft.fftn(pad))
    return np.real(out[:Nz, :Ny, :Nx]).copy()


class Plan:
    """Grid, box, dipole axis and the precomputed multiplier (the set-up
    step of Algorithm 1; §2.2: once per domain and mesh)."""

    def __init__(self, N, L, n):
        nn = math.sqrt(sum(v * v for v in n))
        if abs(nn - 1.0) > 1e-12:
            raise ValueError("dipole axis must be a unit vector")
        self.grid = Grid(N, L)
        self.n = tuple(float(v) for v in n)
        self.U0 = truncated_coulomb_fourier(self.grid.N, self.grid.L)
        self.K = dipolar_multiplier(self.grid.N, self.grid.L, self.n, self.U0)

    def dipolar_potential(self, rho):
        """Phi = U_dip * rho by ATKM (Eq. (DDI2Cou3D) + §2.2 three steps)."""
        return truncated_convolution(rho, self.K)


# ---------------------------------------------------------------------------
# §2.3 Discrete functional, gradient, projection, preconditioner
# ---------------------------------------------------------------------------
@dataclass
class Params:
    gamma: tuple
    beta: float
    lam: float
    Omega: float


def apply_H(plan: Plan, prm: Params, f, phi, Phi):
    """H_phi f = -1/2 [[Delta]] f + V f + beta |phi|^2 f + lambda Phi f
    - Omega [[L_z]] f  (§2.3, gradient of the discrete energy)."""
    g = plan.grid
    V = trap(g, prm.gamma)
    return (-0.5 * laplacian(f, g) + V * f + prm.beta * np.abs(phi) ** 2 * f
            + prm.lam * Phi * f - prm.Omega * L_z(f, g))


def energy_parts(plan: Plan, prm: Params, phi, Phi):
    """Terms of the discrete energy (§2.3) and the virial residual of
    Eq. (vir_iden): E_kin, E_pot, E_int, E_dip, E_rot, E, I."""
    g = plan.grid
    V = trap(g, prm.gamma)
    Ekin = inner(-0.5 * laplacian(phi, g), phi, g)
    Epot = inner(V * phi, phi, g)
    Eint = inner(0.5 * prm.beta * np.abs(phi) ** 2 * phi, phi, g)
    Edip = inner(0.5 * prm.lam * Phi * phi, phi, g)
    Erot = inner(-prm.Omega * L_z(phi, g), phi, g)
    E = Ekin + Epot + Eint + Edip + Erot
    vir = 2 * Ekin - 2 * Epot + 3 * Eint + 3 * Edip
    return dict(E_kin=Ekin, E_pot=Epot, E_int=Eint, E_dip=Edip, E_rot=Erot, E=E, virial=vir)


def energy(plan: Plan, prm: Params, phi, Phi) -> float:
    """Discrete energy E(phi) (§2.3) summed term by term."""
    return energy_parts(plan, prm, phi, Phi)["E"]


def project(f, phi, g: Grid):
    """J_phi(f) = f - <f, phi> phi  (§2.3, tangent projection)."""
    return f - inner(f, phi, g) * phi


def precond_shift(plan: Plan, prm: Params, phi, Phi) -> float:
    """alpha_Delta = alpha_V = <-1/2 [[Delta]] phi + V phi + beta|phi|^2 phi, phi>
    + |lambda <Phi phi, phi>|  (§2.3)."""
    g = plan.grid
    V = trap(g, prm.gamma)
    a = inner(-0.5 * laplacian(phi, g) + V * phi + prm.beta * np.abs(phi) ** 2 * phi, phi, g)
    return a + abs(prm.lam * inner(Phi * phi, phi, g))


def apply_precond(plan: Plan, prm: Params, r, phi, Phi, alpha):
    """P r = P_V^{1/2} P_Delta P_V^{1/2} r with P_Delta = (alpha - [[Delta]]/2)^{-1}
    and P_V = (alpha + V + beta|phi|^2 + |lambda|(1 + sign Phi) Phi / 2)^{-1} (§2.3)."""
    g = plan.grid
    V = trap(g, prm.gamma)
    PV = 1.0 / (alpha + V + prm.beta * np.abs(phi) ** 2
                + abs(prm.lam) * (1.0 + np.sign(Phi)) * Phi / 2.0)
    sq = np.sqrt(PV)
    return sq * spectral_apply(sq * r, 1.0 / (alpha + 0.5 * g.nu2))


# ---------------------------------------------------------------------------
# Algorithm 1 (PCG-ATKM)
# ---------------------------------------------------------------------------
@dataclass
class PcgOptions:
    tol_residual: float = 1e-8
    tol_linf: float = 0.0
    max_iter: int = 10000
    max_halvings: int = 20
    energy_tol_ulps: float = 32.0


@dataclass
class PcgResult:
    phi: np.ndarray
    Phi: np.ndarray
    status: int
    iters: int
    residual: float
    mu: float
    parts: dict
    halvings: int
    linf_step: float
    log: list = field(default_factory=list)


def pcg_ground_state(plan: Plan, prm: Params, phi0, opts: PcgOptions = PcgOptions()) -> PcgResult:
    """Algorithm 1 (PCG-ATKM) with the step control of §2.3 (i)-(iii)."""
    g = plan.grid
    phi = phi0 / norm(phi0, g)
    Phi = plan.dipolar_potential(np.abs(phi) ** 2)             # Step 1 (n = 0)
    E = energy(plan, prm, phi, Phi)
    p_prev = r_prev = None
    den_prev = None
    force_sd = False
    caps = 0
    total_halvings = 0
    linf = float("inf")
    log = []
    status = NOT_CONVERGED
    n = 0
    while True:
        # Step 2: residual and chemical potential.
        Hphi = apply_H(plan, prm, phi, phi, Phi)
        mu = inner(Hphi, phi, g)
        r = Hphi - mu * phi
        res = norm(r, g)
        entry = dict(n=n, E=E, mu=mu, residual=res, linf_step=linf)
        log.append(entry)
        if not (np.isfinite(E) and np.isfinite(res)):
            status = ERR_NAN
            break
        if res <= opts.tol_residual or (opts.tol_linf > 0 and linf <= opts.tol_linf):
            status = OK
            break
        if n >= opts.max_iter:
            status = NOT_CONVERGED
            break
        # Step 3: preconditioned conjugate direction (Polak-Ribiere+).
        alpha = precond_shift(plan, prm, phi, Phi)
        Pr = apply_precond(plan, prm, r, phi, Phi, alpha)
        JPr = project(Pr, phi, g)
        den = inner(r, JPr, g)
        d = project(-Pr, phi, g)
        beta_cg = 0.0
        if n > 0 and not force_sd:
            num = inner(r - project(r_prev, phi, g), JPr, g)
            beta_cg = max(num / den_prev, 0.0)
            p = d + beta_cg * project(p_prev, phi, g)
        else:
            p = d
        # Step 4 (i): fall back to preconditioned steepest descent if needed.
        d1 = inner(Hphi, p, g)
        reset = False
        if d1 >= 0.0:
            p = d
            beta_cg = 0.0
            reset = True
            d1 = inner(Hphi, p, g)
        # Step 4 (ii): quadratic model of Q(t) = E(R_phi(t p)), Eq. (Energy_Expend).
        Hp = apply_H(plan, prm, p, phi, Phi)
        rho1 = np.real(np.conj(phi) * p)
        Phi1 = plan.dipolar_potential(rho1)
        gn = 2.0 * phi * (prm.beta * rho1 + prm.lam * Phi1)
        pn2 = inner(p, p, g)
        curv = inner(Hp, p, g) + inner(gn, p, g) - mu * pn2
        t = -d1 / curv if curv > 0.0 else 0.3
        t0 = t
        pn = math.sqrt(pn2)
        # Step 4 (iii) + Step 5: retraction, halve until the energy decreases.
        tolE = opts.energy_tol_ulps * EPS * abs(E)
        best = None
        accepted = False
        nh = 0
        while True:
            phin = math.cos(t * pn) * phi + math.sin(t * pn) * p / pn
            phin = phin / norm(phin, g)
            Phin = plan.dipolar_potential(np.abs(phin) ** 2)
            En = energy(plan, prm, phin, Phin)
            if En <= E + tolE:
                accepted = True
                break
            if best is None or En < best[0]:
                best = (En, phin, Phin, t)
            if nh >= opts.max_halvings:
                break
            t *= 0.5
            nh += 1
        total_halvings += nh
        if accepted:
            caps = 0
            force_sd = False
        else:
            En, phin, Phin, t = best
            caps += 1
            force_sd = True
        entry.update(alpha=alpha, beta_cg=beta_cg, reset=reset, d1=d1, curv=curv,
                     t0=t0, t=t, halvings=nh, accepted=accepted)
        linf = float(np.max(np.abs(phin - phi)))
        r_prev, p_prev, den_prev = r, p, den
        phi, Phi, E = phin, Phin, En
        n += 1
        if caps >= 3:
            status = STAGNATED
            Hphi = apply_H(plan, prm, phi, phi, Phi)
            mu = inner(Hphi, phi, g)
            res = norm(Hphi - mu * phi, g)
            break
    parts = energy_parts(plan, prm, phi, Phi)
    return PcgResult(phi=phi, Phi=Phi, status=status, iters=n, residual=res, mu=mu,
                     parts=parts, halvings=total_halvings, linf_step=linf, log=log)


# ---------------------------------------------------------------------------
# Algorithm 2: cascadic multigrid (PCG-ATKM-MG)
# ---------------------------------------------------------------------------

def spectral_upsample(psi_c, Nf) -> np.ndarray:
    """Fourier interpolant (Eq. (Fourphi)) of a coarse grid function evaluated
    on a finer grid of the same box: the coefficients of k in Lambda_Nc are
    kept, every other coefficient of the fine grid is zero."""
    Nz, Ny, Nx = psi_c.shape
    c = np.fft.fftn(psi_c) / psi_c.size
    fine = np.zeros((Nf[2], Nf[1], Nf[0]), dtype=np.complex128)
    for kz in range(-Nz // 2, Nz // 2):
        for ky in range(-Ny // 2, Ny // 2):
            fine[kz % Nf[2], ky % Nf[1], np.arange(-Nx // 2, Nx // 2) % Nf[0]] = \
                c[kz % Nz, ky % Ny, np.arange(-Nx // 2, Nx // 2) % Nx]
    return np.fft.ifftn(fine) * fine.size


def pcg_ground_state_mg(plans, prm: Params, phi0, opts: PcgOptions = PcgOptions()) -> list:
    """Algorithm 2: on each mesh from the coarsest to the finest, Step 1 runs
    Algorithm 1 from the current initial data, Step 2 interpolates its ground
    state onto the next mesh (the Fourier interpolant above).  Returns the
    PcgResult of every level."""
    out = []
    phi = phi0
    for i, plan in enumerate(plans):
        res = pcg_ground_state(plan, prm, phi, opts)
        out.append(res)
        if i + 1 < len(plans):
            phi = spectral_upsample(res.phi, plans[i + 1].grid.N)
    return out

