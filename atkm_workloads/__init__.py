"""Seeded synthetic inputs for the PCG-ATKM ground-state solver.

This module is shared by the CPU oracle, the GPU tests and ``bench.py``.  It
holds only input recipes: the five workload configurations (physical
parameters, boxes, grids), grid coordinates, initial wave functions and test
densities.  It contains none of the solver's arithmetic (no FFT, no kernel
multiplier, no energy, no inner product of the method), so both sides of a
parity comparison see identical input bytes while sharing no method code.

Every random draw comes from SplitMix64 (S. Vigna, "Further scramblings of
Marsaglia's xorshift generators", 2014 / the public-domain reference
``splitmix64.c``), restated here from its published definition, so the same
seed gives the same inputs on any machine.

Grid convention (the paper's §2.1): the box is prod_a [-L_a, L_a], N_a is
even, h_a = 2 L_a / N_a and x_j = -L_a + j h_a for j = 0..N_a-1.  Arrays are
row-major with shape (N_z, N_y, N_x): x is the fastest index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter generator (Vigna 2014), 53-bit doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_array(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)


@dataclass
class Workload:
    """One ground-state problem: grid, box, trap, interactions, dipole axis."""

    name: str
    N: tuple  # (N_x, N_y, N_z), each even
    L: tuple  # box half-lengths (L_x, L_y, L_z)
    gamma: tuple  # trap frequencies (gamma_x, gamma_y, gamma_z)
    beta: float
    lam: float
    n: tuple  # dipole axis, unit vector
    Omega: float
    guess: str = "phi_d"  # initial-guess recipe name
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        """Array shape (N_z, N_y, N_x)."""
        return (self.N[2], self.N[1], self.N[0])


def axis_coords(N: int, L: float) -> np.ndarray:
    """x_j = -L + j h, h = 2L/N, j = 0..N-1 (left end in, right end out)."""
    h = 2.0 * L / N
    return -L + h * np.arange(N, dtype=np.float64)


def mesh(N, L):
    """Broadcastable coordinate arrays (X, Y, Z) for shape (N_z, N_y, N_x)."""
    x = axis_coords(N[0], L[0])[None, None, :]
    y = axis_coords(N[1], L[1])[None, :, None]
    z = axis_coords(N[2], L[2])[:, None, None]
    return x, y, z


def _l2(f, N, L) -> float:
    h3 = (2.0 * L[0] / N[0]) * (2.0 * L[1] / N[1]) * (2.0 * L[2] / N[2])
    return math.sqrt(h3 * float(np.sum(np.abs(f) ** 2)))


def gaussian_G(N, L, gamma) -> np.ndarray:
    """G = exp(-sum_a gamma_a x_a^2 / 2): the harmonic ground-state shape."""
    x, y, z = mesh(N, L)
    return np.exp(-0.5 * (gamma[0] * x * x + gamma[1] * y * y + gamma[2] * z * z))


def guess_phi_d(N, L, gamma, Omega) -> np.ndarray:
    """Initial guess (d) of §3: ((1-Omega) phi_a + Omega phi_b) normalised,
    with phi_a = G/|G| and phi_b = (x+iy)G/|(x+iy)G|, G of widths 1/sqrt(gamma)."""
    x, y, _ = mesh(N, L)
    G = gaussian_G(N, L, gamma).astype(np.complex128)
    pa = G / _l2(G, N, L)
    b = (x + 1j * y) * G
    pb = b / _l2(b, N, L)
    d = (1.0 - Omega) * pa + Omega * pb
    return d / _l2(d, N, L)


def vortex_positions(count: int, radius: float, seed: int):
    """Area-uniform points in a disc: r = R sqrt(u), theta = 2 pi v."""
    g = SplitMix64(seed)
    pts = []
    for _ in range(count):
        u = g.uniform()
        v = g.uniform()
        r = radius * math.sqrt(u)
        th = 2.0 * math.pi * v
        pts.append((r * math.cos(th), r * math.sin(th)))
    return pts


def guess_vortex_product(N, L, gamma, count=8, radius=4.0, seed=1) -> np.ndarray:
    """G times prod_j ((x - x_j) + i (y - y_j)) at seeded vortex positions."""
    x, y, _ = mesh(N, L)
    f = gaussian_G(N, L, gamma).astype(np.complex128)
    for (xj, yj) in vortex_positions(count, radius, seed):
        f = f * ((x - xj) + 1j * (y - yj))
    return f / _l2(f, N, L)


def initial_guess(w: Workload) -> np.ndarray:
    """psi_0 of a workload, complex128 of shape (N_z, N_y, N_x), unit norm."""
    if w.guess == "phi_d":
        return guess_phi_d(w.N, w.L, w.gamma, w.Omega)
    if w.guess == "vortex8":
        return guess_vortex_product(w.N, w.L, w.gamma, 8, 4.0, w.seed)
    if w.guess == "phi_a":
        G = gaussian_G(w.N, w.L, w.gamma).astype(np.complex128)
        return G / _l2(G, w.N, w.L)
    raise ValueError(f"unknown guess {w.guess}")


def gaussian_density(N, L, sigma, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """rho = prod_a (2 pi sigma_a^2)^(-1/2) exp(-(x_a - c_a)^2 / (2 sigma_a^2))."""
    x, y, z = mesh(N, L)
    s = sigma
    return (np.exp(-((x - center[0]) ** 2) / (2 * s[0] ** 2)) / math.sqrt(2 * math.pi * s[0] ** 2)
            * np.exp(-((y - center[1]) ** 2) / (2 * s[1] ** 2)) / math.sqrt(2 * math.pi * s[1] ** 2)
            * np.exp(-((z - center[2]) ** 2) / (2 * s[2] ** 2)) / math.sqrt(2 * math.pi * s[2] ** 2))


def random_smooth_field(N, L, gamma, seed: int, terms: int = 6, complex_valued=True) -> np.ndarray:
    """A seeded smooth, decaying field: G times a random low-order polynomial
    in (x, y, z) with SplitMix64 coefficients (tests of linear operators)."""
    g = SplitMix64(seed)
    x, y, z = mesh(N, L)
    G = gaussian_G(N, L, gamma)
    acc = np.zeros(G.shape, dtype=np.complex128 if complex_valued else np.float64)
    for _ in range(terms):
        px, py, pz = (int(3 * g.uniform()) for _ in range(3))
        c = 2 * g.uniform() - 1
        if complex_valued:
            c = c + 1j * (2 * g.uniform() - 1)
        sx = 1 + 0.5 * g.uniform()
        acc = acc + c * (x ** px) * (y ** py) * (z ** pz) * G ** sx
    return acc


def random_field(shape, seed: int, complex_valued=True) -> np.ndarray:
    """Seeded i.i.d. uniform(-1, 1) entries (non-smooth; for exactness tests)."""
    g = SplitMix64(seed)
    n = int(np.prod(shape))
    re = 2 * g.uniform_array(n) - 1
    if not complex_valued:
        return re.reshape(shape)
    im = 2 * g.uniform_array(n) - 1
    return (re + 1j * im).reshape(shape)


_S30 = math.sin(math.radians(30.0))
_C30 = math.cos(math.radians(30.0))

CONFIGS = {
    # Plain FP64 PCG, pancake 32x32x16 (the small oracle-checkable case).
    "cfg1_32x32x16": Workload("cfg1_32x32x16", (32, 32, 16), (8.0, 8.0, 2.0), (1.0, 1.0, 4.0),
                              50.0, 15.0, (0.0, 0.0, 1.0), 0.4, "phi_d"),
    # Strongly anisotropic pancake with 8 seeded vortices in the guess.
    "cfg2_128x128x32": Workload("cfg2_128x128x32", (128, 128, 32), (12.0, 12.0, 1.0), (1.0, 1.0, 50.0),
                                500.0, 200.0, (0.0, 0.0, 1.0), 0.8, "vortex8", seed=1),
    # Headline grid: tilted dipole, fast rotation.
    "cfg3_256x256x64": Workload("cfg3_256x256x64", (256, 256, 64), (16.0, 16.0, 1.5), (1.0, 1.2, 30.0),
                                1000.0, 400.0, (_S30, 0.0, _C30), 0.9, "phi_d"),
}


# Setups of the paper's own experiments (§3), as input recipes.
PAPER_WORKLOADS = {
    # Example 3.1, Case II at Omega = 0.2 (no vortex: one ground state):
    # beta = 100, lambda = 0.8 beta, n = z, gamma = (1, 2, 10), [-16,16]^2 x [-10,10].
    "ex31_caseII_256": Workload("ex31_caseII_256", (256, 256, 256), (16.0, 16.0, 10.0), (1.0, 2.0, 10.0),
                                100.0, 80.0, (0.0, 0.0, 1.0), 0.2, "phi_d"),
    # Example 3.2: U-shape vortex line in a cigar, attractive dipoles along z.
    "ex32_256": Workload("ex32_256", (256, 256, 256), (10.0, 10.0, 100.0), (1.0, 1.0, 0.05),
                         1000.0, -300.0, (0.0, 0.0, 1.0), 0.75, "phi_d"),
}


def sweep_instances(count: int = 48, seed: int = 4):
    """Uneven-grid Omega/anisotropy sweep (48 instances): Omega ~ U[0.5, 0.95],
    gamma_z in {10, 20, 40}, beta = 200, lambda/beta in {0.2, 0.4}, n = z,
    in-plane edge from a 2/3/5-smooth list, N_z = edge/4, box
    [-16,16]^2 x [-sqrt(64/gamma_z), sqrt(64/gamma_z)]."""
    g = SplitMix64(seed)
    edges = [64, 72, 80, 96, 120, 128, 144, 160, 192]
    out = []
    for i in range(count):
        Om = 0.5 + 0.45 * g.uniform()
        gz = [10.0, 20.0, 40.0][min(2, int(3 * g.uniform()))]
        lr = [0.2, 0.4][min(1, int(2 * g.uniform()))]
        e = edges[min(len(edges) - 1, int(len(edges) * g.uniform()))]
        Lz = math.sqrt(64.0 / gz)
        out.append(Workload(f"sweep{i:02d}_{e}x{e}x{e // 4}", (e, e, e // 4), (16.0, 16.0, Lz),
                            (1.0, 1.0, gz), 200.0, 200.0 * lr, (0.0, 0.0, 1.0), Om, "phi_d"))
    return out


GUESS_COARSE_N = (64, 64, 16)
GUESS_FINE_N = (128, 128, 32)


def guess_draws(count: int, seed: int = 5, N=GUESS_COARSE_N):
    """Seeded parameter draws of the learned-guess workload: Omega ~ U[0.3, 0.95],
    gamma = (1, 1, gamma_z) with gamma_z ~ U[5, 50], beta ~ U[100, 1000],
    lambda/beta ~ U[0, 0.45], dipole tilt
    theta ~ U[0, 60 deg] in the xz plane (n = (sin theta, 0, cos theta)); box
    [-16,16]^2 x [-sqrt(64/gamma_z), sqrt(64/gamma_z)]; initial guess (d)."""
    g = SplitMix64(seed)
    out = []
    for i in range(count):
        Om = 0.3 + 0.65 * g.uniform()
        gz = 5.0 + 45.0 * g.uniform()
        beta = 100.0 + 900.0 * g.uniform()
        lr = 0.45 * g.uniform()
        th = math.radians(60.0) * g.uniform()
        Lz = math.sqrt(64.0 / gz)
        out.append(Workload(f"guess{seed}_{i:04d}", tuple(N), (16.0, 16.0, Lz), (1.0, 1.0, gz), beta, lr * beta,
                            (math.sin(th), 0.0, math.cos(th)), Om, "phi_d", seed=i))
    return out


def with_grid(w: Workload, N) -> Workload:
    """The same problem on another grid of the same box."""
    return Workload(w.name, tuple(N), w.L, w.gamma, w.beta, w.lam, w.n, w.Omega, w.guess, w.seed, dict(w.extra))


PAPER_GUESS_NAMES = ("a", "b", "bbar", "c", "cbar", "d", "dbar", "e", "ebar", "f")


def paper_guesses(N, L, gamma, beta, Omega) -> dict:
    """The ten initial guesses of §3, each normalised in the discrete norm:
    (a) the unit-width Gaussian exp(-|x|^2/2); (b) (x + i y) times it; (c) a + b;
    (d) (1 - Omega) a + Omega b; (e) Omega a + (1 - Omega) b, each of b-e with
    its complex conjugate; (f) the Thomas-Fermi profile sqrt(max(mu_TF - V, 0)/beta)
    with V = (gamma_x^2 x^2 + gamma_y^2 y^2 + gamma_z^2 z^2)/2 and
    mu_TF = (1/2) (15 beta gamma_x gamma_y gamma_z / (4 pi))^(2/5)."""
    x, y, z = mesh(N, L)
    shape = (N[2], N[1], N[0])

    def nrm(f):
        f = np.broadcast_to(f, shape).astype(np.complex128)
        return f / _l2(f, N, L)

    pa = nrm(np.exp(-(x * x + y * y + z * z) / 2))
    pb = nrm((x + 1j * y) * pa)
    V = 0.5 * (gamma[0] ** 2 * x * x + gamma[1] ** 2 * y * y + gamma[2] ** 2 * z * z)  # the trap, Eq. (Vpoten)
    mu_tf = 0.5 * (15.0 * beta * gamma[0] * gamma[1] * gamma[2] / (4.0 * math.pi)) ** 0.4
    g = {"a": pa, "b": pb, "c": nrm(pa + pb), "d": nrm((1 - Omega) * pa + Omega * pb),
         "e": nrm(Omega * pa + (1 - Omega) * pb)}
    for k in ("b", "c", "d", "e"):
        g[k + "bar"] = np.conj(g[k])
    g["f"] = nrm(np.sqrt(np.maximum(mu_tf - V, 0.0) / beta))
    return {k: g[k] for k in PAPER_GUESS_NAMES}
