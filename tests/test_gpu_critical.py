"""The critical rotation frequency Omega_c on the batched solver against what
the paper states in §3 (Examples 3.4 and 3.5; its figures are not in the text,
so the checks are the trends it states), on 64^3 grids of [-10,10]^3:
  * isotropic trap, n = z: Omega_c increases with lambda (Example 3.5, Case I);
  * isotropic trap, lambda = 0: Omega_c decreases as beta increases
    (Example 3.4, Case III);
  * beta = 400, n = (sin theta, 0, cos theta): from theta = 0 to 90 degrees
    Omega_c decreases for lambda > 0 and increases for lambda < 0, by less for
    +100 than for -100 (Example 3.5, Case III);
and the physics the method must keep: in an axially symmetric setup the
vortex-free ground state does not depend on Omega (E, and <L_z> = 0), and the
one-vortex state carries <L_z> = 1 (to the discretisation error) with its
energy falling at that slope in Omega."""
import math

import pytest

from paper_2603_05194_gb300 import critical as CR

pytestmark = pytest.mark.gpu

N = (64, 64, 64)
BOX = (10.0, 10.0, 10.0)
Z = (0.0, 0.0, 1.0)
OMEGAS = [0.15, 0.25, 0.35, 0.45, 0.55, 0.65, 0.75]


def oc(beta, lam, n=Z):
    r = CR.omega_c((1.0, 1.0, 1.0), beta, lam, n, N, BOX, OMEGAS)
    assert r["Omega_c"] is not None and len(r["points"]) >= 2, r["points"]
    return r


@pytest.fixture(scope="module")
def case1():
    return {lam: oc(200.0, lam) for lam in (-100.0, 0.0, 100.0)}


def test_omega_c_increases_with_lambda_along_z(lib, case1):
    c = [case1[lam]["Omega_c"] for lam in (-100.0, 0.0, 100.0)]
    assert c[0] < c[1] < c[2], c
    assert all(0.1 < v < 0.9 for v in c), c


def test_vortex_free_state_independent_of_omega(lib, case1):
    for r in case1.values():
        free = [row["a"] for row in r["rows"] if row["a"]["status"] == "OK" and abs(row["a"]["Lz"]) < 0.5]
        assert len(free) >= 2
        E = [s["E"] for s in free]
        assert max(E) - min(E) <= 1e-9 * abs(E[0])
        assert all(abs(s["Lz"]) < 1e-6 for s in free)
        # the one-vortex state: <L_z> = 1 up to the discretisation (the square
        # grid's spectral operator commutes with quarter turns only), and its
        # energy falls with slope -<L_z> in Omega
        one = [(row["Omega"], row["b"]) for row in r["rows"]
               if row["b"]["status"] == "OK" and 0.5 <= row["b"]["Lz"] < 1.5]
        assert len(one) >= 2 and all(abs(s["Lz"] - 1.0) < 1e-2 for _, s in one)
        (o1, s1), (o2, s2) = one[0], one[-1]
        assert abs((s2["E"] - s1["E"]) / (o2 - o1) + 0.5 * (s1["Lz"] + s2["Lz"])) < 1e-2


def test_omega_c_decreases_with_beta(lib):
    lo, hi = oc(200.0, 0.0)["Omega_c"], oc(800.0, 0.0)["Omega_c"]
    assert hi < lo, (lo, hi)


def test_omega_c_against_dipole_tilt(lib):
    def tilt(th):
        t = math.radians(th)
        return (math.sin(t), 0.0, math.cos(t))

    c = {(lam, th): oc(400.0, lam, tilt(th))["Omega_c"] for lam in (100.0, -100.0) for th in (0.0, 90.0)}
    assert c[(100.0, 90.0)] < c[(100.0, 0.0)], c
    assert c[(-100.0, 90.0)] > c[(-100.0, 0.0)], c
    assert abs(c[(100.0, 90.0)] - c[(100.0, 0.0)]) < abs(c[(-100.0, 90.0)] - c[(-100.0, 0.0)]), c
