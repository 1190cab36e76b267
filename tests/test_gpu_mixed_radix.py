"""The mixed-radix register FFT engine (lengths 3 * 2^a with 12 elements a
thread, 5 * 2^a with 20) against the oracle, through the C-ABI: every length
it serves (20, 24, 40, 48, 80, 96, 160, 192, 320, 384) in every axis role --
the x pass runs on N_x, the padded y and z passes of the ATKM on 2 N_y and
2 N_z, the H and preconditioner passes on N_x, N_y, N_z -- in binary64 and
FP32; and against the generic shared-memory engine on the same inputs
(ATKM_PLAN_GENERIC_FFT), where the two differ only by rounding.
Bars as in the other parity tests: Phi 1e-11 (FP64), 5e-6 (FP32); H and
P r 1e-12 (FP64)."""
import math

import numpy as np
import pytest
import torch

import atkm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# (N_x, N_y, N_z): x pass N_x, padded y 2 N_y, padded z 2 N_z
MIX_CASES = [
    ((96, 20, 12), (0.6, 0.0, 0.8)),     # x 96, y 40, z 24; unpadded y 20
    ((80, 48, 10), (0.0, 0.0, 1.0)),     # x 80, y 96, z 20; unpadded y 48
    ((40, 80, 24), (0.5, 0.5, math.sqrt(0.5))),  # x 40, y 160, z 48; unpadded y 80, z 24
    ((24, 160, 20), (0.6, 0.0, 0.8)),    # x 24, y 320, z 40; unpadded y 160, z 20
    ((20, 96, 40), (0.0, 0.6, 0.8)),     # x 20, y 192, z 80; unpadded z 40
    ((48, 24, 96), (0.6, 0.0, 0.8)),     # x 48, y 48, z 192; unpadded z 96
    ((160, 12, 48), (0.0, 0.0, 1.0)),    # x 160, y 24, z 96
    ((192, 10, 80), (0.6, 0.0, 0.8)),    # x 192, y 20, z 160; unpadded z 80
    ((320, 10, 20), (0.5, 0.5, math.sqrt(0.5))),  # x 320, y 20, z 40
    ((384, 12, 160), (0.0, 0.6, 0.8)),   # x 384, y 24, z 320; unpadded z 160
    ((24, 192, 10), (0.6, 0.0, 0.8)),    # y 384, unpadded y 192
]


@pytest.mark.parametrize("N,n", MIX_CASES)
def test_mixed_radix_passes_match_oracle(lib, N, n):
    L = (4.0, 3.0, 2.0)
    plan = lib.Plan(N, L, n, f32=True)
    oplan = O.Plan(N, L, n)
    shape = (N[2], N[1], N[0])
    psi = W.random_smooth_field(N, L, (1.0, 1.3, 2.0), seed=501)
    white = W.random_field(shape, 502)
    for f in (psi, white):
        ref = oplan.dipolar_potential(np.abs(f) ** 2)
        assert rel2(host(plan.dipolar_potential_from_psi(dev(f))), ref) <= 1e-11
        assert rel2(host(plan.dipolar_potential_from_psi(dev(f), f32=True)), ref) <= 5e-6
    b = W.random_field(shape, 503)
    assert rel2(host(plan.dipolar_potential_from_pair(dev(white), dev(b))),
                oplan.dipolar_potential(np.real(np.conj(white) * b))) <= 1e-11
    # H and the preconditioner on the unpadded lengths
    gamma, beta, lam, Om = (1.0, 1.3, 6.0), 40.0, -12.0, 0.55
    oprm = O.Params(gamma, beta, lam, Om)
    prm = lib.make_params(gamma, beta, lam, Om)
    h3 = np.prod([2 * L[i] / N[i] for i in range(3)])
    phi = psi / math.sqrt(h3 * np.sum(np.abs(psi) ** 2))
    Phi = oplan.dipolar_potential(np.abs(phi) ** 2)
    assert rel2(host(plan.apply_H(prm, dev(white), dev(phi), dev(Phi))), O.apply_H(oplan, oprm, white, phi, Phi)) <= 1e-12
    e = plan.energy_parts(prm, dev(phi), dev(Phi))
    p = O.energy_parts(oplan, oprm, phi, Phi)
    assert abs(e["E"] - p["E"]) <= 1e-12 * (abs(p["E"]) + abs(p["E_kin"]) + abs(p["E_pot"]))
    alpha = O.precond_shift(oplan, oprm, phi, Phi)
    got = host(plan.apply_preconditioner(prm, alpha, dev(white), dev(phi), dev(Phi)))
    assert rel2(got, O.apply_precond(oplan, oprm, white, phi, Phi, alpha)) <= 1e-12


@pytest.mark.parametrize("N,n", MIX_CASES[:6])
def test_mixed_radix_equals_generic_engine(lib, N, n):
    L = (4.0, 3.0, 2.0)
    shape = (N[2], N[1], N[0])
    mix = lib.Plan(N, L, n, f32=True)
    gen = lib.Plan(N, L, n, f32=True, generic_fft=True)
    f = dev(W.random_field(shape, 504))
    a, b = host(mix.dipolar_potential_from_psi(f)), host(gen.dipolar_potential_from_psi(f))
    assert rel2(a, b) <= 1e-13
    a, b = host(mix.dipolar_potential_from_psi(f, f32=True)), host(gen.dipolar_potential_from_psi(f, f32=True))
    assert rel2(a, b) <= 2e-6


def test_mixed_radix_pcg_matches_oracle(lib):
    """A whole Algorithm 1 run on a grid whose every pass is mixed-radix."""
    N, L, n = (48, 40, 20), (7.0, 6.0, 2.5), (0.6, 0.0, 0.8)
    gamma, beta, lam, Om = (1.0, 1.2, 4.0), 40.0, 12.0, 0.35
    psi0 = W.guess_phi_d(N, L, gamma, Om)
    ref = O.pcg_ground_state(O.Plan(N, L, n), O.Params(gamma, beta, lam, Om), psi0,
                             O.PcgOptions(tol_residual=1e-10, max_iter=1500))
    plan = lib.Plan(N, L, n)
    psi = dev(psi0)
    r = plan.pcg_ground_state(lib.make_params(gamma, beta, lam, Om), psi, tol_residual=1e-10, max_iter=1500)
    assert ref.status == O.OK and r["status_name"] == "OK" and r["iters"] == ref.iters
    assert abs(r["E"] - ref.parts["E"]) <= 1e-10 * abs(ref.parts["E"])
    assert abs(r["mu"] - ref.mu) <= 1e-10 * abs(ref.mu)
