"""The FFT-tile autotuner (atkm_plan_autotune / ATKM_PLAN_AUTOTUNE) through
the C-ABI: it records one choice per non-power-of-two line length, layout and
arithmetic of the plan, never slower than the fixed rule on its own timing,
and the tuned plan's operators and a full Algorithm 1 run agree with the
oracle to the usual bars (Phi 1e-11 in binary64, 5e-6 in FP32; H and P r
1e-12; E and mu 1e-10)."""
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


CASES = [((48, 40, 20), (7.0, 6.0, 2.5), (0.6, 0.0, 0.8)),   # mixed-radix candidates (48, 80, 40, 20)
         ((72, 36, 18), (8.0, 6.0, 2.0), (0.0, 0.0, 1.0))]   # generic-engine candidates only (72, 36, 18)


@pytest.mark.parametrize("N,L,n", CASES)
def test_autotuned_plan_matches_oracle(lib, N, L, n):
    plan = lib.Plan(N, L, n, f32=True, df32=True, autotune=True)
    tun = plan.tuning()
    lengths = {N[0], 2 * N[1], 2 * N[2], N[1], N[2]}
    expect = {(r, Lx, lm) for r in (0, 1, 2) for Lx, lm in ((N[0], 1), (2 * N[1], 0), (2 * N[2], 0), (N[1], 0),
                                                             (N[2], 0)) if Lx & (Lx - 1)}
    assert {(t["precision"], t["length"], t["line_major"]) for t in tun} == expect
    for t in tun:
        assert t["length"] in lengths and t["engine"] in (1, 2)
        assert 0 < t["ms_best"] <= t["ms_default"]
        if t["engine"] == 1:
            assert t["precision"] != 2 and t["length"] in (20, 24, 40, 48, 80, 96, 160, 192, 320, 384)
        else:
            assert 0 <= t["tile_shift"] <= 2
    oplan = O.Plan(N, L, n)
    shape = (N[2], N[1], N[0])
    psi = W.random_smooth_field(N, L, (1.0, 1.3, 2.0), seed=601)
    ref = oplan.dipolar_potential(np.abs(psi) ** 2)
    assert rel2(host(plan.dipolar_potential_from_psi(dev(psi))), ref) <= 1e-11
    assert rel2(host(plan.dipolar_potential_from_psi(dev(psi), f32=True)), ref) <= 5e-6
    assert rel2(host(plan.dipolar_potential_from_psi(dev(psi), df32=True)), ref) <= 1e-11
    gamma, beta, lam, Om = (1.0, 1.2, 4.0), 40.0, 12.0, 0.35
    oprm, prm = O.Params(gamma, beta, lam, Om), lib.make_params(gamma, beta, lam, Om)
    h3 = np.prod([2 * L[i] / N[i] for i in range(3)])
    phi = psi / math.sqrt(h3 * np.sum(np.abs(psi) ** 2))
    Phi = oplan.dipolar_potential(np.abs(phi) ** 2)
    white = W.random_field(shape, 602)
    assert rel2(host(plan.apply_H(prm, dev(white), dev(phi), dev(Phi))), O.apply_H(oplan, oprm, white, phi, Phi)) <= 1e-12
    alpha = O.precond_shift(oplan, oprm, phi, Phi)
    got = host(plan.apply_preconditioner(prm, alpha, dev(white), dev(phi), dev(Phi)))
    assert rel2(got, O.apply_precond(oplan, oprm, white, phi, Phi, alpha)) <= 1e-12
    # a whole solve in binary64 and in the double-word split form
    psi0 = W.guess_phi_d(N, L, gamma, Om)
    o = O.pcg_ground_state(oplan, oprm, psi0, O.PcgOptions(tol_residual=1e-10, max_iter=1500))
    assert o.status == O.OK
    for prec in (0, 3):
        r = plan.pcg_ground_state(prm, dev(psi0), tol_residual=1e-10, max_iter=1500, precision=prec)
        assert r["status_name"] == "OK", prec
        assert abs(r["E"] - o.parts["E"]) <= 1e-10 * abs(o.parts["E"]), prec
        assert abs(r["mu"] - o.mu) <= 1e-10 * abs(o.mu), prec
    # tuning after the plan's first solve is refused
    with pytest.raises(lib.AtkmError):
        plan.autotune()


def test_autotune_skips_power_of_two_plans(lib):
    plan = lib.Plan((32, 32, 16), (8.0, 8.0, 2.0), (0.0, 0.0, 1.0), f32=True)
    plan.autotune()
    assert plan.tuning() == []
