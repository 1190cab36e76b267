"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle on the
same seeded inputs.  Tolerances follow the arithmetic of each row:
  * U0 / K (FP64 precompute, two independent quadratures): 1e-12 relative to
    max|U0| (absolute in K, which is O(1));
  * Phi (FP64 FFT convolution): ||dPhi||_2 / ||Phi||_2 <= 1e-11;
  * H f, P r (FP64 spectral operators): relative 2-norm <= 1e-12;
  * energies and mu: relative <= 1e-10 (full PCG runs), 1e-12 for a fixed state.
"""
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


SMALL_CASES = [
    # (N, L, n): several tiles, ragged tails, radix 2/3/5 mixes, tilted axes
    ((32, 32, 16), (8.0, 8.0, 2.0), (0.0, 0.0, 1.0)),
    ((24, 20, 12), (5.0, 4.0, 1.2), (0.6, 0.0, 0.8)),
    ((40, 36, 10), (6.0, 5.5, 1.0), (0.5, 0.5, math.sqrt(0.5))),
    ((6, 4, 2), (1.0, 0.8, 0.5), (1.0, 0.0, 0.0)),
    ((96, 80, 18), (10.0, 9.0, 1.5), (0.0, 0.6, 0.8)),
]


@pytest.mark.parametrize("N,L,n", SMALL_CASES)
def test_U0_and_multiplier_match_oracle(lib, N, L, n):
    plan = lib.Plan(N, L, n)
    U0 = host(plan.U0())
    ref = O.truncated_coulomb_fourier(N, L)
    assert np.max(np.abs(U0 - ref)) <= 1e-12 * np.max(np.abs(ref))
    K = host(plan.multiplier())
    Kref = O.dipolar_multiplier(N, L, n, ref)
    assert np.max(np.abs(K - Kref)) <= 1e-11


@pytest.mark.parametrize("N,L,n", SMALL_CASES)
def test_dipolar_potential_parity(lib, N, L, n):
    plan = lib.Plan(N, L, n)
    oplan = O.Plan(N, L, n)
    shape = (N[2], N[1], N[0])
    # smooth density and a white-noise density (stresses every frequency)
    rho_s = np.abs(W.random_smooth_field(N, L, (1.0, 1.1, 5.0), seed=101)) ** 2
    rho_w = W.random_field(shape, 102, complex_valued=False)
    for rho in (rho_s, rho_w):
        got = host(plan.dipolar_potential(dev(rho)))
        ref = oplan.dipolar_potential(rho)
        assert rel2(got, ref) <= 1e-11
    psi = W.random_smooth_field(N, L, (1.0, 1.1, 5.0), seed=103)
    got = host(plan.dipolar_potential_from_psi(dev(psi)))
    assert rel2(got, oplan.dipolar_potential(np.abs(psi) ** 2)) <= 1e-11
    a = W.random_field(shape, 104)
    b = W.random_field(shape, 105)
    got = host(plan.dipolar_potential_from_pair(dev(a), dev(b)))
    assert rel2(got, oplan.dipolar_potential(np.real(np.conj(a) * b))) <= 1e-11


def test_dipolar_potential_gaussian_closed_form(lib):
    """Standalone check of the 32x32x16 workload family: isotropic sigma=1
    Gaussian on [-8,8]^3 at 64^3 against the exact dipolar potential."""
    from tests.test_oracle_kernel import iso_gaussian_dipolar
    N, L = (64, 64, 64), (8.0, 8.0, 8.0)
    n = (0.0, 0.0, 1.0)
    rho, _, Phi = iso_gaussian_dipolar(N, L, n)
    plan = lib.Plan(N, L, n)
    got = host(plan.dipolar_potential(dev(rho)))
    assert np.max(np.abs(got - Phi)) <= 1e-12 * np.max(np.abs(Phi))


def _state(N, L, gamma, seed):
    phi = W.random_smooth_field(N, L, gamma, seed=seed)
    h3 = np.prod([2 * L[i] / N[i] for i in range(3)])
    return phi / math.sqrt(h3 * np.sum(np.abs(phi) ** 2))


@pytest.mark.parametrize("N,L,n", SMALL_CASES)
def test_apply_H_energy_and_preconditioner_parity(lib, N, L, n):
    _check_H_energy_P(lib, N, L, n)


# Unpadded line lengths 16 ... 1024 of the fast engine in each axis role of
# the H and preconditioner passes (x: N_x, y: N_y, z: N_z).
H_FAST_LENGTH_GRIDS = [(1024, 16, 32), (32, 1024, 16), (16, 32, 1024), (512, 64, 16), (16, 512, 64),
                       (64, 16, 512), (128, 256, 16), (16, 16, 256), (32, 32, 128)]


@pytest.mark.parametrize("N", H_FAST_LENGTH_GRIDS)
def test_H_and_preconditioner_every_fast_length(lib, N):
    _check_H_energy_P(lib, N, (4.0, 3.0, 2.0), (0.6, 0.0, 0.8))


def _check_H_energy_P(lib, N, L, n):
    gamma, beta, lam, Om = (1.0, 1.3, 6.0), 40.0, -12.0, 0.55
    plan = lib.Plan(N, L, n)
    oplan = O.Plan(N, L, n)
    oprm = O.Params(gamma, beta, lam, Om)
    prm = lib.make_params(gamma, beta, lam, Om)
    phi = _state(N, L, gamma, 201)
    f = W.random_field(oplan.grid.shape, 202)
    Phi = oplan.dipolar_potential(np.abs(phi) ** 2)
    Hf = host(plan.apply_H(prm, dev(f), dev(phi), dev(Phi)))
    assert rel2(Hf, O.apply_H(oplan, oprm, f, phi, Phi)) <= 1e-12
    e = plan.energy_parts(prm, dev(phi), dev(Phi))
    p = O.energy_parts(oplan, oprm, phi, Phi)
    scale = abs(p["E"]) + abs(p["E_kin"]) + abs(p["E_pot"])
    for k in ("E", "E_kin", "E_pot", "E_int", "E_dip", "E_rot", "virial"):
        assert abs(e[k] - p[k]) <= 1e-12 * scale, k
    mu = O.inner(O.apply_H(oplan, oprm, phi, phi, Phi), phi, oplan.grid)
    assert abs(e["mu"] - mu) <= 1e-12 * abs(mu)
    alpha = O.precond_shift(oplan, oprm, phi, Phi)
    Pr = host(plan.apply_preconditioner(prm, alpha, dev(f), dev(phi), dev(Phi)))
    assert rel2(Pr, O.apply_precond(oplan, oprm, f, phi, Phi, alpha)) <= 1e-12


def _run_pair(lib, w, max_iter, tol=1e-8, precision=0):
    plan = lib.Plan(w.N, w.L, w.n, f32=(precision != 0), df32=(precision == 3))
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    psi = dev(W.initial_guess(w))
    res = plan.pcg_ground_state(prm, psi, tol_residual=tol, max_iter=max_iter, log_capacity=max_iter + 2,
                                precision=precision)
    return plan, psi, res


@pytest.fixture(scope="module")
def cfg1_oracle():
    w = W.CONFIGS["cfg1_32x32x16"]
    oplan = O.Plan(w.N, w.L, w.n)
    oprm = O.Params(w.gamma, w.beta, w.lam, w.Omega)
    return w, O.pcg_ground_state(oplan, oprm, W.initial_guess(w), O.PcgOptions(max_iter=400))


def test_pcg_cfg1_full_run_parity(lib, cfg1_oracle):
    w, ref = cfg1_oracle
    plan, psi, res = _run_pair(lib, w, 400)
    assert res["status"] == 0 and ref.status == O.OK
    assert res["residual"] <= 1e-8
    assert abs(res["E"] - ref.parts["E"]) <= 1e-10 * abs(ref.parts["E"])
    assert abs(res["mu"] - ref.mu) <= 1e-10 * abs(ref.mu)
    # trajectory: energies agree while they are well above roundoff
    for a, b in zip(res["log"][:20], ref.log[:20]):
        assert abs(a["E"] - b["E"]) <= 1e-10 * abs(b["E"])
    # final states agree up to a global phase
    phi = host(psi)
    kappa = np.vdot(ref.phi, phi) / np.vdot(ref.phi, ref.phi)
    assert np.linalg.norm(phi - kappa * ref.phi) / np.linalg.norm(ref.phi) <= 1e-6


def test_pcg_harmonic_oscillator(lib):
    N, L = (32, 32, 32), (8.0, 8.0, 4.0)
    plan = lib.Plan(N, L, (0, 0, 1))
    prm = lib.make_params((1.0, 1.0, 4.0), 0.0, 0.0, 0.0)
    psi = dev(W.random_smooth_field(N, L, (0.8, 0.9, 3.0), seed=7))
    res = plan.pcg_ground_state(prm, psi, tol_residual=1e-10, max_iter=500)
    assert res["status"] == 0
    assert abs(res["E"] - 3.0) < 1e-10 and abs(res["mu"] - 3.0) < 1e-10


def test_pcg_invariants_along_run(lib):
    w = W.CONFIGS["cfg1_32x32x16"]
    plan, psi, res = _run_pair(lib, w, 400)
    Es = [e["E"] for e in res["log"]]
    for a, b in zip(Es, Es[1:]):
        assert b <= a + 32 * np.finfo(float).eps * abs(a)
    # mu - E identity and unit norm of the final state
    assert abs(res["mu"] - (res["E"] + res["E_int"] + res["E_dip"])) <= 1e-12 * abs(res["mu"])
    h3 = np.prod([2 * w.L[i] / w.N[i] for i in range(3)])
    assert abs(h3 * float(torch.sum(torch.abs(psi) ** 2)) - 1.0) < 1e-13


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_mixed_precision_reaches_fp64_energy(lib, precision):
    """FP32 bulk then FP64 polish (1), the split polish with FP32
    direction/step-model operators (2), and that polish with H phi and the
    trial ATKM in double-word arithmetic (3): the same FP64 ground state."""
    w = W.CONFIGS["cfg1_32x32x16"]
    _, _, r64 = _run_pair(lib, w, 400)
    _, _, rmx = _run_pair(lib, w, 400, precision=precision)
    assert rmx["status"] == 0 and rmx["residual"] <= 1e-8
    assert rmx["f32_iters"] > 0
    assert abs(rmx["E"] - r64["E"]) <= 1e-9 * abs(r64["E"])
    assert abs(rmx["mu"] - r64["mu"]) <= 1e-9 * abs(r64["mu"])


@pytest.mark.parametrize("precision", [2, 3])
def test_split_precision_matches_oracle_ground_state(lib, precision):
    """The split form on a tilted-dipole anisotropic case against the FP64
    oracle's Algorithm 1: E and mu within 1e-10 relative."""
    N, L, n = (24, 20, 12), (5.0, 4.0, 1.2), (0.6, 0.0, 0.8)
    gamma, beta, lam, Om = (1.0, 1.3, 6.0), 40.0, -12.0, 0.3
    psi0 = W.guess_phi_d(N, L, gamma, Om)
    ref = O.pcg_ground_state(O.Plan(N, L, n), O.Params(gamma, beta, lam, Om), psi0,
                             O.PcgOptions(tol_residual=1e-9, max_iter=600))
    plan = lib.Plan(N, L, n, f32=True, df32=(precision == 3))
    psi = dev(psi0)
    r = plan.pcg_ground_state(lib.make_params(gamma, beta, lam, Om), psi, tol_residual=1e-9, max_iter=600,
                              precision=precision)
    assert ref.status == O.OK and r["status"] == 0
    assert abs(r["E"] - ref.parts["E"]) <= 1e-10 * abs(ref.parts["E"])
    assert abs(r["mu"] - ref.mu) <= 1e-10 * abs(ref.mu)


@pytest.mark.parametrize("N,L,n", SMALL_CASES)
def test_df32_atkm_matches_oracle(lib, N, L, n):
    """Double-word (double-FP32) ATKM: same 1e-11 bar as the FP64 path; the
    arithmetic carries about 48 bits (observed 5e-15 - 8e-15 relative)."""
    plan = lib.Plan(N, L, n, df32=True)
    oplan = O.Plan(N, L, n)
    psi = W.random_smooth_field(N, L, (1.0, 1.1, 5.0), seed=103)
    got = host(plan.dipolar_potential_from_psi(dev(psi), df32=True))
    assert rel2(got, oplan.dipolar_potential(np.abs(psi) ** 2)) <= 1e-11
    a = W.random_field((N[2], N[1], N[0]), 104)
    got = host(plan.dipolar_potential_from_psi(dev(a), df32=True))
    assert rel2(got, oplan.dipolar_potential(np.abs(a) ** 2)) <= 1e-11
    with pytest.raises(lib.AtkmError):
        lib.Plan(N, L, n).dipolar_potential_from_psi(dev(psi), df32=True)


# Every power-of-two line length of the fast FFT engine (16 ... 1024) in each
# role: x pass L = N_x, y pass L = 2 N_y, z pass L = 2 N_z.  The ATKM passes
# skip the zero upper half of a forward transform's input and form only the
# lower half of a cropped inverse transform's output; the stage structure
# (one to three radix-8 stages, then a radix-2 or radix-4 tail or none)
# differs between these lengths.
FAST_LENGTH_CASES = [
    ((1024, 16, 32), (0.6, 0.0, 0.8)),   # x 1024, y 32, z 64
    ((512, 32, 8), (0.5, 0.5, math.sqrt(0.5))),  # x 512, y 64, z 16
    ((256, 16, 128), (0.0, 0.6, 0.8)),   # x 256, y 32, z 256
    ((128, 512, 8), (0.6, 0.0, 0.8)),    # x 128, y 1024, z 16
    ((64, 256, 16), (0.5, 0.5, math.sqrt(0.5))),  # x 64, y 512, z 32
    ((32, 128, 64), (0.0, 0.0, 1.0)),    # x 32, y 256, z 128
    ((16, 64, 256), (0.6, 0.0, 0.8)),    # x 16, y 128, z 512
    ((16, 8, 512), (0.5, 0.5, math.sqrt(0.5))),  # x 16, y 16, z 1024
]


@pytest.mark.parametrize("N,n", FAST_LENGTH_CASES)
def test_atkm_every_fast_length_matches_oracle(lib, N, n):
    L = (4.0, 3.0, 2.0)
    plan = lib.Plan(N, L, n, f32=True, df32=True)
    oplan = O.Plan(N, L, n)
    shape = (N[2], N[1], N[0])
    psi = W.random_smooth_field(N, L, (1.0, 1.3, 2.0), seed=401)
    white = W.random_field(shape, 402)
    for f in (psi, white):
        ref = oplan.dipolar_potential(np.abs(f) ** 2)
        assert rel2(host(plan.dipolar_potential_from_psi(dev(f))), ref) <= 1e-11
        assert rel2(host(plan.dipolar_potential_from_psi(dev(f), df32=True)), ref) <= 1e-11
        assert rel2(host(plan.dipolar_potential_from_psi(dev(f), f32=True)), ref) <= 5e-6
    b = W.random_field(shape, 403)
    got = host(plan.dipolar_potential_from_pair(dev(white), dev(b)))
    assert rel2(got, oplan.dipolar_potential(np.real(np.conj(white) * b))) <= 1e-11


def test_f32_atkm_close_to_oracle(lib):
    N, L, n = (32, 32, 16), (8.0, 8.0, 2.0), (0.6, 0.0, 0.8)
    plan = lib.Plan(N, L, n, f32=True)
    psi = W.random_smooth_field(N, L, (1.0, 1.1, 5.0), seed=301)
    got = host(plan.dipolar_potential_from_psi(dev(psi), f32=True))
    ref = O.Plan(N, L, n).dipolar_potential(np.abs(psi) ** 2)
    assert rel2(got, ref) <= 2e-6


@pytest.mark.parametrize("N,L,n,code", [
    ((31, 32, 16), (8, 8, 2), (0, 0, 1), 2),      # odd
    ((28, 32, 16), (8, 8, 2), (0, 0, 1), 2),      # factor 7
    ((32, 32, 16), (8, 8, 2), (0, 0, 1.001), 1),  # |n| != 1
    ((32, 32, 16), (8, -8, 2), (0, 0, 1), 1),     # negative box
    ((2048, 32, 16), (8, 8, 2), (0, 0, 1), 2),    # beyond the line limit
])
def test_plan_rejects_bad_arguments(lib, N, L, n, code):
    with pytest.raises(lib.AtkmError) as ei:
        lib.Plan(N, L, n)
    assert ei.value.code == code


def test_smallest_grid_and_degenerate_inputs(lib):
    N, L, n = (2, 2, 2), (1.0, 1.0, 1.0), (0, 0, 1)
    plan = lib.Plan(N, L, n)
    oplan = O.Plan(N, L, n)
    rho = W.random_field((2, 2, 2), 401, complex_valued=False)
    assert rel2(host(plan.dipolar_potential(dev(rho))), oplan.dipolar_potential(rho)) <= 1e-11
    # zero density gives a zero potential; a zero initial state is rejected
    z = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    assert float(plan.dipolar_potential(z).abs().max()) == 0.0
    prm = lib.make_params((1, 1, 1), 0, 0, 0)
    psi0 = torch.zeros((2, 2, 2), dtype=torch.complex128, device="cuda")
    res = plan.pcg_ground_state(prm, psi0, check=False)
    assert res["status"] == 7


@pytest.mark.slow
def test_cfg3_dipolar_potential_full_size(lib):
    """256x256x64 (the bench grid): full ATKM against the oracle, FP64 and FP32."""
    w = W.CONFIGS["cfg3_256x256x64"]
    plan = lib.Plan(w.N, w.L, w.n, f32=True)
    psi = W.initial_guess(w)
    ref = O.Plan(w.N, w.L, w.n).dipolar_potential(np.abs(psi) ** 2)
    got = host(plan.dipolar_potential_from_psi(dev(psi)))
    assert rel2(got, ref) <= 1e-11
    got32 = host(plan.dipolar_potential_from_psi(dev(psi), f32=True))
    assert rel2(got32, ref) <= 2e-6


def test_graph_replay_is_bitwise_identical_to_direct_launches(lib):
    w = W.CONFIGS["cfg2_128x128x32"]
    plan = lib.Plan(w.N, w.L, w.n, f32=True)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    outs = []
    for graphs in (True, False):
        for prec in (0, 1):
            psi = dev(W.initial_guess(w))
            r = plan.pcg_ground_state(prm, psi, max_iter=12, precision=prec, graphs=graphs, log_capacity=20)
            outs.append((graphs, prec, host(psi), [l["E"] for l in r["log"]]))
    for prec in (0, 1):
        a = [o for o in outs if o[0] and o[1] == prec][0]
        b = [o for o in outs if not o[0] and o[1] == prec][0]
        assert np.array_equal(a[2], b[2])
        assert a[3] == b[3]


def test_resume_continues_the_same_solve(lib):
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = lib.Plan(w.N, w.L, w.n)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    psi1 = dev(W.initial_guess(w))
    r1 = plan.pcg_ground_state(prm, psi1, max_iter=20, tol_residual=0.0)
    psi2 = dev(W.initial_guess(w))
    plan.pcg_ground_state(prm, psi2, max_iter=8, tol_residual=0.0)
    r2 = plan.pcg_ground_state(prm, psi2, max_iter=12, tol_residual=0.0, resume=True)
    assert r2["iters"] == 20 == r1["iters"]
    assert np.array_equal(host(psi1), host(psi2))
    assert r1["E"] == r2["E"]


def test_batched_sweep_matches_single_instance_solves(lib):
    """Uneven grids (radix 2 and 3, fast and generic engines) and different
    rotation speeds in one batched call: each instance equals its own solve."""
    cases = [((32, 32, 16), (8.0, 8.0, 2.0), 0.40), ((24, 24, 12), (6.0, 6.0, 1.5), 0.55),
             ((48, 40, 16), (8.0, 7.0, 2.0), 0.70), ((20, 30, 10), (5.0, 6.0, 1.5), 0.30)]
    gamma, beta, lam, n = (1.0, 1.0, 4.0), 40.0, 12.0, (0.0, 0.0, 1.0)
    plans, prms, psis, refs = [], [], [], []
    for N, L, Om in cases:
        plans.append(lib.Plan(N, L, n))
        prms.append(lib.make_params(gamma, beta, lam, Om))
        psis.append(dev(W.guess_phi_d(N, L, gamma, Om)))
    for pl, pr, (N, L, Om) in zip(plans, prms, cases):
        solo = lib.Plan(N, L, n)
        ps = dev(W.guess_phi_d(N, L, gamma, Om))
        r = solo.pcg_ground_state(pr, ps, max_iter=80)
        refs.append((host(ps), r))
    outs = lib.pcg_ground_state_batched(plans, prms, psis, max_iter=80)
    for (ref_psi, ref_r), ps, o in zip(refs, psis, outs):
        assert o["status"] == ref_r["status"] and o["iters"] == ref_r["iters"]
        assert o["E"] == ref_r["E"]
        assert np.array_equal(host(ps), ref_psi)


def test_batched_rejects_shared_plan(lib):
    plan = lib.Plan((8, 8, 4), (2.0, 2.0, 1.0), (0, 0, 1))
    prm = lib.make_params((1, 1, 1), 1.0, 0.0, 0.0)
    a = dev(W.guess_phi_d((8, 8, 4), (2.0, 2.0, 1.0), (1, 1, 1), 0.0))
    b = a.clone()
    with pytest.raises(lib.AtkmError):
        lib.pcg_ground_state_batched([plan, plan], [prm, prm], [a, b], max_iter=2)


def test_profiling_over_graph_replay(lib):
    """Per-pass CUDA-event timing works on the captured-graph path and does
    not change results."""
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = lib.Plan(w.N, w.L, w.n, f32=True)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    ref = dev(W.initial_guess(w))
    r0 = plan.pcg_ground_state(prm, ref, max_iter=6, precision=1)
    psi = dev(W.initial_guess(w))
    plan.set_profiling(True)
    r1 = plan.pcg_ground_state(prm, psi, max_iter=6, precision=1)
    stats = {s["name"]: s for s in plan.kernel_stats()}
    plan.set_profiling(False)
    assert np.array_equal(host(psi), host(ref)) and r0["E"] == r1["E"]
    z = stats["atkm_z_f32"]
    assert z["launches"] >= 12 and z["ms_total"] > 0 and z["bytes_total"] > 0
    assert stats["H_x_f32"]["launches"] >= 6
