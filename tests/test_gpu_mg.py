"""GPU parity of the cascadic multigrid driver (Algorithm 2) through the
C-ABI against the oracle's: per-level energies within 1e-10 relative (the
same tolerance as every full PCG run; each level's ground state is unique
below the critical rotation)."""
import numpy as np
import pytest
import torch

import atkm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu

L, GAMMA, NAX = (8.0, 8.0, 2.0), (1.0, 1.0, 4.0), (0.0, 0.0, 1.0)
GRIDS = [(8, 8, 4), (16, 16, 8), (32, 32, 16)]


@pytest.mark.parametrize("precision", [0, 1])
def test_mg_matches_oracle(lib, precision):
    prm_o = O.Params(GAMMA, 50.0, 15.0, 0.4)
    opts = O.PcgOptions(tol_residual=1e-9, max_iter=400)
    ref = O.pcg_ground_state_mg([O.Plan(N, L, NAX) for N in GRIDS], prm_o, W.guess_phi_d(GRIDS[0], L, GAMMA, 0.4),
                                opts)
    plans = [lib.Plan(N, L, NAX, f32=True) for N in GRIDS]
    psis = [torch.from_numpy(W.guess_phi_d(GRIDS[0], L, GAMMA, 0.4)).cuda()] + \
           [torch.zeros(p.shape, dtype=torch.complex128, device="cuda") for p in plans[1:]]
    out = lib.pcg_ground_state_mg(plans, lib.make_params(GAMMA, 50.0, 15.0, 0.4), psis, tol_residual=1e-9,
                                  max_iter=400, precision=precision)
    assert [r["status_name"] for r in out] == ["OK"] * 3
    for r, o in zip(out, ref):
        assert abs(r["E"] - o.parts["E"]) <= 1e-10 * abs(o.parts["E"])
        assert abs(r["mu"] - o.mu) <= 1e-10 * abs(o.mu)
        assert r["residual"] <= 1e-9
    # the finest state is the oracle's up to a global phase
    g = O.Grid(GRIDS[-1], L)
    a, b = psis[-1].cpu().numpy(), ref[-1].phi
    ov = abs(O.inner(a, b, g) + 1j * O.inner(a, 1j * b, g))
    assert abs(ov - 1.0) < 1e-8


def test_mg_rejects_bad_levels(lib):
    p1 = lib.Plan((16, 16, 8), L, NAX)
    p0 = lib.Plan((8, 8, 4), L, NAX)
    a = torch.zeros(p1.shape, dtype=torch.complex128, device="cuda")
    b = torch.zeros(p0.shape, dtype=torch.complex128, device="cuda")
    prm = lib.make_params(GAMMA, 50.0, 15.0, 0.4)
    with pytest.raises(lib.AtkmError):
        lib.pcg_ground_state_mg([p1, p0], prm, [a, b], max_iter=2)   # coarser
    with pytest.raises(lib.AtkmError):
        lib.pcg_ground_state_mg([p1, p1], prm, [a, a], max_iter=2)   # same plan


def test_mg_f64_levels(lib):
    """mg_f64_levels: with a precision form, the coarsest levels run in FP64
    (bitwise the FP64 cascade's levels, no FP32 iterations there), the rest in
    the form; every level ends at the oracle's energy."""
    prm = lib.make_params(GAMMA, 50.0, 15.0, 0.4)

    def run(precision, **kw):
        plans = [lib.Plan(N, L, NAX, f32=True) for N in GRIDS]
        psis = [torch.from_numpy(W.guess_phi_d(GRIDS[0], L, GAMMA, 0.4)).cuda()] + \
               [torch.zeros(p.shape, dtype=torch.complex128, device="cuda") for p in plans[1:]]
        return lib.pcg_ground_state_mg(plans, prm, psis, tol_residual=1e-9, max_iter=400, precision=precision,
                                       **kw), psis

    f64, p64 = run(0)
    mix, pmix = run(1, mg_f64_levels=2)
    assert [r["f32_iters"] for r in mix][:2] == [0, 0] and mix[2]["f32_iters"] > 0
    for i in range(2):
        assert torch.equal(p64[i], pmix[i]) and mix[i]["E"] == f64[i]["E"] and mix[i]["iters"] == f64[i]["iters"]
    assert mix[2]["status_name"] == "OK" and abs(mix[2]["E"] - f64[2]["E"]) <= 1e-10 * abs(f64[2]["E"])
