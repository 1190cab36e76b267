"""GPU test of the allocation-free inner-product entry point.

Some callers cannot call cudaMalloc (a host framework that owns all device
memory, or a process whose device footprint is fixed after start-up).  For
them, atkm_inner_products_noalloc keeps its reduction scratch in a static
device array.  This checks it, through the C-ABI, against the existing entry
points: mu = <H phi, phi> and norm2 = <phi, phi> from atkm_energy_parts (with
H phi from apply_H), on two calls in a row with different inputs, so a stale
scratch from the first call would show up in the second.  The file sorts last
so a run that stops at the first failure has run every other test first.
"""
import math

import numpy as np
import pytest
import torch

import atkm_workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative, as the other FP64 parity tests of reductions


def _state(N, L, seed):
    phi = W.random_smooth_field(N, L, (1.0, 1.2, 5.0), seed=seed)
    h3 = np.prod([2 * L[i] / N[i] for i in range(3)])
    return phi / math.sqrt(h3 * np.sum(np.abs(phi) ** 2)), h3


def test_noalloc_inner_products_match_existing_entry_points(lib):
    N, L, n = (48, 40, 16), (6.0, 5.0, 1.5), (0.6, 0.0, 0.8)
    plan = lib.Plan(N, L, n)
    prm = lib.make_params((1.0, 1.2, 5.0), 30.0, -9.0, 0.4)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for seed in (11, 12):  # two calls in a row on different inputs
        phi_np, h3 = _state(N, L, seed)
        phi_np = phi_np * (1.0 + 0.25 * (seed - 11))  # different norms for the two calls
        phi = torch.from_numpy(phi_np).cuda()
        Phi = plan.dipolar_potential_from_psi(phi)
        Hphi = plan.apply_H(prm, phi, phi, Phi)
        ref = plan.energy_parts(prm, phi, Phi)
        lib.inner_products_noalloc([Hphi, phi, Hphi], [phi, phi, Hphi], h3, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref["mu"]) <= TOL * abs(ref["mu"])
        assert abs(got[1] - ref["norm2"]) <= TOL * abs(ref["norm2"])
        hh = float(h3 * torch.sum(torch.abs(Hphi) ** 2))
        assert abs(got[2] - hh) <= TOL * hh


def test_noalloc_rejects_too_many_pairs(lib):
    v = torch.zeros(8, dtype=torch.complex128, device="cuda")
    out = torch.empty(9, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.AtkmError) as ei:
        lib.inner_products_noalloc([v] * 9, [v] * 9, 1.0, out)
    assert ei.value.code == lib.ATKM_ERR_ARG
