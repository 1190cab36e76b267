"""Pins of the learned-guess oracle (network, loss, gradient) and of the
spectral upsampling (Fourier interpolant of §2.1 evaluated on a finer grid).

The network oracle is checked against library routines it does not use
(torch's conv_transpose3d and autograd), against central finite differences,
and against invariants of the loss; the upsampler against band-limited fields
whose fine-grid values are known in closed form.
"""
import math

import numpy as np
import pytest
import torch

import atkm_workloads as W
from oracle import guess_net as GN


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    fan = {"W1": GN.F, "W2": GN.H, "W3": GN.C0, "W4": GN.C1, "W5": GN.C2}
    for name, shape in GN.SHAPES:
        if name.startswith("W"):
            a = scale * math.sqrt(3.0 / fan[name])
            w = rng.uniform(-a, a, size=shape)
            if name == "W1":
                w[GN.F:, :] = 0.0
        else:
            w = rng.uniform(-0.1, 0.1, size=shape)
        parts.append(w.ravel())
    return np.concatenate(parts)


def _feats(B, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=(B, GN.F))


def _targets(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B,) + GN.OUT) + 1j * rng.standard_normal((B,) + GN.OUT)


def test_bf16_round_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(GN.bf16_round(x), ref)
    one = np.float32(1.0)
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)], dtype=np.float32)
    assert np.array_equal(GN.bf16_round(ties), np.array([one, 1 + 2.0 ** -6, -one], dtype=np.float32))


def _torch_net(params, feats):
    """The same network written with torch's conv_transpose3d (weights
    (C_in, C_out, k_z, k_y, k_x), stride = kernel)."""
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in GN.unpack(params, np.float64).items()}
    B = feats.shape[0]
    f = torch.zeros(B, GN.FPAD, dtype=torch.float64)
    f[:, :GN.F] = torch.tensor(feats)
    F = torch.nn.functional
    h1 = F.relu(f @ P["W1"] + P["b1"])
    z = h1 @ P["W2"] + P["b2"]
    x0 = z.reshape(B, 4, 8, 8, GN.C0).permute(0, 4, 1, 2, 3)
    w1 = P["W3"].reshape(GN.C0, 2, 2, 2, GN.C1).permute(0, 4, 1, 2, 3)
    x1 = F.relu(F.conv_transpose3d(x0, w1, P["b3"], stride=2))
    w2 = P["W4"].reshape(GN.C1, 2, 2, 2, GN.C2).permute(0, 4, 1, 2, 3)
    x2 = F.relu(F.conv_transpose3d(x1, w2, P["b4"], stride=2))
    w3 = P["W5"].reshape(GN.C2, 1, 2, 2, GN.C3).permute(0, 4, 1, 2, 3)
    x3 = F.conv_transpose3d(x2, w3, P["b5"], stride=(1, 2, 2))
    return P, x3


def test_forward_equals_transposed_convolutions():
    params, feats = _params(1), _feats(3, 2)
    a = GN.forward(params, feats, bf16=False)
    psi = GN.out_to_psi(a["o"], 3)
    _, x3 = _torch_net(params, feats)
    ref = x3[:, 0].detach().numpy() + 1j * x3[:, 1].detach().numpy()
    assert psi.shape == ref.shape == (3,) + GN.OUT
    assert np.max(np.abs(psi - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_out_index_is_a_bijection():
    B = 2
    b, z, y, x, ch = GN.out_index(B)
    flat = ((((b * GN.OUT[0] + z) * GN.OUT[1] + y) * GN.OUT[2] + x) * 2 + ch).ravel()
    assert np.array_equal(np.sort(flat), np.arange(B * np.prod(GN.OUT) * 2))


def test_gradient_equals_autograd():
    params, feats, t = _params(3), _feats(2, 4), _targets(2, 5)
    loss, grad = GN.loss_and_grad(params, feats, t, bf16=False)
    P, x3 = _torch_net(params, feats)
    tr, ti = torch.tensor(t.real), torch.tensor(t.imag)
    ur, ui = x3[:, 0], x3[:, 1]
    sr = (ur * tr + ui * ti).sum(dim=(1, 2, 3))
    si = (ui * tr - ur * ti).sum(dim=(1, 2, 3))
    uu = (ur * ur + ui * ui).sum(dim=(1, 2, 3))
    tt = (tr * tr + ti * ti).sum(dim=(1, 2, 3))
    L = (1.0 - (sr * sr + si * si) / (uu * tt)).mean()
    L.backward()
    assert abs(loss - L.item()) < 1e-13
    ref = GN.pack({k: v.grad.numpy() for k, v in P.items()})
    # padded rows of W1 see zero features: their gradient is zero on both sides
    for (name, shape), lo in zip(GN.SHAPES, np.cumsum([0] + [int(np.prod(s)) for _, s in GN.SHAPES])):
        n = int(np.prod(shape))
        g, r = grad[lo:lo + n], ref[lo:lo + n]
        assert np.linalg.norm(g - r) <= 1e-10 * max(np.linalg.norm(r), 1e-300), name


def test_gradient_equals_finite_differences():
    params, feats, t = _params(6), _feats(2, 7), _targets(2, 8)
    _, grad = GN.loss_and_grad(params, feats, t, bf16=False)
    rng = np.random.default_rng(9)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in GN.SHAPES])
    for k, (name, shape) in enumerate(GN.SHAPES):
        lo, hi = offs[k], offs[k + 1]
        if name == "W1":
            hi = lo + GN.F * GN.H  # the live rows
        for i in rng.integers(lo, hi, size=3):
            h = 1e-7
            p1, p2 = params.copy(), params.copy()
            p1[i] += h
            p2[i] -= h
            fd = (GN.loss(p1, feats, t, bf16=False) - GN.loss(p2, feats, t, bf16=False)) / (2 * h)
            # ReLU kinks crossed inside [-h, h] and FP64 cancellation bound the agreement
            assert abs(fd - grad[i]) <= 1e-3 * abs(fd) + 1e-8, (name, i, fd, grad[i])


def test_loss_is_phase_and_scale_invariant_and_zero_at_target():
    params, feats = _params(10), _feats(2, 11)
    a = GN.forward(params, feats, bf16=False)
    u = GN.out_to_psi(a["o"], 2)
    t = u * np.array([2.5 * np.exp(0.7j), 0.3 * np.exp(-2.1j)])[:, None, None, None]
    loss, grad = GN.loss_and_grad(params, feats, t, bf16=False)
    assert abs(loss) < 1e-14
    assert np.max(np.abs(grad)) < 1e-12
    t2 = _targets(2, 12)
    l1 = GN.loss(params, feats, t2, bf16=False)
    l2 = GN.loss(params, feats, t2 * np.exp(1.3j) * 7.0, bf16=False)
    assert 0.0 < l1 < 1.0 and abs(l1 - l2) < 1e-13


def test_bf16_network_is_close_to_fp64_network():
    params, feats, t = _params(13), _feats(2, 14), _targets(2, 15)
    a64 = GN.out_to_psi(GN.forward(params, feats, bf16=False)["o"], 2)
    a16 = GN.out_to_psi(GN.forward(params, feats, bf16=True)["o"], 2)
    rel = np.linalg.norm(a16 - a64) / np.linalg.norm(a64)
    assert 1e-5 < rel < 3e-2  # BF16 operands: a few 2^-9 relative errors per layer
    _, g64 = GN.loss_and_grad(params, feats, t, bf16=False)
    _, g16 = GN.loss_and_grad(params, feats, t, bf16=True)
    assert np.linalg.norm(g16 - g64) < 0.1 * np.linalg.norm(g64)


# ---------------------------------------------------------------- upsampling

def _trig_poly(N, L, modes):
    x, y, z = W.mesh(N, L)
    f = np.zeros((N[2], N[1], N[0]), dtype=np.complex128)
    for (kx, ky, kz, c) in modes:
        f = f + c * np.exp(1j * math.pi * (kx * (x + L[0]) / L[0] + ky * (y + L[1]) / L[1] + kz * (z + L[2]) / L[2]))
    return f


def test_upsample_exact_on_band_limited_fields():
    Nc, Nf, L = (12, 10, 6), (24, 30, 12), (3.0, 2.0, 1.0)
    rng = np.random.default_rng(16)
    modes = [(int(rng.integers(-5, 6)), int(rng.integers(-4, 5)), int(rng.integers(-2, 3)),
              complex(rng.standard_normal(), rng.standard_normal())) for _ in range(12)]
    fc, ff = _trig_poly(Nc, L, modes), _trig_poly(Nf, L, modes)
    up = GN.spectral_upsample(fc, Nf)
    assert np.max(np.abs(up - ff)) < 1e-12 * np.max(np.abs(ff))


def test_upsample_identity_and_norm():
    Nc, L = (8, 6, 4), (2.0, 2.0, 1.0)
    f = W.random_field((Nc[2], Nc[1], Nc[0]), 17)
    assert np.max(np.abs(GN.spectral_upsample(f, Nc) - f)) < 1e-13
    Nf = (16, 18, 8)
    up = GN.spectral_upsample(f, Nf)
    hc = np.prod([2 * L[a] / Nc[a] for a in range(3)])
    hf = np.prod([2 * L[a] / Nf[a] for a in range(3)])
    assert abs(hf * np.sum(np.abs(up) ** 2) - hc * np.sum(np.abs(f) ** 2)) < 1e-12 * hc * np.sum(np.abs(f) ** 2)
    # coarse points are fine points (the fine grid refines by integers): values agree there
    assert np.max(np.abs(up[::2, ::3, ::2] - f)) < 1e-12


def test_upsample_keeps_the_coarse_nyquist_mode_unsplit():
    """The coarse coefficient of k = -N/2 goes to fine k = -N/2 whole."""
    Nc, Nf, L = (8, 4, 4), (16, 8, 8), (1.0, 1.0, 1.0)
    f = _trig_poly(Nc, L, [(-4, 0, 0, 1.0)])  # (-1)^j along x: real on the coarse grid
    assert np.max(np.abs(f.imag)) < 1e-13
    up = GN.spectral_upsample(f, Nf)
    assert np.max(np.abs(up - _trig_poly(Nf, L, [(-4, 0, 0, 1.0)]))) < 1e-12
