"""GPU parity of the learned-guess network (BF16 operands, FP32 accumulation)
and of spectral upsampling, through the C-ABI, against the CPU oracle.

Tolerances: the oracle rounds the same operands to BF16 and stores the same
FP32 layer outputs, so the two sides differ only by FP32 summation (the
tensor cores' FP32 accumulation is not round-to-nearest, and split-K adds
partial tiles atomically in any order) and by the rare BF16 rounding or ReLU
decision that such a difference flips.  Relative 2-norm bounds: 2e-3 on psi
(four GEMMs, K <= 256); 5e-3 per parameter block of the gradient; 1e-2 for
W1 and b1, which sit behind all six backward GEMMs (K up to 8192, with
cancellation) and are summed over only B samples.  A wrong index or dropped
term anywhere moves a block by O(1).  Upsampling is FP64 FFT arithmetic:
1e-12 relative.
"""
import math

import numpy as np
import pytest
import torch

import atkm_workloads as W
from oracle import guess_net as GN

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _params(seed):
    rng = np.random.default_rng(seed)
    fan = {"W1": GN.F, "W2": GN.H, "W3": GN.C0, "W4": GN.C1, "W5": GN.C2}
    parts = []
    for name, shape in GN.SHAPES:
        if name.startswith("W"):
            a = math.sqrt(3.0 / fan[name])
            w = rng.uniform(-a, a, size=shape)
            if name == "W1":
                w[GN.F:, :] = 0.0
        else:
            w = rng.uniform(-0.1, 0.1, size=shape)
        parts.append(w.ravel())
    return np.concatenate(parts).astype(np.float32)


def _feats(B, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=(B, GN.F)).astype(np.float32)


def _targets(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B,) + GN.OUT) + 1j * rng.standard_normal((B,) + GN.OUT)


ENGINES = {"tcgen05": 0, "mma_sync": 1}


@pytest.mark.parametrize("engine", list(ENGINES))
@pytest.mark.parametrize("B", [1, 3, 33])
def test_forward_matches_oracle(lib, B, engine):
    net = lib.GuessNet(seed=1)
    net.set_gemm_engine(ENGINES[engine])
    p = _params(20 + B)
    net.set_params(dev(p))
    f = _feats(B, 30 + B)
    got = host(net.forward(dev(f)))
    ref = GN.out_to_psi(GN.forward(p, f, bf16=True)["o"], B)
    assert got.shape == ref.shape
    assert rel2(got, ref) <= 2e-3
    net.check()


@pytest.mark.parametrize("engine", list(ENGINES))
@pytest.mark.parametrize("B", [2, 5, 32])
def test_gradient_matches_oracle(lib, B, engine):
    net = lib.GuessNet(seed=2)
    net.set_gemm_engine(ENGINES[engine])
    p = _params(40 + B)
    net.set_params(dev(p))
    f, t = _feats(B, 50 + B), _targets(B, 60 + B)
    g, loss = net.grad(dev(f), dev(t))
    g = host(g).astype(np.float64)
    ref_loss, ref = GN.loss_and_grad(p, f, t, bf16=True)
    assert abs(float(host(loss)[0]) - ref_loss) <= 1e-4 * abs(ref_loss) + 1e-7
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in GN.SHAPES])
    errs = {}
    for k, (name, _) in enumerate(GN.SHAPES):
        a, b = g[offs[k]:offs[k + 1]], ref[offs[k]:offs[k + 1]]
        errs[name] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    tol = {name: (1e-2 if name in ("W1", "b1") else 5e-3) for name, _ in GN.SHAPES}
    assert all(errs[k] <= tol[k] for k in errs), errs
    net.check()


def test_tcgen05_and_mma_sync_engines_agree(lib):
    """The two engines round the same operands to BF16 and sum in FP32, so
    they differ only by summation order (and the rare BF16 rounding of a
    staged activation that it flips): forward outputs and every gradient
    block agree well inside the oracle bars, at the training batch (32) and at
    a ragged one (37), and the tensor-core waits all completed."""
    p = _params(77)
    for B in (32, 37):
        f, t = _feats(B, 78 + B), _targets(B, 79 + B)
        outs = {}
        for name, eng in ENGINES.items():
            net = lib.GuessNet(seed=5)
            net.set_gemm_engine(eng)
            net.set_params(dev(p))
            psi = host(net.forward(dev(f)))
            g, loss = net.grad(dev(f), dev(t))
            net.check()
            outs[name] = (psi, host(g).astype(np.float64), float(host(loss)[0]))
        a, b = outs["tcgen05"], outs["mma_sync"]
        assert rel2(a[0], b[0]) <= 5e-4
        assert abs(a[2] - b[2]) <= 1e-4 * abs(b[2])
        offs = np.cumsum([0] + [int(np.prod(s)) for _, s in GN.SHAPES])
        for k, (name, _) in enumerate(GN.SHAPES):
            x, y = a[1][offs[k]:offs[k + 1]], b[1][offs[k]:offs[k + 1]]
            assert np.linalg.norm(x - y) <= 2e-3 * max(np.linalg.norm(y), 1e-30), name


def test_tcgen05_wait_limit_reports_timeout_and_context_survives(lib):
    """Failure path of the tensor-core GEMMs without a fault: under
    ATKM_GEMM_TCGEN05_WAIT_TEST every tcgen05 GEMM waits (1000 polls) on a
    barrier that nothing completes, gives up before issuing any MMA and sets
    the network's flag; the host reads ATKM_ERR_TIMEOUT, the flag clears, and
    the next forward pass on the same context matches the oracle."""
    net = lib.GuessNet(seed=8)
    p = _params(81)
    net.set_params(dev(p))
    f = _feats(3, 82)
    net.set_gemm_engine(lib.ATKM_GEMM_TCGEN05_WAIT_TEST)
    net.forward(dev(f))
    with pytest.raises(lib.AtkmError) as ei:
        net.check()
    assert ei.value.code == lib.ATKM_ERR_TIMEOUT
    net.check()  # the flag was cleared
    net.set_gemm_engine(lib.ATKM_GEMM_TCGEN05)
    got = host(net.forward(dev(f)))
    ref = GN.out_to_psi(GN.forward(p, f, bf16=True)["o"], 3)
    assert rel2(got, ref) <= 2e-3
    net.check()


def test_gemm_engine_rejects_unknown_value(lib):
    net = lib.GuessNet(seed=6)
    with pytest.raises(lib.AtkmError):
        net.set_gemm_engine(7)


def test_init_and_param_roundtrip(lib):
    net = lib.GuessNet(seed=7)
    p = host(net.get_params())
    assert p.shape == (GN.NUM_PARAMS,) and net.num_params == GN.NUM_PARAMS
    P = GN.unpack(p)
    fan = {"W1": GN.F, "W2": GN.H, "W3": GN.C0, "W4": GN.C1, "W5": GN.C2}
    for name, _ in GN.SHAPES:
        if name.startswith("W"):
            a = math.sqrt(3.0 / fan[name])
            live = P[name][:GN.F] if name == "W1" else P[name]
            assert np.max(np.abs(live)) <= a * (1 + 1e-6) and np.std(live) > 0.4 * a
        else:
            assert not np.any(P[name])
    assert not np.any(P["W1"][GN.F:])
    # same seed, same parameters; set/get round-trips exactly
    assert np.array_equal(host(lib.GuessNet(seed=7).get_params()), p)
    q = _params(8)
    net.set_params(dev(q))
    assert np.array_equal(host(net.get_params()), q)


def test_first_adam_step_is_lr_times_gradient_sign(lib):
    """Adam's first step with bias correction: m_hat = g and v_hat = g^2, so
    each weight moves by lr g / (|g| + eps), eps = 1e-8."""
    net = lib.GuessNet(seed=4)
    p = _params(90)
    net.set_params(dev(p))
    B = 3
    f, t = _feats(B, 91), _targets(B, 92)
    lr = 1e-3
    net.train_step(dev(f), dev(t), lr)
    step = p.astype(np.float64) - host(net.get_params()).astype(np.float64)
    _, g = GN.loss_and_grad(p, f, t, bf16=True)
    expect = lr * g / (np.abs(g) + 1e-8)
    # where |g| is not tiny the GPU/oracle gradient difference is a small
    # relative error, and the step's sensitivity to it is at most a quarter
    big = np.abs(g) > 1e-2 * np.max(np.abs(g))
    assert big.sum() > 1000
    assert np.max(np.abs(step[big] - expect[big])) <= 5e-3 * lr + 1e-7
    assert np.all(np.abs(step) <= lr * (1 + 1e-3) + 1e-7)


def test_training_reduces_loss(lib):
    """Adam steps on one batch of smooth targets lower the loss."""
    net = lib.GuessNet(seed=3)
    B = 4
    f = dev(_feats(B, 70))
    N, L = (64, 64, 16), (16.0, 16.0, 1.5)
    t = np.stack([W.guess_phi_d(N, L, (1.0, 1.0, 10.0 + 5 * i), 0.3 + 0.1 * i) for i in range(B)])
    t = dev(t)
    losses = [float(host(net.train_step(f, t, 1e-3))[0]) for _ in range(60)]
    assert losses[-1] < 0.8 * losses[0]
    assert min(losses[-10:]) < min(losses[:10])


def test_bad_arguments(lib):
    net = lib.GuessNet(seed=0)
    with pytest.raises(TypeError):
        net.forward(dev(_feats(2, 0).astype(np.float64)))
    with pytest.raises(ValueError):
        net.grad(dev(_feats(2, 0)), dev(_targets(3, 0)))


# ---------------------------------------------------------------- upsampling

@pytest.mark.parametrize("Nc,Nf,L", [
    ((12, 10, 6), (24, 30, 12), (3.0, 2.0, 1.0)),
    ((64, 64, 16), (128, 128, 32), (16.0, 16.0, 1.5)),
    ((8, 6, 4), (8, 12, 4), (2.0, 2.0, 1.0)),
])
def test_spectral_upsample_matches_oracle(lib, Nc, Nf, L):
    pc = lib.Plan(Nc, L, (0.0, 0.0, 1.0))
    pf = lib.Plan(Nf, L, (0.0, 0.0, 1.0))
    f = W.random_field((Nc[2], Nc[1], Nc[0]), 80)
    got = host(lib.spectral_upsample(pc, pf, dev(f)))
    ref = GN.spectral_upsample(f, Nf)
    assert rel2(got, ref) <= 1e-12
    smooth = W.guess_phi_d(Nc, L, (1.0, 1.0, 6.0), 0.7)
    got = host(lib.spectral_upsample(pc, pf, dev(smooth)))
    assert rel2(got, GN.spectral_upsample(smooth, Nf)) <= 1e-12


def test_spectral_upsample_rejects_mismatched_plans(lib):
    a = lib.Plan((8, 8, 4), (2.0, 2.0, 1.0), (0.0, 0.0, 1.0))
    b = lib.Plan((16, 16, 8), (2.0, 2.5, 1.0), (0.0, 0.0, 1.0))
    c = lib.Plan((4, 8, 4), (2.0, 2.0, 1.0), (0.0, 0.0, 1.0))
    f = dev(W.random_field((4, 8, 8), 1))
    with pytest.raises(lib.AtkmError):
        lib.spectral_upsample(a, b, f)
    with pytest.raises(lib.AtkmError):
        lib.spectral_upsample(a, c, f)
