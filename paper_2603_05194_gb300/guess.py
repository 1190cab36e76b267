"""Learned initial guess for the PCG ground-state solver.

The paper starts Algorithm 1 from one of a fixed set of formula guesses (§3,
guess (d) among them) or from a coarse solution interpolated upward
(Algorithm 2, Step 2).  This module replaces the choice of guess by a small
network trained on ground states that the plain PCG computes itself:

  problem parameters -> features (8) -> GuessNet (BF16 tensor-core GEMMs,
  FP32 accumulation) -> psi_0 on the 64x64x16 grid of the problem's box ->
  Fourier interpolant on the fine grid (spectral upsampling) -> PCG to the
  residual tolerance, with plain PCG from guess (d) as the fallback and as the
  check of the final energy.

Everything numeric runs in libatkm's kernels; this module only marshals
arguments, orders the calls and keeps the bookkeeping.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B

COARSE_N = (64, 64, 16)          # (N_x, N_y, N_z) of the network's output grid
FEATURES = ("Omega", "gamma_x - 1", "gamma_y - 1", "ln gamma_z", "ln beta", "lambda/beta", "sin theta", "cos theta")


def features(Omega, gamma, beta, lam, n) -> np.ndarray:
    """The 8 network inputs of one problem, each scaled to about [-1, 1] over
    the training ranges (Omega in [0.3, 0.95], gamma_z in [5, 50], beta in
    [100, 1000], lambda/beta in [0, 0.45], dipole tilt theta in [0, 60 deg])."""
    sin_t = math.hypot(n[0], n[1])
    return np.array([(Omega - 0.625) / 0.325, gamma[0] - 1.0, gamma[1] - 1.0,
                     (math.log(gamma[2]) - 2.76) / 1.15, (math.log(beta) - 5.76) / 1.15,
                     (lam / beta) / 0.225 - 1.0, sin_t, n[2]], dtype=np.float32)


def problem_features(problems) -> torch.Tensor:
    f = np.stack([features(p.Omega, p.gamma, p.beta, p.lam, p.n) for p in problems])
    return torch.from_numpy(f).cuda()


def _params(p) -> B.Params:
    return B.make_params(p.gamma, p.beta, p.lam, p.Omega)


def solve_batch(problems, psi0s, N, tol=1e-8, max_iter=5000, precision=B.PRECISION_F32_F64, plans=None):
    """Ground states of `problems` on grid N, one concurrent batched call.
    psi0s: device complex128 tensors (overwritten with the results).
    Returns (results, seconds of wall time around the call)."""
    own = plans is None
    if own:
        plans = [B.Plan(N, p.L, p.n, f32=(precision == B.PRECISION_F32_F64)) for p in problems]
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = B.pcg_ground_state_batched(plans, [_params(p) for p in problems], psi0s, tol_residual=tol,
                                         max_iter=max_iter, precision=precision)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0
    finally:
        if own:
            for pl in plans:
                pl.close()


def make_targets(problems, psi0_fn, tol=1e-7, max_iter=3000, chunk=32, log=print):
    """Training targets: PCG ground states on COARSE_N from guess (d), in
    chunks of concurrent solves.  psi0_fn(problem) -> host complex128 array.
    Returns (targets [M, 16, 64, 64] complex128 on the device, results)."""
    M = len(problems)
    targets = torch.empty((M, COARSE_N[2], COARSE_N[1], COARSE_N[0]), dtype=torch.complex128, device="cuda")
    results = []
    for c0 in range(0, M, chunk):
        part = problems[c0:c0 + chunk]
        for i, p in enumerate(part):
            targets[c0 + i].copy_(torch.from_numpy(psi0_fn(p)))
        res, sec = solve_batch(part, [targets[c0 + i] for i in range(len(part))], COARSE_N, tol, max_iter)
        results += res
        conv = sum(r["status"] == B.ATKM_OK for r in res)
        log(f"targets {c0 + len(part)}/{M}: {conv}/{len(part)} converged, {sec:.1f} s, "
            f"median iters {int(np.median([r['iters'] for r in res]))}")
    return targets, results


def train(net: B.GuessNet, feats: torch.Tensor, targets: torch.Tensor, steps: int, batch: int = 32,
          lr: float = 2e-3, lr_final: float = 1e-4, seed: int = 0, log_every: int = 100, log=print):
    """Adam on contiguous minibatches (the rows are i.i.d. draws), batch order
    shuffled per epoch on the host, cosine learning-rate decay."""
    M = feats.shape[0]
    nb = max(1, M // batch)
    rng = np.random.default_rng(seed)
    order = rng.permutation(nb)
    loss_dev = torch.empty(1, dtype=torch.float32, device="cuda")
    hist = []
    for s in range(steps):
        if s % nb == 0 and s > 0:
            order = rng.permutation(nb)
        b0 = int(order[s % nb]) * batch
        cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * s / max(1, steps)))
        net.train_step(feats[b0:b0 + batch], targets[b0:b0 + batch], cur, loss=loss_dev)
        if (s + 1) % log_every == 0 or s + 1 == steps:
            hist.append((s + 1, float(loss_dev.item())))
            log(f"step {s + 1}: loss {hist[-1][1]:.4e} lr {cur:.2e}")
    return hist


def loss_of(net: B.GuessNet, feats, targets, batch=32) -> float:
    """Mean loss over a set (no parameter update)."""
    tot, n = 0.0, feats.shape[0]
    for b0 in range(0, n, batch):
        _, loss = net.grad(feats[b0:b0 + batch], targets[b0:b0 + batch])
        tot += float(loss.item()) * min(batch, n - b0)
    return tot / n


def infer_fine(net: B.GuessNet, problems, fine_N, fine_plans=None):
    """psi_0 on fine_N for each problem: network output on COARSE_N, then the
    Fourier interpolant on the fine grid of the same box (unit norm is restored
    by the solver).  Returns (list of device tensors, seconds)."""
    feats = problem_features(problems)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    coarse = net.forward(feats)
    out = []
    for i, p in enumerate(problems):
        pc = B.Plan(COARSE_N, p.L, p.n)
        pf = fine_plans[i] if fine_plans is not None else B.Plan(fine_N, p.L, p.n)
        out.append(B.spectral_upsample(pc, pf, coarse[i]))
        torch.cuda.synchronize()
        pc.close()
        if fine_plans is None:
            pf.close()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def evaluate(net: B.GuessNet, problems, psi0_fn, fine_N, tol=1e-8, max_iter=6000, e_tol=1e-9, chunk=40, log=print,
             precision=B.PRECISION_F32_F64):
    """Held-out comparison on fine_N: PCG from the learned guess against PCG
    from guess (d), each arm one batched call per chunk of problems, both in
    `precision`.  The plain run judges the final energy: an instance whose
    learned run does not converge, or ends above the plain energy by more than
    e_tol relative, falls back to the plain result."""
    res_l, res_p, t_inf, t_l, t_p = [], [], 0.0, 0.0, 0.0
    for c0 in range(0, len(problems), chunk):
        part = problems[c0:c0 + chunk]
        plans = [B.Plan(fine_N, p.L, p.n, f32=True) for p in part]
        try:
            learned, ti = infer_fine(net, part, fine_N, fine_plans=plans)
            rl, tl = solve_batch(part, learned, fine_N, tol, max_iter, precision=precision, plans=plans)
            del learned
            plain = [torch.from_numpy(psi0_fn(p)).cuda() for p in part]
            rp, tp = solve_batch(part, plain, fine_N, tol, max_iter, precision=precision, plans=plans)
            del plain
        finally:
            for pl in plans:
                pl.close()
        res_l += rl
        res_p += rp
        t_inf, t_l, t_p = t_inf + ti, t_l + tl, t_p + tp
    rows, fallbacks = [], 0
    for p, rl, rp in zip(problems, res_l, res_p):
        dE = (rl["E"] - rp["E"]) / abs(rp["E"])
        fb = rl["status"] != B.ATKM_OK or dE > e_tol
        fallbacks += fb
        rows.append(dict(name=p.name, Omega=p.Omega, gamma_z=p.gamma[2], beta=p.beta, lam=p.lam,
                         theta_deg=math.degrees(math.atan2(math.hypot(p.n[0], p.n[1]), p.n[2])),
                         iters_learned=rl["iters"], iters_plain=rp["iters"], status_learned=rl["status_name"],
                         status_plain=rp["status_name"], E_learned=rl["E"], E_plain=rp["E"], dE_rel=dE,
                         fallback=bool(fb)))
        log(f"{p.name}: iters {rl['iters']} vs {rp['iters']}, dE/|E| {dE:+.2e} "
            f"({rl['status_name']}/{rp['status_name']})")
    il = np.array([r["iters_learned"] for r in rows])
    ip = np.array([r["iters_plain"] for r in rows])
    return dict(instances=len(rows), fine_grid=list(fine_N), tol=tol, max_iter=max_iter,
                inference_s=t_inf, solve_s_learned=t_l, solve_s_plain=t_p,
                iters_learned_median=float(np.median(il)), iters_plain_median=float(np.median(ip)),
                iters_learned_total=int(il.sum()), iters_plain_total=int(ip.sum()),
                converged_learned=int(sum(r["status_learned"] == "OK" for r in rows)),
                converged_plain=int(sum(r["status_plain"] == "OK" for r in rows)),
                lower_energy_learned=int(sum(r["dE_rel"] < -e_tol for r in rows)),
                same_energy=int(sum(abs(r["dE_rel"]) <= e_tol for r in rows)),
                higher_energy_learned=int(sum(r["dE_rel"] > e_tol for r in rows)),
                fallbacks=int(fallbacks), rows=rows)


def main(argv=None):
    import atkm_workloads as W
    ap = argparse.ArgumentParser(description="train the learned guess on PCG ground states and compare on held-out draws")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--holdout", type=int, default=200, help="held-out draws for the loss")
    ap.add_argument("--eval", type=int, default=200, help="held-out draws solved on the fine grid")
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--target-tol", type=float, default=1e-7)
    ap.add_argument("--target-iters", type=int, default=3000)
    ap.add_argument("--eval-iters", type=int, default=6000)
    ap.add_argument("--chunk", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-params", default=None, help="write the trained parameters (.npy)")
    a = ap.parse_args(argv)
    B.load_library()
    psi0 = lambda p: W.initial_guess(p)  # noqa: E731  guess (d) on the problem's grid
    t0 = time.perf_counter()
    train_p = W.guess_draws(a.train + a.holdout, seed=5)
    tgt, res_t = make_targets(train_p, psi0, a.target_tol, a.target_iters, a.chunk)
    t_targets = time.perf_counter() - t0
    ok = [i for i, r in enumerate(res_t) if r["residual"] < 1e-4]
    tr = [i for i in ok if i < a.train]
    ho = [i for i in ok if i >= a.train]
    feats = problem_features(train_p)
    idx_tr = torch.tensor(tr, device="cuda")
    idx_ho = torch.tensor(ho, device="cuda")
    f_tr, t_tr = feats[idx_tr].contiguous(), tgt[idx_tr].contiguous()
    f_ho, t_ho = feats[idx_ho].contiguous(), tgt[idx_ho].contiguous()
    del tgt
    net = B.GuessNet(seed=a.seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = train(net, f_tr, t_tr, a.steps, a.batch, a.lr, seed=a.seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    loss_tr, loss_ho = loss_of(net, f_tr, t_tr), loss_of(net, f_ho, t_ho)
    if a.save_params:
        np.save(a.save_params, net.get_params().cpu().numpy())
    print(f"train loss {loss_tr:.4e}, held-out loss {loss_ho:.4e}")
    eval_p = [W.with_grid(p, W.GUESS_FINE_N) for p in W.guess_draws(a.eval, seed=6)]
    ev = evaluate(net, eval_p, psi0, W.GUESS_FINE_N, 1e-8, a.eval_iters, chunk=a.chunk)
    out = dict(train_draws=a.train, train_used=len(tr), holdout_used=len(ho), target_tol=a.target_tol,
               target_seconds=t_targets, train_steps=a.steps, batch=a.batch, train_seconds=t_train,
               loss_train=loss_tr, loss_holdout=loss_ho, loss_history=hist, eval=ev)
    js = json.dumps(out)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(js + "\n")
    summary = {k: v for k, v in ev.items() if k != "rows"}
    print(json.dumps(dict(loss_train=loss_tr, loss_holdout=loss_ho, **summary)))


if __name__ == "__main__":
    main()
