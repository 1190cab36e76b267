"""The device-driven solve (one CUDA graph whose conditional nodes loop over
the iterations and halvings, with the FP32-to-FP64 hand-over on the device)
against the host-driven loop (the same kernels with the decisions taken on
the host between iterations: graphs off, or per-pass profiling on): states,
logs and counts must be bitwise identical; and the wall-clock limit
(ATKM_ERR_TIMEOUT) in both."""
import numpy as np
import pytest
import torch

import atkm_workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


LOG_KEYS = ("n", "halvings", "reset_to_sd", "accepted", "f32_phase", "E", "mu", "residual", "linf_step", "alpha",
            "beta_cg", "d1", "curvature", "t0", "t")


def _solve(lib, plan, w, precision, mode, max_iter=600, **kw):
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    psi = dev(W.initial_guess(w))
    if mode == "profiled":
        plan.set_profiling(True)
    try:
        r = plan.pcg_ground_state(prm, psi, max_iter=max_iter, precision=precision, graphs=(mode != "direct"),
                                  log_capacity=max_iter + 4, **kw)
    finally:
        if mode == "profiled":
            plan.set_profiling(False)
    return r, psi.cpu().numpy()


@pytest.mark.parametrize("precision,kw", [(0, {}), (1, {}), (2, {}), (3, {}), (1, dict(f32_gain=0.9, f32_window=5)),
                                          (3, dict(switch_tol=-1e-5))])
def test_device_loop_equals_host_loop(lib, precision, kw):
    """Full solves of the 32x32x16 workload in every precision form (the
    FP32 forms hand over to their polish on the device), and with another
    FP32 stagnation rule (progress factor 0.9 within 5 iterations)."""
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = lib.Plan(w.N, w.L, w.n, f32=precision != 0, df32=precision == 3)
    runs = {m: _solve(lib, plan, w, precision, m, **kw) for m in ("graph", "direct", "profiled")}
    rg, pg = runs["graph"]
    assert rg["status_name"] == "OK"
    assert rg["device_loop"] == 1 and runs["direct"][0]["device_loop"] == 0 and runs["profiled"][0]["device_loop"] == 0
    if precision:
        assert rg["f32_iters"] > 0
    for m in ("direct", "profiled"):
        r, p = runs[m]
        assert np.array_equal(p, pg), m
        for k in ("iters", "halvings", "f32_iters", "status", "E", "mu", "residual", "virial", "log_count"):
            assert r[k] == rg[k], (m, k, r[k], rg[k])
        assert len(r["log"]) == len(rg["log"])
        for a, b in zip(r["log"], rg["log"]):
            for k in LOG_KEYS:
                assert a[k] == b[k], (m, a["n"], k, a[k], b[k])


def test_device_loop_resume_and_iteration_cap(lib):
    """max_iter stops the device loop exactly; resume continues it to the
    same state as one uninterrupted solve."""
    w = W.CONFIGS["cfg2_128x128x32"]
    plan = lib.Plan(w.N, w.L, w.n)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    a = dev(W.initial_guess(w))
    ra = plan.pcg_ground_state(prm, a, max_iter=30, tol_residual=0.0)
    b = dev(W.initial_guess(w))
    r1 = plan.pcg_ground_state(prm, b, max_iter=13, tol_residual=0.0)
    assert r1["iters"] == 13 and r1["status_name"] == "NOT_CONVERGED"
    r2 = plan.pcg_ground_state(prm, b, max_iter=17, tol_residual=0.0, resume=True)
    assert r2["iters"] == 30 == ra["iters"]
    assert torch.equal(a, b) and r2["E"] == ra["E"]


@pytest.mark.parametrize("graphs", [True, False])
def test_time_limit_stops_with_timeout(lib, graphs):
    """time_limit_s: the run stops at an iteration top once the limit has
    passed (device global timer or host clock) with ATKM_ERR_TIMEOUT, returns
    the state reached, and the solve can be resumed."""
    w = W.CONFIGS["cfg2_128x128x32"]
    plan = lib.Plan(w.N, w.L, w.n)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    plan.pcg_ground_state(prm, dev(W.initial_guess(w)), max_iter=2, graphs=graphs)  # builds the solve graph
    psi = dev(W.initial_guess(w))
    r = plan.pcg_ground_state(prm, psi, max_iter=100000, tol_residual=0.0, time_limit_s=0.25, graphs=graphs,
                              log_capacity=100000)
    assert r["status"] == lib.ATKM_ERR_TIMEOUT and r["device_loop"] == int(graphs)
    assert 0 < r["iters"] < 100000
    Es = [e["E"] for e in r["log"]]
    assert Es[-1] < Es[0]
    r2 = plan.pcg_ground_state(prm, psi, max_iter=5, tol_residual=0.0, resume=True, graphs=graphs)
    assert r2["iters"] == r["iters"] + 5 and r2["E"] <= r["E"]
    # an already expired limit stops before the first step
    psi = dev(W.initial_guess(w))
    r = plan.pcg_ground_state(prm, psi, max_iter=100, time_limit_s=1e-9, graphs=graphs)
    assert r["status"] == lib.ATKM_ERR_TIMEOUT and r["iters"] == 0


def test_batched_single_launch_equals_single_solves_with_handover(lib):
    """The batched call (one graph, one chain per instance) in the FP32-bulk
    form with its on-device hand-over equals each instance solved alone."""
    cases = [((32, 32, 16), (8.0, 8.0, 2.5), 0.40), ((24, 24, 12), (6.0, 6.0, 2.5), 0.55),
             ((48, 40, 16), (8.0, 7.0, 2.5), 0.30), ((20, 30, 10), (5.0, 6.0, 2.5), 0.25)]
    gamma, beta, lam, n = (1.0, 1.0, 4.0), 40.0, 12.0, (0.0, 0.0, 1.0)
    plans, prms, psis, refs = [], [], [], []
    for N, L, Om in cases:
        prms.append(lib.make_params(gamma, beta, lam, Om))
        solo = lib.Plan(N, L, n, f32=True)
        ps = dev(W.guess_phi_d(N, L, gamma, Om))
        refs.append((solo.pcg_ground_state(prms[-1], ps, max_iter=800, precision=1), ps.cpu().numpy()))
        plans.append(lib.Plan(N, L, n, f32=True))
        psis.append(dev(W.guess_phi_d(N, L, gamma, Om)))
    launches0 = lib.launch_count()
    outs = lib.pcg_ground_state_batched(plans, prms, psis, max_iter=800, precision=1)
    assert lib.launch_count() > launches0
    for (ref, ref_psi), ps, o in zip(refs, psis, outs):
        assert o["device_loop"] == 1
        assert o["status_name"] == ref["status_name"] == "OK"
        assert o["iters"] == ref["iters"] and o["f32_iters"] == ref["f32_iters"] > 0
        assert o["E"] == ref["E"]
        assert np.array_equal(ps.cpu().numpy(), ref_psi)


def test_automatic_handover_at_fp32_noise(lib):
    """switch_tol < 0: the FP32 phase hands over at the larger of |switch_tol|
    and 4x the residual's FP32 noise measured at phi_0; that noise is the
    level at which an FP32 phase that never hands over stops making progress
    (its residual floor), within a factor of 10."""
    w = W.CONFIGS["cfg1_32x32x16"]
    plan = lib.Plan(w.N, w.L, w.n, f32=True)
    prm = lib.make_params(w.gamma, w.beta, w.lam, w.Omega)
    r = plan.pcg_ground_state(prm, dev(W.initial_guess(w)), max_iter=3000, precision=1, switch_tol=-1e-12,
                              log_capacity=3002)
    sw = r["switch_residual"]
    assert r["status_name"] == "OK" and r["f32_iters"] > 0 and sw > 1e-12
    f32_log = [e for e in r["log"] if e["f32_phase"]]
    assert all(e["residual"] > sw for e in f32_log)
    noise = sw / 4.0
    # the same start in FP32 only: its residual floor
    q = plan.pcg_ground_state(prm, dev(W.initial_guess(w)), max_iter=len(f32_log) + 400, tol_residual=0.0,
                              precision=1, switch_tol=1e-14, f32_window=10 ** 8, log_capacity=4000)
    res = [e["residual"] for e in q["log"] if e["f32_phase"]]
    floor = min(res)
    assert floor / 10 <= noise <= 10 * floor, (noise, floor)
    # a plain switch_tol reports itself
    r2 = plan.pcg_ground_state(prm, dev(W.initial_guess(w)), max_iter=3000, precision=1, switch_tol=1e-5)
    assert r2["switch_residual"] == 1e-5
