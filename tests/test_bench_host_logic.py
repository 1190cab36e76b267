"""Host-side bookkeeping of the benchmark's extra lines, on the CPU: the
sweep's per-form summaries and its instance-by-instance energy agreement
(what counts as the same energy, a lower or a higher one), and the command
line of every bench case (the cases themselves need the GPU)."""
import sys

import pytest

import bench
from paper_2603_05194_gb300 import binding as B
from paper_2603_05194_gb300 import sweep as S


def _res(E, status=B.ATKM_OK, iters=10, residual=1e-9):
    return {"E": E, "status": status, "status_name": B.STATUS_NAMES.get(status, str(status)), "iters": iters,
            "residual": residual, "device_loop": True}


def test_sweep_agreement_counts_energies_of_converged_pairs_only():
    ref = [_res(10.0), _res(20.0), _res(30.0), _res(40.0), _res(50.0, status=B.ATKM_NOT_CONVERGED)]
    res = [_res(10.0 * (1 + 5e-10)),             # same within 1e-9
           _res(20.0 * (1 - 2e-9)),              # lower
           _res(30.0 * (1 + 3e-6)),              # higher
           _res(40.0, status=B.ATKM_NOT_CONVERGED),  # not compared
           _res(50.0)]                           # reference did not converge: not compared
    a = S._agreement(res, ref)
    assert a["both_converged"] == 3
    assert (a["same_energy"], a["lower_energy"], a["higher_energy"]) == (1, 1, 1)
    assert a["max_abs_rel_dE_same"] == pytest.approx(5e-10, rel=1e-6)


def test_sweep_summary_keeps_per_instance_records():
    res = [_res(1.0, iters=5), _res(2.0, status=B.ATKM_NOT_CONVERGED, iters=7, residual=1e-5)]
    s = S._summary(res, 3.5)
    assert s["seconds"] == 3.5 and s["iters"] == [5, 7] and s["E"] == [1.0, 2.0]
    assert s["statuses"] == {"OK": 1, "NOT_CONVERGED": 1} and s["device_loop"] is True
    assert s["residual"] == [1e-9, 1e-5]


@pytest.mark.parametrize("argv, key, value", [
    (["--case", "sweep", "--sweep-max-iter", "5000"], "case", "sweep"),
    (["--case", "guess"], "case", "guess"),
    (["--profile-case", "autotune"], "profile_case", "autotune"),
    (["--profile-case", "guess_gemm"], "profile_case", "guess_gemm"),
    (["--ttt", "f64,f32_split"], "ttt", "f64,f32_split"),
    ([], "case", "step"),
])
def test_bench_command_line(monkeypatch, argv, key, value):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    a = bench.parse()
    assert getattr(a, key) == value
    if argv[:2] == ["--case", "sweep"]:
        assert a.sweep_max_iter == 5000


def test_bench_default_times_every_precision_form():
    """The default run times binary64 and each precision form to 1e-8."""
    saved = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = saved
    assert a.ttt.split(",") == ["f64", "f32_f64", "f32_split", "df32_split", "df32_split_all"]
    assert a.steps >= 1 and a.warmup >= 3 and a.gpus == 1
