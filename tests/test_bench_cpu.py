"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle on host cores) and the
helpers the GPU arm uses for its roofline and rank timing."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def _check_line(j, unit):
    for k in KEYS:
        assert k in j, k
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == unit
    assert j["value"] > 0 and j["higher_is_better"] is True and j["vs_baseline"] is None
    assert j["steps"] == 1 and j["n_gpus"] == 1
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == unit
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in j["config"]


def test_reference_arm_lowd_line():
    """lowd_2m: the oracle's full-size solve to convergence (no row sample), one per step."""
    j = _run("--workload", "lowd_2m", "--steps", "1", "--warmup", "0")
    _check_line(j, "solves/s")
    assert j["config"]["workload"] == "lowd_2m" and j["config"]["N"] == 2_000_000
    assert "full-size Algorithm 1 solves (N=2000000" in j["cpu_baseline"]["sample"]
    assert j["ms_per_step"] == pytest.approx(1e3 / j["value"])


def test_dense_reference_pass_count_is_the_oracles():
    """The dense reference arm scales its full-size per-pass time by the assignment passes of the
    oracle's own full-size solve, stored by tests/golden/make_dense_1m.py."""
    p = bench.oracle_dense_passes()
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "dense_1m_oracle.json")))
    assert p == g["aa"]["assign_passes"] and p > g["aa"]["iters"] >= 1
    assert bench.oracle_dense_passes("/nonexistent.json") is None


def test_result_errors_against_oracle_arithmetic():
    import numpy as np
    import datagen
    import oracle
    X, C0 = datagen.small_2d(2)
    C, rho, info = oracle.solve(X, C0)
    e = bench.result_errors(X, [(C, rho, info["E"])], sample_rows=3000)
    assert e["E_rel_max"] < 1e-14 and e["C_rel_max"] < 1e-14 and e["labels_off_argmin_clear_rows"] == 0
    # a planted error in each field is seen
    e = bench.result_errors(X, [(C * (1 + 1e-5), rho, info["E"] * (1 + 1e-4))], sample_rows=3000)
    assert 0.5e-4 < e["E_rel_max"] and e["C_rel_max"] > 1e-6
    r2 = rho.copy()
    r2[:] = (rho + 1) % C.shape[0]
    e = bench.result_errors(X, [(C, r2, info["E"])], sample_rows=3000)
    assert e["labels_off_argmin_clear_rows"] > 2000


def test_reference_arm_batched_line():
    j = _run("--workload", "batched_512", "--steps", "1", "--warmup", "0")
    _check_line(j, "instance solves/s")
    assert j["config"]["workload"] == "batched_512"


def test_profiled_traffic_reads_the_committed_summary():
    t = bench.profiled_traffic("k_pass_lowd_lowd_2m.md")
    assert isinstance(t, int) and 20_000_000 < t < 60_000_000
    assert bench.profiled_traffic("no_such_profile.md") is None


def test_rank_helpers():
    assert bench.max_over_ranks([1, 2.5], None, None) == [1.0, 2.5]
    assert bench.pct([3, 1, 2], 50) == 2 and bench.pct([], 50) is None
    assert bench.pct(list(range(101)), 99) == 99


def test_solve_launch_count():
    # lowd_2m: Hamerly bounds, separate mix -> 5 kernels in the prologue and per loop pass, 2 after
    assert bench.solve_launches(152, dense=False, ham=True, fused_mix=False) == 5 * 153 + 2
    assert bench.solve_launches(10, dense=False, ham=False, fused_mix=True) == 3 * 11 + 2
    assert bench.solve_launches(160, dense=True, ham=False, fused_mix=False, rejected=23,
                                inc=False) == 19 + 13 * 160 + 10 * 23
    # the incremental update: three more kernels in every INIT, TRIAL and REVERT chain
    assert bench.solve_launches(160, dense=True, ham=False, fused_mix=False, rejected=23) == 22 + 16 * 160 + 13 * 23


def test_same_energy_speed():
    r, n = bench.same_energy_speed([10.0, 20.0, 30.0], [15.0, 25.0, 60.0], [1.0, 2.0, 3.0],
                                   [1.0 + 1e-9, 2.5, 3.0])
    assert n == 2 and r == pytest.approx((15.0 + 60.0) / (10.0 + 30.0))
    assert bench.same_energy_speed([1.0], [2.0], [1.0], [2.0]) == (None, 0)


def test_batched_launch_count(monkeypatch):
    # 3 groups, bounds and a separate mix: 2 + 1 + 3 + 1 in the prologue, 1 + 6 + 2 + 1 per step, 3 + 1 after
    assert bench.batched_launches(10, 3, True, True, []) == 7 + 10 * 10 + 4
    assert bench.batched_launches(10, 3, False, False, []) == 5 + 10 * 8 + 4
    # the dense instances with the incremental update (the default; KM_DINC=0 removes the 3s)
    monkeypatch.delenv("KM_DINC", raising=False)
    assert bench.batched_launches(5, 2, True, True, [(7, 1), (9, 0)]) == \
        (6 + 5 * 8 + 3) + (22 + 16 * 7 + 13) + (22 + 16 * 9)
    assert bench.batched_launches(0, 0, False, False, [(4, 2)]) == 22 + 16 * 4 + 13 * 2
    monkeypatch.setenv("KM_DINC", "0")
    assert bench.batched_launches(0, 0, False, False, [(4, 2)]) == 19 + 13 * 4 + 10 * 2


def test_oracle_thread_count_is_restored():
    import numpy as np
    import oracle
    import datagen
    X, C0 = datagen.small_2d(0)
    before = oracle.num_threads()
    t, info, cores, C1, r1 = bench.oracle_timed(X, C0, 1000, 10, threads=1)
    assert cores == 1 and t > 0 and info["converged"] == 1
    assert oracle.num_threads() == before
    # the thread count does not change the result
    t, info2, cores, C2, r2 = bench.oracle_timed(X, C0, 1000, 10)
    np.testing.assert_array_equal(C1, C2)
    assert info["iters"] == info2["iters"]


def test_parse_tuning_reads_the_chosen_variant_and_grid():
    desc = ("f32 d=2 cls=4 ops=1.5e+09 items=4676 v0(occ 3) 152:528.4us 4676:239.8us "
            "v1(occ 3) 152:517.0us 4676:243.9us -> variant 0 grid 4676; "
            "f32 d=16 cls=4 ops=1.3e+09 items=2872 v0(occ 2) 2872:468.5us v1(occ 2) 2872:428.9us "
            "-> variant 1 grid 2872; fin items=13859 grid=608")
    assert bench.parse_tuning(desc) == [(2, 1.5e9, 4676, 239.8), (16, 1.3e9, 2872, 428.9)]
