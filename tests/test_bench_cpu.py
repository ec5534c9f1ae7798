"""bench.py's host-side contract on CPU: the reference arm (the FP64 oracle timed on this
host's cores) prints one JSON line with the main arm's metric, unit and workload, and the
helpers that set the per-frame consistency controls and report the oracle's threads."""
import argparse
import json

import bench


def _args(**kw):
    a = dict(steps=1, warmup=0, latency=0, solver_iters=0, flow_downscale=1, precision="bf16")
    a.update(kw)
    return argparse.Namespace(**a)


def test_reference_arm_prints_one_line_of_the_main_arms_workload(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    args = _args()
    bench.run_reference(args)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["dtype"] == "f64"
    want = bench.workload_config(args)
    assert d["config"]["workload"] == want["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "1920x128" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_nothing_on_other_ranks(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(_args())
    assert capsys.readouterr().out.strip() == ""


def test_workload_config_names_the_settings():
    base = bench.workload_config(_args())["workload"]
    assert "k1 swept" in base and "latency" not in base and "solver" not in base
    w = bench.workload_config(_args(latency=1, solver_iters=150, flow_downscale=2))["workload"]
    assert "one frame of latency" in w and "150 Eq. 8 solver iterations" in w and "half-size" in w


def test_consistency_controls():
    # causal stream: k1 cycles through the sweep, frame by frame
    ks = [bench.consistency_controls(i, 0, 0)["k1"] for i in range(2 * len(bench.K1_SWEEP))]
    assert ks == list(bench.K1_SWEEP) * 2
    # one frame of latency: k1 + k2 below 1, which tc_set_latency requires
    c = bench.consistency_controls(3, 50, 1)
    assert c["k1"] + c["k2"] < 1 and c["solver_iters"] == 50


def test_oracle_threads(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.oracle_threads() == 3
    monkeypatch.setenv("OMP_NUM_THREADS", "2,1")
    assert bench.oracle_threads() == 2
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.oracle_threads() >= 1
