"""bench.py's host-side contract on CPU: the reference arm (the FP64 oracle timed on this
host's cores) prints one JSON line with the main arm's metric, unit and workload; the helpers
that set the per-frame consistency controls and report the oracle's threads; the FLOP count
behind the roofline, against torch's own FLOP counter; and the summary of the clock samples
that decides whether a run saw a throttle reason."""
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


def test_conv_flops_match_torch_flop_counter():
    """The roofline's numerator, counted independently: torch's FLOP counter over meta-device
    convolutions (no arithmetic is done) with the network's layer shapes at the padded 1080p
    frame, and the correlation as one (1 x c) by (c x (2R+1)^2) product per pixel."""
    import torch
    import torch.nn.functional as F
    from torch.utils.flop_counter import FlopCounterMode

    spec = bench.net_spec()
    got = bench.conv_flops_per_frame(spec)
    m = 1 << spec.levels
    hp, wp = -(-bench.HEIGHT // m) * m, -(-bench.WIDTH // m) * m
    layers = spec.layer_table()
    meta = dict(device="meta")

    def count(fn):
        with FlopCounterMode(display=False) as fc:
            fn()
        return fc.get_total_flops()

    def pyramid():  # one frame, the levels chained
        x = torch.empty(1, 3, hp, wp, **meta)
        for name, cin, cout, stride, _ in layers:
            if name.startswith("pyr"):
                x = F.conv2d(x, torch.empty(cout, cin, 3, 3, **meta), stride=stride, padding=1)

    def estimators(head):  # both flow directions as a batch of two
        for name, cin, cout, _, _ in layers:
            if name.startswith("est") and name.endswith("c5") == head:
                l = int(name[3])
                F.conv2d(torch.empty(2, cin, hp >> l, wp >> l, **meta), torch.empty(cout, cin, 3, 3, **meta),
                         padding=1)

    def correlation():
        d = (2 * spec.radius + 1) ** 2
        for l in range(2, spec.levels + 1):
            px, c = 2 * (hp >> l) * (wp >> l), spec.chans[l - 1]
            torch.bmm(torch.empty(px, 1, c, **meta), torch.empty(px, c, d, **meta))

    assert got["pyramid_conv"] == count(pyramid)
    assert got["estimator_conv"] == count(lambda: estimators(False))
    assert got["head"] == count(lambda: estimators(True))
    assert got["correlation"] == count(correlation)


def test_clock_samples_summary():
    off = "Not Active"
    lines = [f"0, 2032, 2032, 700.5, 0x0, {off}, {off}, {off}, {off}",
             f"0, 1965, 2032, 1099.0, 0x4, {off}, {off}, {off}, Active",
             f"0, 2032, 2032, 810.0, 0x0, {off}, {off}, {off}, {off}",
             "", "0, [N/A], 2032, 0, 0x0, , , , "]  # an empty and an unparsable line are skipped
    assert bench.ClockSampler.summarize(lines) == dict(sm_mhz=2032.0, sm_max_mhz=2032.0,
                                                       reasons=["sw_power_cap"], samples=3)
    hot = [f"0, 1500, 2032, 900.0, 0x40, {off}, {off}, Active, {off}"] * 2
    r = bench.ClockSampler.summarize(hot)
    assert r["reasons"] == ["sw_thermal_slowdown"] and r["sm_mhz"] == 1500.0
    assert bench.ClockSampler.summarize([])["samples"] == 0


def test_train_flops_match_torch_flop_counter():
    """The training roofline's numerator, counted independently: forward and autograd backward
    of meta-device convolutions with the network's layer shapes (pyramids of 2B images chained
    from an input that takes no gradient, so the first conv has no data gradient; estimators on
    B pairs), and the correlation as a per-pixel product whose two operands take gradients."""
    import torch
    import torch.nn.functional as F
    from torch.utils.flop_counter import FlopCounterMode

    spec = bench.net_spec()
    B, S = bench.TRAIN_BATCH, bench.TRAIN_SIZE
    meta = dict(device="meta")
    with FlopCounterMode(display=False) as fc:
        outs = []
        x = torch.empty(2 * B, 3, S, S, **meta)
        for name, cin, cout, stride, _ in spec.layer_table():
            w = torch.empty(cout, cin, 3, 3, requires_grad=True, **meta)
            if name.startswith("pyr"):
                x = F.conv2d(x, w, stride=stride, padding=1)
                outs.append(x)
            else:
                l = int(name[3])
                xe = torch.empty(B, cin, S >> l, S >> l, requires_grad=True, **meta)
                outs.append(F.conv2d(xe, w, padding=1))
        d = (2 * spec.radius + 1) ** 2
        for l in range(2, spec.levels + 1):
            px, c = B * (S >> l) ** 2, spec.chans[l - 1]
            a = torch.empty(px, 1, c, requires_grad=True, **meta)
            b = torch.empty(px, c, d, requires_grad=True, **meta)
            outs.append(torch.bmm(a, b))
        sum(o.sum() for o in outs).backward()
    assert bench.train_flops_per_step(spec)["total"] == fc.get_total_flops()


def test_epe_px_closed_forms():
    """The end-point error behind `at_fixed_epe` (Eq. 10): the mean over pixels of the
    Euclidean norm of the flow difference, on cases with a closed-form answer."""
    import torch

    z = torch.zeros(2, 4, 6)
    d = torch.stack([torch.full((4, 6), 3.0), torch.full((4, 6), -4.0)])
    assert bench.epe_px(z, d) == 5.0  # |(3, -4)| at every pixel
    half = torch.zeros(2, 4, 6)
    half[1, :2] = 2.0  # half of the pixels off by (0, 2), the rest exact
    assert bench.epe_px(half, z) == 1.0
    assert bench.epe_px(d, d) == 0.0
