"""Failure detection without a GPU fault.

* A stride-1 tensor-core conv whose producer issues nothing (tc_test_stall_next_convs):
  every bounded mbarrier wait of its CTAs runs out after the wait limit (2 s), the kernels
  record a code in the device error word, free their tensor memory and exit.  The stream
  reports TC_ERR_TIMEOUT, is poisoned, the device stays usable, and a fresh stream gives the
  same results as before.
* A device allocation that fails inside tc_create_stream (tc_test_fail_device_allocation):
  TC_ERR_OOM, nothing leaked, and the next creation works."""
import time

import numpy as np
import pytest

import synth
from gpu_common import nchw_to_nhwc, round16, to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _two_frames(s, d, H, W):
    import torch
    O = torch.empty((3, H, W), device="cuda")
    s.process_frame(to_dev(d["I0"]), to_dev(d["P0"]), O)
    s.process_frame(to_dev(d["I1"]), to_dev(d["P1"]), O)
    Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
    s.get_flows(Fb, Ff)
    s.synchronize()
    return to_np(O), to_np(Fb), to_np(Ff)


def test_stalled_conv_times_out_poisons_stream_and_device_recovers():
    import torch
    path, _ = weights_file()
    d = synth.pair64()
    ref = tc.Stream(64, 64, "fp16", weights_path=path)
    want = _two_frames(ref, d, 64, 64)
    ref.destroy()

    s = tc.Stream(64, 64, "fp16", weights_path=path)
    s.set_graphs(False)
    O = torch.empty((3, 64, 64), device="cuda")
    s.process_frame(to_dev(d["I0"]), to_dev(d["P0"]), O)
    s.synchronize()
    tc.inject_stall_next_convs(1)
    t0 = time.perf_counter()
    try:
        s.process_frame(to_dev(d["I1"]), to_dev(d["P1"]), O)
        with pytest.raises(tc.TcError) as e:
            s.synchronize()
    finally:
        tc.inject_stall_next_convs(0)
    dt = time.perf_counter() - t0
    assert e.value.status == tc.TC_ERR_TIMEOUT, str(e.value)
    assert 1.5 < dt < 60.0, dt  # the 2 s wait limit, not a hang
    with pytest.raises(tc.TcError) as e2:
        s.process_frame(to_dev(d["I0"]), to_dev(d["P0"]), O)
    assert e2.value.status == tc.TC_ERR_STATE
    s.destroy()
    torch.cuda.synchronize()  # the context is intact

    fresh = tc.Stream(64, 64, "fp16", weights_path=path)
    got = _two_frames(fresh, d, 64, 64)
    fresh.destroy()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_stalled_stage_conv_reports_timeout():
    import torch
    g = synth.rng(70)
    x = to_dev(nchw_to_nhwc(round16("fp16", g.normal(size=(1, 64, 12, 40)).astype(np.float32))))
    wt = (g.normal(size=(64, 64, 3, 3)) / 24.0).astype(np.float32)
    b = np.zeros(64, np.float32)
    tc.inject_stall_next_convs(1)
    try:
        with pytest.raises(tc.TcError) as e:
            tc.op_conv3x3(x, wt, b, precision="fp16")
    finally:
        tc.inject_stall_next_convs(0)
    assert e.value.status == tc.TC_ERR_TIMEOUT
    out = tc.op_conv3x3(x, wt, b, precision="fp16")  # the next call runs normally
    torch.cuda.synchronize()
    assert tc.op_last_used_tensor_cores() and np.isfinite(to_np(out)).all()


@pytest.mark.parametrize("nth", [1, 2, 9, 40])
def test_allocation_failure_in_create_stream_returns_oom(nth):
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    tc.Stream(200, 136, "fp16", weights_path=path).destroy()  # module loading, library state
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    tc.inject_device_allocation_failure(nth)
    try:
        with pytest.raises(tc.TcError) as e:
            tc.Stream(200, 136, "fp16", weights_path=path)
    finally:
        tc.inject_device_allocation_failure(0)
    assert e.value.status == tc.TC_ERR_OOM, str(e.value)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) <= 4 << 20, (free0, free1)  # everything allocated was freed
    s = tc.Stream(200, 136, "fp16", weights_path=path)
    s.destroy()
