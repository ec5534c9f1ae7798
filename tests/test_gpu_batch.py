"""Batches (tc_create_batch / tc_process_lanes): several streams of one size as lanes whose
pyramids and flow estimations run in shared launches.  Every lane's outputs and flows must
equal, bit for bit, those of an independent stream given the same frames, whichever other
lanes run in the same step -- over schedules where the set of lanes with a frame changes
from step to step (so the shared launches cover idle lanes too), with per-lane controls,
graph capture and replay of the repeated lane ranges, and a lane reset for a new stream."""
import numpy as np
import pytest

import synth
from gpu_common import to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

NET = ((16, 32, 64, 96, 128), 4)
W, H = 200, 136
SCHEDULE = [[0, 1, 2], [0, 2], [1], [0, 1, 2], [2], [0, 1], [0, 1, 2], [1, 2], [0, 2], [0, 1, 2], [1]]


def _seq(seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(16, 30), max_vel=2.0)
    I = [seq.frame(t) for t in range(n)]
    return I, [seq.stylized(t, f) for t, f in enumerate(I)]


def _stream_run(path, prec, frames, styl, k1):
    """An independent stream: per frame (O, wc, mask, Fb, Ff) (flows None on the first)."""
    import torch
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_consistency(k1=k1)
    out = []
    for t, (I, P) in enumerate(zip(frames, styl)):
        O, wc = torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda")
        m = torch.empty((H, W), device="cuda", dtype=torch.uint8)
        s.process_frame(to_dev(I), to_dev(P), O, wc, m)
        fl = None
        if t > 0:
            Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            fl = (Fb, Ff)
        s.synchronize()
        out.append((to_np(O), to_np(wc), to_np(m)) + ((to_np(fl[0]), to_np(fl[1])) if fl else (None, None)))
    s.destroy()
    return out


@pytest.mark.parametrize("prec", ["fp16", "fp32", "bf16"])
def test_batch_lanes_equal_independent_streams(prec):
    import torch
    path, _ = weights_file(*NET)
    n_lanes = 3
    counts = [sum(ln in step for step in SCHEDULE) for ln in range(n_lanes)]
    data = [_seq(40 + ln, counts[ln]) for ln in range(n_lanes)]
    k1 = [0.3, 0.6, 0.9]
    want = [_stream_run(path, prec, *data[ln], k1[ln]) for ln in range(n_lanes)]
    b = tc.Batch(W, H, n_lanes, prec, weights_path=path)
    for ln in range(n_lanes):
        b.set_lane_consistency(ln, k1=k1[ln])
    t = [0] * n_lanes
    for step in SCHEDULE:
        I = [to_dev(data[ln][0][t[ln]]) for ln in step]
        P = [to_dev(data[ln][1][t[ln]]) for ln in step]
        O = [torch.empty((3, H, W), device="cuda") for _ in step]
        wc = [torch.empty((H, W), device="cuda") for _ in step]
        m = [torch.empty((H, W), device="cuda", dtype=torch.uint8) for _ in step]
        b.process(step, I, P, O, wc, m)
        flows = {}
        for ln in step:
            if t[ln] > 0:
                Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
                b.get_lane_flows(ln, Fb, Ff)
                flows[ln] = (Fb, Ff)
        b.synchronize()
        for k, ln in enumerate(step):
            w = want[ln][t[ln]]
            assert np.array_equal(to_np(O[k]), w[0]), (step, ln, t[ln])
            assert np.array_equal(to_np(wc[k]), w[1]), (step, ln, t[ln])
            assert np.array_equal(to_np(m[k]), w[2]), (step, ln, t[ln])
            if t[ln] > 0:
                assert np.array_equal(to_np(flows[ln][0]), w[3]) and np.array_equal(to_np(flows[ln][1]), w[4])
            t[ln] += 1
    assert b.tensor_core_layers == (0 if prec == "fp32" else 34)
    b.destroy()


def test_batch_lane_reset_starts_a_new_stream():
    import torch
    path, _ = weights_file(*NET)
    a_frames, a_styl = _seq(50, 3)
    c_frames, c_styl = _seq(51, 3)
    want = _stream_run(path, "fp16", c_frames, c_styl, 0.5)
    b = tc.Batch(W, H, 2, "fp16", weights_path=path)
    b.set_consistency(k1=0.5)
    O = [torch.empty((3, H, W), device="cuda") for _ in range(2)]
    for t in range(3):  # lane 1 runs sequence a
        b.process([1], [to_dev(a_frames[t])], [to_dev(a_styl[t])], [O[1]])
    b.reset_lane(1)
    b.set_lane_consistency(1, k1=0.5)
    for t in range(3):  # lane 1 now runs sequence c from its first frame, beside lane 0
        b.process([0, 1], [to_dev(a_frames[t]), to_dev(c_frames[t])], [to_dev(a_styl[t]), to_dev(c_styl[t])], O)
        b.synchronize()
        assert np.array_equal(to_np(O[1]), want[t][0]), t
    b.destroy()


def test_batch_refuses_stream_only_calls_and_unsupported_settings():
    import torch
    path, _ = weights_file(*NET)
    b = tc.Batch(W, H, 2, "fp16", weights_path=path)
    O = torch.empty((3, H, W), device="cuda")
    with pytest.raises(tc.TcError) as e:
        b.process_frame(O, O, O)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        b.set_pipelined(True)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        b.set_consistency(k1=0.5, solver_iters=10)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
    with pytest.raises(tc.TcError) as e:
        b.process([0, 0], [O, O], [O, O], [O, O])
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    b.destroy()
    with pytest.raises(tc.TcError) as e:
        tc.Batch(W, H, 2, "fp8", weights_path=path)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
