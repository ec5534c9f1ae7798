"""The fast preset (Table 3: the flow network on frames downscaled by 2, 50 solver
iterations) on the GPU against the FP64 oracle: the 2x2 downscale, the flows of a stream
with flow_downscale = 2, the frame outputs stage by stage with the solver, graph replay and
argument checks."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


@pytest.mark.parametrize("c,h,w", [(3, 1080, 1920), (3, 137, 201), (1, 1, 7), (2, 5, 1)])
def test_downscale2_matches_oracle(c, h, w):
    x = synth.rng(95).random((c, h, w)).astype(np.float32)
    got = to_np(tc.op_downscale2(to_dev(x)))
    want = oracle.downscale2(x)
    assert got.shape == want.shape
    # four float32 values summed in two pairs: within 2 ulp of the FP64 mean
    assert np.abs(got - want).max() <= 2 * 2.0 ** -24


def _frames(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


@pytest.mark.parametrize("chans,radius,W,H", [((16, 32, 48), 3, 64, 64), ((16, 32, 64, 96, 128), 4, 200, 136),
                                              ((16, 32, 48), 3, 67, 45)])
def test_fast_preset_flows_fp32(chans, radius, W, H):
    import torch
    path, net = weights_file(chans, radius)
    frames, styl = _frames(W, H, seed=1, n=3)
    s = tc.Stream(W, H, "fp32", weights_path=path, flow_downscale=2)
    ref = oracle.Stream(net, flow_downscale=2)
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, H, W), device="cuda")
        s.process_frame(to_dev(I), to_dev(P), O)
        r = ref.step(I, P)
        if t == 0:
            continue
        Fb = torch.empty((2, H, W), device="cuda")
        Ff = torch.empty((2, H, W), device="cuda")
        s.get_flows(Fb, Ff)
        s.synchronize()
        eb, ef = oracle.epe(to_np(Fb), r["Fb"]), oracle.epe(to_np(Ff), r["Ff"])
        assert eb <= 1e-3 and ef <= 1e-3, (t, eb, ef)
    s.destroy()


def _hw2(f):
    return f.permute(1, 2, 0).contiguous()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_fast_preset_stage_by_stage(prec):
    """Frames of a fast-preset stream (flow at half size, 50 iterations): the stream's own
    full-size flows and previous output give A_t and w_c through the consistency stage, and
    the output is the FP64 solve of that A_t."""
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    W, H = 200, 136
    frames, styl = _frames(W, H, seed=7, n=4)
    params = dict(k1=0.5, alpha=6.5e3, lam=2.0)
    s = tc.Stream(W, H, prec, weights_path=path, flow_downscale=2)
    s.set_consistency(solver_iters=50, **params)
    prev = None
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, H, W), device="cuda")
        wc = torch.empty((H, W), device="cuda")
        s.process_frame(to_dev(I), to_dev(P), O, wc)
        if t > 0:
            Fb = torch.empty((2, H, W), device="cuda")
            Ff = torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            s.synchronize()
            A, wc_ref, _ = tc.op_consistency(to_dev(I), to_dev(P), to_dev(prev[0]), to_dev(prev[1]), prev[2],
                                             _hw2(Fb), _hw2(Ff), scale=1, **params)
            torch.cuda.synchronize()
            assert np.array_equal(to_np(wc), to_np(wc_ref)), t
            want = oracle.poisson_solve(P, to_np(A), to_np(wc_ref), iters=50)
            assert np.abs(to_np(O) - want).max() <= 5e-5, t
        prev = (I, P, O)
    s.destroy()


def test_fast_preset_graph_replay_matches_eager():
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(200, 136, seed=4, n=5)
    runs = []
    for graphs in (False, True):
        s = tc.Stream(200, 136, "bf16", weights_path=path, flow_downscale=2)
        s.set_graphs(graphs)
        outs = []
        for t, (I, P) in enumerate(zip(frames, styl)):
            s.set_consistency(k1=(0.2, 0.5, 0.9)[t % 3], solver_iters=50)
            O = torch.empty((3, 136, 200), device="cuda")
            wc = torch.empty((136, 200), device="cuda")
            s.process_frame(to_dev(I), to_dev(P), O, wc)
            s.synchronize()
            outs.append((to_np(O), to_np(wc)))
        s.destroy()
        runs.append(outs)
    for t in range(len(frames)):
        assert np.array_equal(runs[0][t][0], runs[1][t][0]) and np.array_equal(runs[0][t][1], runs[1][t][1]), t


def test_fast_preset_argument_checks():
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    with pytest.raises(tc.TcError) as e:
        tc.Stream(64, 64, "bf16", weights_path=path, flow_downscale=3)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    # half of 40 is below 2^5
    with pytest.raises(tc.TcError) as e:
        tc.Stream(40, 64, "bf16", weights_path=path, flow_downscale=2)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    s = tc.Stream(64, 64, "bf16", weights_path=path, flow_downscale=2)
    s.destroy()
