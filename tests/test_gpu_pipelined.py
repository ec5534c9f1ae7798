"""Pipelined mode (tc_set_pipelined): frame t + 1's feature pyramid runs on its own stream
while earlier frames' flows are estimated, with four pyramid slots, two sets of estimator
buffers (two estimations in flight) and the frame split into pyramid, estimation and blend
graphs.  The results must equal the default mode's bit for bit, frame by frame, over enough
frames that every graph is captured and replayed (t % 4 for each of the three graph kinds)."""
import numpy as np
import pytest

import synth
from gpu_common import to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

W, H = 200, 136


def _frames(n, seed):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(16, 34), max_vel=2.0)
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


def _run(path, frames, styl, prec, pipelined, latency=0, flow_downscale=0, solver_iters=0):
    """Every frame's outputs (O, w_c, mask) and, at the end, the last frame's flows."""
    import torch
    s = tc.Stream(W, H, prec, weights_path=path, flow_downscale=flow_downscale)
    k2 = 0.4 if latency else 0.0
    if latency:
        s.set_consistency(k1=0.3, k2=k2, solver_iters=solver_iters)
        s.set_latency(1)
    s.set_pipelined(pipelined)
    # inputs resident and unmodified, one output set per frame (pipelined frames overlap)
    dI, dP = [to_dev(I) for I in frames], [to_dev(P) for P in styl]
    outs = [(torch.empty((3, H, W), device="cuda"), torch.empty((H, W), device="cuda"),
             torch.empty((H, W), device="cuda", dtype=torch.uint8)) for _ in range(len(frames) + 1)]
    for t in range(len(frames)):
        s.set_consistency(k1=(0.2, 0.5, 0.9)[t % 3] * (0.5 if latency else 1.0), k2=k2, solver_iters=solver_iters)
        s.process_frame(dI[t], dP[t], *outs[t])
    if latency:
        s.flush(*outs[len(frames)])
    Fb = torch.empty((2, H, W), device="cuda")
    Ff = torch.empty((2, H, W), device="cuda")
    if not latency:
        s.get_flows(Fb, Ff)
    s.join()
    torch.cuda.synchronize()
    res = [tuple(to_np(x) for x in o) for o in outs[:len(frames) + (1 if latency else 0)]]
    flows = (to_np(Fb), to_np(Ff)) if not latency else None
    s.destroy()
    return res, flows


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_pipelined_matches_default(prec):
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(14, seed=11)
    a, fa = _run(path, frames, styl, prec, False)
    b, fb = _run(path, frames, styl, prec, True)
    for t in range(len(frames)):
        for k in range(3):
            assert np.array_equal(a[t][k], b[t][k]), (t, k)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])


def test_pipelined_latency_and_flush():
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(9, seed=12)
    a, _ = _run(path, frames, styl, "bf16", False, latency=1)
    b, _ = _run(path, frames, styl, "bf16", True, latency=1)
    for t in range(1, len(a)):  # the first call of a latency-1 sequence writes nothing
        for k in range(3):
            assert np.array_equal(a[t][k], b[t][k]), (t, k)


@pytest.mark.parametrize("flow_downscale,solver_iters", [(2, 0), (1, 12)])
def test_pipelined_fast_preset_and_solver(flow_downscale, solver_iters):
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(8, seed=13)
    a, _ = _run(path, frames, styl, "bf16", False, flow_downscale=flow_downscale, solver_iters=solver_iters)
    b, _ = _run(path, frames, styl, "bf16", True, flow_downscale=flow_downscale, solver_iters=solver_iters)
    for t in range(len(frames)):
        for k in range(3):
            assert np.array_equal(a[t][k], b[t][k]), (t, k)


def test_pipelined_refinement():
    """The network with the depthwise-separable refinement: its buffers are per set too."""
    path, _ = weights_file((16, 32, 64, 96, 128), 4, refine=True)
    frames, styl = _frames(8, seed=15)
    a, fa = _run(path, frames, styl, "bf16", False)
    b, fb = _run(path, frames, styl, "bf16", True)
    for t in range(len(frames)):
        for k in range(3):
            assert np.array_equal(a[t][k], b[t][k]), (t, k)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])


_REF_1080 = {}


def _ref_1080p():
    """Frames 0-2 of the seeded 1920x1080 sequence, the FP64 oracle's flows of the pair
    (2, 1), and the FP32 path's flows of the same pair (computed once per process)."""
    import oracle
    import torch
    if not _REF_1080:
        path, net = weights_file((16, 32, 64, 96, 128), 4)
        seq = synth.Sequence(seed=0)
        frames = [seq.frame(t) for t in range(3)]
        styl = [seq.stylized(t, f) for t, f in enumerate(frames)]
        _, h, w = frames[0].shape
        s = tc.Stream(w, h, "fp32", weights_path=path)
        O = torch.empty((3, h, w), device="cuda")
        for t in (1, 2):
            s.process_frame(to_dev(frames[t]), to_dev(styl[t]), O)
        Fb, Ff = torch.empty((2, h, w), device="cuda"), torch.empty((2, h, w), device="cuda")
        s.get_flows(Fb, Ff)
        torch.cuda.synchronize()
        fp32 = (to_np(Fb), to_np(Ff))
        s.destroy()
        _REF_1080.update(path=path, frames=frames, styl=styl, oracle=oracle.flow_pair(net, frames[2], frames[1]),
                         fp32=fp32)
    return _REF_1080


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_pipelined_1080p_matches_default_and_fixed_epe(prec):
    """The configuration the benchmark times: 1920x1080, the 5-level r = 4 network, pipelined
    mode with CUDA graphs (frame 2 is captured and replayed).  Every frame's outputs equal the
    default mode's bit for bit.  The flows of the last pair are compared with the FP32 path's
    flows and with the FP64 oracle's.

    FP16 is held to the fixed-EPE bar of the precision variants: EPE <= 0.05 px per direction
    against the FP32 result, and against the FP64 oracle (measured ~0.02 px at a 21 px mean
    flow).  BF16 cannot meet that bar with these weights: rounding the He-init weights alone
    to bfloat16, with every activation exact, moves the flows by ~0.12 px (the FP64
    attribution in test_precision_cpu.py), so BF16 is held to its representation bound
    2 u sqrt(n) of the mean flow (u = 2^-9, n = 35 conv layers on the path to the flow) and
    reported as not at fixed EPE."""
    import oracle
    import torch
    R = _ref_1080p()
    frames, styl = R["frames"], R["styl"]
    _, h, w = frames[0].shape
    dI, dP = [to_dev(I) for I in frames], [to_dev(P) for P in styl]
    res = []
    for pipelined in (False, True):
        s = tc.Stream(w, h, prec, weights_path=R["path"])
        s.set_pipelined(pipelined)
        outs = [(torch.empty((3, h, w), device="cuda"), torch.empty((h, w), device="cuda"),
                 torch.empty((h, w), device="cuda", dtype=torch.uint8)) for _ in frames]
        for t in range(len(frames)):
            s.set_consistency(k1=(0.0, 0.5, 1.0)[t])
            s.process_frame(dI[t], dP[t], *outs[t])
        Fb, Ff = torch.empty((2, h, w), device="cuda"), torch.empty((2, h, w), device="cuda")
        s.get_flows(Fb, Ff)
        s.join()
        torch.cuda.synchronize()
        res.append(([tuple(to_np(x) for x in o) for o in outs], (to_np(Fb), to_np(Ff))))
        s.destroy()
    (a, fa), (b, fb) = res
    for t in range(len(frames)):
        for k in range(3):
            assert np.array_equal(a[t][k], b[t][k]), (t, k)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    ref_b, ref_f = R["oracle"]
    f32_b, f32_f = R["fp32"]
    eb, ef = oracle.epe(fb[0], ref_b), oracle.epe(fb[1], ref_f)
    qb, qf = oracle.epe(fb[0], f32_b), oracle.epe(fb[1], f32_f)
    mag = float(np.sqrt((ref_b ** 2).sum(0)).mean())
    print(f"1080p {prec} pipelined EPE vs FP32 path: Fb {qb:.4f} px, Ff {qf:.4f} px; vs FP64 oracle: "
          f"Fb {eb:.4f} px, Ff {ef:.4f} px (mean |F| {mag:.2f} px)")
    # the FP32 path itself is within 1e-3 px of the oracle at this size
    assert oracle.epe(f32_b, ref_b) <= 1e-3 and oracle.epe(f32_f, ref_f) <= 1e-3
    if prec == "fp16":
        assert max(qb, qf) <= 0.05, (qb, qf)
        assert max(eb, ef) <= 0.05, (eb, ef)
    else:
        bound = 2 * 2.0 ** -9 * np.sqrt(35) * mag
        assert max(qb, qf, eb, ef) <= bound, (qb, qf, eb, ef, bound)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_pipelined_host_async_matches_default(prec):
    """tc_process_frame_host_async and its 8-bit form in pipelined mode (four staging slots,
    each upload fenced to the frame's pyramid and blend streams, each download to its blend):
    14 frames enqueued back to back from page-locked buffers give the default mode's outputs
    bit for bit (the 8-bit form: the default mode on the decoded frames, quantised)."""
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(14, seed=21)
    q8 = lambda a: np.ascontiguousarray(np.moveaxis(
        np.floor(np.clip(np.asarray(a, np.float64), 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8), 0, -1))
    dec = lambda q: np.ascontiguousarray(np.moveaxis(q, -1, 0).astype(np.float32) / np.float32(255.0))
    quant = lambda O: np.ascontiguousarray(np.moveaxis(np.floor(
        np.clip(O, np.float32(0), np.float32(1)) * np.float32(255.0) + np.float32(0.5)).astype(np.uint8), 0, -1))
    f8, s8 = [q8(a) for a in frames], [q8(a) for a in styl]
    want32, _ = _run(path, frames, styl, prec, False)
    want8, _ = _run(path, [dec(a) for a in f8], [dec(a) for a in s8], prec, False)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    for rgb8 in (False, True):
        s = tc.Stream(W, H, prec, weights_path=path)
        s.set_pipelined(True)
        hI = [pin(a) for a in (f8 if rgb8 else frames)]
        hP = [pin(a) for a in (s8 if rgb8 else styl)]
        outs = [((torch.empty((H, W, 3), dtype=torch.uint8) if rgb8 else torch.empty((3, H, W))).pin_memory(),
                 torch.empty((H, W)).pin_memory(), torch.empty((H, W), dtype=torch.uint8).pin_memory())
                for _ in frames]
        call = s.process_frame_host_rgb8_async if rgb8 else s.process_frame_host_async
        for t in range(len(frames)):
            s.set_consistency(k1=(0.2, 0.5, 0.9)[t % 3])
            call(hI[t], hP[t], *outs[t])
        s.synchronize()
        s.destroy()
        for t in range(len(frames)):
            O, wc, m = (o.numpy() for o in outs[t])
            want = want8[t] if rgb8 else want32[t]
            assert np.array_equal(O, quant(want[0]) if rgb8 else want[0]), (rgb8, t)
            assert np.array_equal(wc, want[1]) and np.array_equal(m, want[2]), (rgb8, t)


def test_pipelined_state_errors():
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(2, seed=14)
    s = tc.Stream(W, H, "bf16", weights_path=path)
    O = torch.empty((3, H, W), device="cuda")
    s.process_frame(to_dev(frames[0]), to_dev(styl[0]), O)
    with pytest.raises(tc.TcError, match="TC_ERR_STATE"):
        s.set_pipelined(True)  # after the first frame of a sequence
    s.destroy()
    s = tc.Stream(W, H, "bf16", weights_path=path)
    s.set_pipelined(True)
    with pytest.raises(tc.TcError, match="TC_ERR_STATE"):
        s.process_frame_host(np.ascontiguousarray(frames[0]), np.ascontiguousarray(styl[0]),
                             np.empty((3, H, W), np.float32))
    with pytest.raises(tc.TcError, match="TC_ERR_STATE"):
        s.set_amax_recording(True)
    s.destroy()
    torch.cuda.synchronize()


def test_pipelined_frame_timing_records_every_frame():
    """tc_set_frame_timing: one latency per frame given in pipelined mode (device time from
    the moment its pyramid may start to the end of its blend), positive and finite; the
    recording changes no result."""
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(10, seed=16)
    a, _ = _run(path, frames, styl, "fp16", True)
    import torch
    s = tc.Stream(W, H, "fp16", weights_path=path)
    s.set_pipelined(True)
    s.set_frame_timing(True)
    dI, dP = [to_dev(I) for I in frames], [to_dev(P) for P in styl]
    outs = [torch.empty((3, H, W), device="cuda") for _ in frames]
    for t in range(len(frames)):
        s.set_consistency(k1=(0.2, 0.5, 0.9)[t % 3])
        s.process_frame(dI[t], dP[t], outs[t])
    times = s.get_frame_times()
    s.join()
    torch.cuda.synchronize()
    assert len(times) == len(frames) and np.isfinite(times).all() and (times > 0).all()
    for t in range(len(frames)):
        assert np.array_equal(to_np(outs[t]), a[t][0]), t
    s.destroy()
