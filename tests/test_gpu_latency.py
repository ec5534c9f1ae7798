"""One frame of latency (Sec. 3.1: the next frame in the local term, w_n of Eqs. 2, 3, 6)
on the GPU: the fused consistency stage with the next frame against the FP64 oracle on
identical flows, and streams with tc_set_latency(1) checked stage by stage, end to end
against the oracle's latency stream, against the causal stream at k2 = 0, and for graph
replay, the host entry point, flush and argument checks."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import planar_to_hw2, to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _k8_inputs(W, H, seed=0):
    seq = synth.Sequence(width=W, height=H, seed=seed)
    I = [seq.frame(t) for t in range(3)]
    P = [seq.stylized(t, f) for t, f in enumerate(I)]
    O0 = P[0] + synth.rng(seed + 7).normal(0, 0.01, P[0].shape).astype(np.float32)
    return dict(It=I[1], Pt=P[1], Ip=I[0], Pp=P[0], Op=O0, Fb=seq.flow_backward(1), Ff=seq.flow_forward(1),
                In=I[2], Pn=P[2], Fn=seq.flow_forward(2), Fnb=seq.flow_backward(2))


IMGS = ("It", "Pt", "Ip", "Pp", "Op")
FLOWS = ("Fb", "Ff")
NEXT_IMGS = ("In", "Pn")
NEXT_FLOWS = ("Fn", "Fnb")


def _gpu_next(d, scale=1, lowres=None, **params):
    fl = lowres if lowres is not None else d
    args = [to_dev(d[k]) for k in IMGS] + [to_dev(planar_to_hw2(fl[k])) for k in FLOWS] + \
           [to_dev(d[k]) for k in NEXT_IMGS] + [to_dev(planar_to_hw2(fl[k])) for k in NEXT_FLOWS]
    O, wc, mask = tc.op_consistency_next(*args, scale=scale, **params)
    return to_np(O), to_np(wc), to_np(mask)


def _check_k8(got, ref, wc_tol=2e-4):
    O, wc, mask = got
    band = ref["band"] != 0
    assert band.mean() < 2e-3
    ok = ~band
    mism = (mask != ref["mask"]) & ok
    assert mism.sum() == 0, f"{mism.sum()} mask mismatches outside the band"
    err = np.abs(O - ref["O"]).max(0)
    assert err[ok].max() <= 1e-4, err[ok].max()
    lam = max(1.0, np.abs(ref["wc"]).max())
    assert np.abs(wc - ref["wc"])[ok].max() <= wc_tol * lam


@pytest.mark.parametrize("W,H", [(1920, 1080), (333, 197)])
@pytest.mark.parametrize("alpha,k1,k2", [(6.5e3, 0.3, 0.5), (0.0, 0.45, 0.5), (6.5e3, 0.0, 0.9)])
def test_consistency_next_given_flows(W, H, alpha, k1, k2):
    d = _k8_inputs(W, H)
    params = dict(k1=k1, k2=k2, alpha=alpha, lam=2.0)
    got = _gpu_next(d, **params)
    ref = oracle.consistency_next(*[d[k] for k in IMGS + FLOWS + NEXT_IMGS + NEXT_FLOWS], **params)
    assert 0.3 < (ref["mask"] & 1).mean() < 1.0 and 0.3 < (ref["mask"] >> 1).mean() < 1.0
    _check_k8(got, ref)


@pytest.mark.parametrize("W,H,scale", [(1920, 1080, 4), (250, 130, 4)])
def test_consistency_next_upsampled_flows(W, H, scale):
    d = _k8_inputs(W, H, seed=3)
    fh, fw = -(-H // scale), -(-W // scale)
    fb = synth.random_lowres_flow(fh, fw, 6.0 / scale, 31)
    ff = -fb + synth.random_lowres_flow(fh, fw, 0.6 / scale, 32)
    fn = synth.random_lowres_flow(fh, fw, 6.0 / scale, 33)
    fnb = -fn + synth.random_lowres_flow(fh, fw, 0.6 / scale, 34)
    low = dict(Fb=fb, Ff=ff, Fn=fn, Fnb=fnb)
    full = {k: oracle.upsample_flow(v, scale)[:, :H, :W] for k, v in low.items()}
    params = dict(k1=0.3, k2=0.5, alpha=6.5e3, lam=2.0)
    got = _gpu_next(d, scale=scale, lowres=low, **params)
    ref = oracle.consistency_next(*[d[k] for k in IMGS], full["Fb"], full["Ff"], d["In"], d["Pn"], full["Fn"],
                                  full["Fnb"], **params)
    # in-bounds decisions within 1e-4 px of a frame edge (FP64 vs float32 upsampling)
    yy, xx = np.mgrid[0:H, 0:W]
    for bit, F in ((1, full["Fb"]), (2, full["Fn"])):
        sx, sy = xx + F[0], yy + F[1]
        edge = np.minimum.reduce([np.abs(sx), np.abs(sx - (W - 1)), np.abs(sy), np.abs(sy - (H - 1))]) < 1e-4
        ref["band"] = (ref["band"] | (edge * bit)).astype(np.uint8)
    _check_k8(got, ref)


def test_consistency_next_k2_zero_is_the_causal_stage():
    d = _k8_inputs(333, 197, seed=5)
    params = dict(k1=0.6, alpha=6.5e3, lam=2.0)
    O, wc, mask = _gpu_next(d, k2=0.0, **params)
    Oc, wcc, maskc = tc.op_consistency(*[to_dev(d[k]) for k in IMGS], *[to_dev(planar_to_hw2(d[k])) for k in FLOWS],
                                       scale=1, **params)
    assert np.abs(O - to_np(Oc)).max() <= 1e-6
    assert np.abs(wc - to_np(wcc)).max() <= 1e-6 * 2.0
    assert np.array_equal(mask & 1, to_np(maskc)) and ((mask >> 1) <= 1).all()


def _frames(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


def _hw2(f):
    return f.permute(1, 2, 0).contiguous()


@pytest.mark.parametrize("prec,solver_iters", [("fp32", 0), ("bf16", 0), ("bf16", 150)])
def test_latency_stream_stage_by_stage(prec, solver_iters):
    """Each call with frame n returns frame n - 1: the stream's own flows of the pairs
    (n-1, n-2) and (n, n-1) and its previous output give the expected frame through the
    consistency stage (bit for bit) and, with the solver, the FP64 solve of that A_t."""
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    W, H = 200, 136
    frames, styl = _frames(W, H, seed=6, n=5)
    params = dict(k1=0.3, k2=0.5, alpha=6.5e3, lam=2.0)
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_consistency(solver_iters=solver_iters, **params)
    s.set_latency(1)
    outs, flows = {}, {}
    for n, (I, P) in enumerate(zip(frames, styl)):
        O = torch.full((3, H, W), float("nan"), device="cuda")
        wc = torch.empty((H, W), device="cuda")
        m = torch.empty((H, W), device="cuda", dtype=torch.uint8)
        s.process_frame(to_dev(I), to_dev(P), O, wc, m)
        if n > 0:
            Fb = torch.empty((2, H, W), device="cuda")
            Ff = torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            flows[n] = (Fb, Ff)  # F_{n->n-1}, F_{n-1->n}
        s.synchronize()
        if n == 0:
            assert s.last_output_frame == -1 and torch.isnan(O).all()
            continue
        t = n - 1
        assert s.last_output_frame == t
        outs[t] = O
        if t == 0:
            assert np.array_equal(to_np(O), styl[0]) and (to_np(wc) == 0).all() and (to_np(m) == 0).all()
            continue
        A, wc_ref, m_ref = tc.op_consistency_next(
            to_dev(frames[t]), to_dev(styl[t]), to_dev(frames[t - 1]), to_dev(styl[t - 1]), outs[t - 1],
            _hw2(flows[t][0]), _hw2(flows[t][1]), to_dev(frames[n]), to_dev(styl[n]), _hw2(flows[n][1]),
            _hw2(flows[n][0]), scale=1, **params)
        torch.cuda.synchronize()
        assert np.array_equal(to_np(wc), to_np(wc_ref)) and np.array_equal(to_np(m), to_np(m_ref)), t
        assert (to_np(m) >> 1).any(), "the next frame's warp is never valid"
        if solver_iters == 0:
            assert np.array_equal(to_np(O), to_np(A)), t
        else:
            want = oracle.poisson_solve(styl[t], to_np(A), to_np(wc_ref), iters=solver_iters)
            assert np.abs(to_np(O) - want).max() <= 5e-5, t
    # flush: the last frame, causal blend with the kept flows
    O = torch.empty((3, H, W), device="cuda")
    wc = torch.empty((H, W), device="cuda")
    s.flush(O, wc)
    s.synchronize()
    t = len(frames) - 1
    assert s.last_output_frame == t
    A, wc_ref, _ = tc.op_consistency(to_dev(frames[t]), to_dev(styl[t]), to_dev(frames[t - 1]), to_dev(styl[t - 1]),
                                     outs[t - 1], _hw2(flows[t][0]), _hw2(flows[t][1]), scale=1, **params)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(wc), to_np(wc_ref))
    if solver_iters == 0:
        assert np.array_equal(to_np(O), to_np(A))
    # a new sequence starts after the flush
    s.process_frame(to_dev(frames[0]), to_dev(styl[0]), O)
    assert s.last_output_frame == -1
    s.destroy()


def test_latency_stream_matches_oracle_stream():
    """GPU FP32 against the FP64 oracle's latency stream (alpha = 0, forward-backward test
    off: the blend depends on the flows only through the taps and the in-bounds masks)."""
    import torch
    path, net = weights_file((16, 32, 48), 3)
    d = synth.pair64()
    frames = [d["I0"], d["I1"], d["I1"][:, ::-1].copy(), d["I0"][:, :, ::-1].copy()]
    styl = [d["P0"], d["P1"], d["P1"][:, ::-1].copy(), d["P0"][:, :, ::-1].copy()]
    params = dict(k1=0.3, alpha=0.0, lam=2.0, fb_check=False)
    s = tc.Stream(64, 64, "fp32", weights_path=path)
    s.set_consistency(k2=0.5, **params)
    s.set_latency(1)
    ref = oracle.Stream(net, k2=0.5, latency=1, **params)
    got, want = [], []
    for I, P in zip(frames, styl):
        O = torch.empty((3, 64, 64), device="cuda")
        m = torch.empty((64, 64), device="cuda", dtype=torch.uint8)
        s.process_frame(to_dev(I), to_dev(P), O, None, m)
        s.synchronize()
        r = ref.step(I, P)
        if r is not None:
            got.append((to_np(O), to_np(m)))
            want.append(r)
    O = torch.empty((3, 64, 64), device="cuda")
    m = torch.empty((64, 64), device="cuda", dtype=torch.uint8)
    s.flush(O, None, m)
    s.synchronize()
    got.append((to_np(O), to_np(m)))
    want.append(ref.flush())
    assert len(got) == len(frames)
    for t in range(1, len(frames)):
        O, m = got[t]
        r = want[t]
        same = m == r["mask"]
        assert same.mean() > 0.97, (t, same.mean())
        err = np.abs(O - r["O"]).max(0)
        # pixels whose masks agree: the taps move by the flow deviation (< 1e-3 px; blurred
        # noise has |grad| < 0.5 / px)
        assert err[same].max() <= 2e-3, (t, err[same].max())
    s.destroy()


def test_latency_with_k2_zero_is_the_causal_stream_delayed():
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(200, 136, seed=8, n=4)
    params = dict(k1=0.5, alpha=6.5e3, lam=2.0)
    causal, lat = tc.Stream(200, 136, "bf16", weights_path=path), tc.Stream(200, 136, "bf16", weights_path=path)
    causal.set_consistency(**params)
    lat.set_consistency(k2=0.0, **params)
    lat.set_latency(1)
    a, b = [], []
    for I, P in zip(frames, styl):
        for s, out in ((causal, a), (lat, b)):
            O = torch.empty((3, 136, 200), device="cuda")
            wc = torch.empty((136, 200), device="cuda")
            s.process_frame(to_dev(I), to_dev(P), O, wc)
            s.synchronize()
            if s.last_output_frame >= 0:
                out.append((to_np(O), to_np(wc)))
    O = torch.empty((3, 136, 200), device="cuda")
    wc = torch.empty((136, 200), device="cuda")
    lat.flush(O, wc)
    lat.synchronize()
    b.append((to_np(O), to_np(wc)))
    for t in range(len(frames)):
        assert np.abs(a[t][0] - b[t][0]).max() <= 1e-6, t
        assert np.abs(a[t][1] - b[t][1]).max() <= 2e-6, t
    causal.destroy()
    lat.destroy()


@pytest.mark.parametrize("solver_iters", [0, 40])
def test_latency_graph_replay_matches_eager(solver_iters):
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(200, 136, seed=4, n=6)
    runs = []
    for graphs in (False, True):
        s = tc.Stream(200, 136, "bf16", weights_path=path)
        s.set_graphs(graphs)
        s.set_consistency(solver_iters=solver_iters)
        s.set_latency(1)
        outs = []
        for t, (I, P) in enumerate(zip(frames, styl)):
            s.set_consistency(k1=(0.2, 0.3, 0.4)[t % 3], solver_iters=solver_iters)
            O = torch.empty((3, 136, 200), device="cuda")
            wc = torch.empty((136, 200), device="cuda")
            m = torch.empty((136, 200), device="cuda", dtype=torch.uint8)
            s.process_frame(to_dev(I), to_dev(P), O, wc, m)
            s.synchronize()
            if t > 0:
                outs.append((to_np(O), to_np(wc), to_np(m)))
        O = torch.empty((3, 136, 200), device="cuda")
        s.flush(O)
        s.synchronize()
        outs.append((to_np(O),))
        s.destroy()
        runs.append(outs)
    for t in range(len(runs[0])):
        for k in range(len(runs[0][t])):
            assert np.array_equal(runs[0][t][k], runs[1][t][k]), (t, k)


def test_latency_host_entry_point():
    import torch
    path, _ = weights_file((16, 32, 48), 3)
    frames, styl = _frames(64, 64, seed=2, n=3)
    dev, host = tc.Stream(64, 64, "fp32", weights_path=path), tc.Stream(64, 64, "fp32", weights_path=path)
    for s in (dev, host):
        s.set_latency(1)
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, 64, 64), device="cuda")
        dev.process_frame(to_dev(I), to_dev(P), O)
        hO = np.full((3, 64, 64), -1.0, np.float32)
        host.process_frame_host(np.ascontiguousarray(I), np.ascontiguousarray(P), hO)
        dev.synchronize()
        if t == 0:
            assert (hO == -1.0).all() and host.last_output_frame == -1
        else:
            assert np.array_equal(hO, to_np(O)) and host.last_output_frame == t - 1
    dev.destroy()
    host.destroy()


def test_latency_pipelined_host_entry_point():
    """One frame of latency through tc_process_frame_host_async: the first call writes
    nothing, call t writes frame t - 1, equal to the device entry point's outputs."""
    import torch
    path, _ = weights_file((16, 32, 48), 3)
    frames, styl = _frames(64, 64, seed=3, n=4)
    dev, host = tc.Stream(64, 64, "bf16", weights_path=path), tc.Stream(64, 64, "bf16", weights_path=path)
    for s in (dev, host):
        s.set_latency(1)
    want, outs, keep = [], [], []  # the host buffers live until synchronize()
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, 64, 64), device="cuda")
        dev.process_frame(to_dev(I), to_dev(P), O)
        want.append(to_np(O))
        hI = torch.from_numpy(np.ascontiguousarray(I)).pin_memory()
        hP = torch.from_numpy(np.ascontiguousarray(P)).pin_memory()
        hO = torch.full((3, 64, 64), -1.0).pin_memory()
        host.process_frame_host_async(hI, hP, hO)
        keep += [hI, hP]
        outs.append(hO)
    host.synchronize()
    assert (outs[0].numpy() == -1.0).all()
    for t in range(1, len(frames)):
        assert np.array_equal(outs[t].numpy(), want[t]), t
    dev.destroy()
    host.destroy()


def test_latency_argument_checks():
    import torch
    path, _ = weights_file((16, 32, 48), 3)
    s = tc.Stream(64, 64, "fp32", weights_path=path)
    O = torch.empty((3, 64, 64), device="cuda")
    with pytest.raises(tc.TcError) as e:
        s.flush(O)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        s.set_latency(2)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    s.set_consistency(k1=0.6, k2=0.5)
    with pytest.raises(tc.TcError) as e:
        s.set_latency(1)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    s.set_consistency(k1=0.3, k2=0.5)
    s.set_latency(1)
    with pytest.raises(tc.TcError) as e:
        s.set_consistency(k1=0.6, k2=0.5)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    with pytest.raises(tc.TcError) as e:
        s.flush(O)
    assert e.value.status == tc.TC_ERR_STATE
    d = synth.pair64()
    s.process_frame(to_dev(d["I0"]), to_dev(d["P0"]), O)
    with pytest.raises(tc.TcError) as e:
        s.set_latency(0)
    assert e.value.status == tc.TC_ERR_STATE
    s.flush(O)
    s.synchronize()
    assert np.array_equal(to_np(O), d["P0"]) and s.last_output_frame == 0
    s.set_latency(0)
    s.destroy()
