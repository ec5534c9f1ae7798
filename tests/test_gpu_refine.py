"""The refinement network with depthwise-separable convs ("-sepref", Sec. 3.2; TCW2 weight
files) on the GPU against the FP64 oracle: one layer at a time (depthwise on the CUDA cores,
pointwise on the CUDA cores for FP32 and on the tensor cores for BF16), the flows of
streams whose network carries the refinement, graph replay and the precisions that reject
it."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import REL16, nchw_to_nhwc, nhwc_to_nchw, round16, to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

LAYER_CASES = [
    # n, h, w, cin, cout, dil, leaky
    (2, 17, 200, 104, 128, 1, True),
    (2, 33, 130, 128, 96, 16, True),
    (1, 9, 64, 64, 32, 4, True),
    (2, 20, 150, 32, 2, 1, False),
]


def _layer(g, cin, cout):
    return (g.normal(0, 0.3, (cin, 3, 3)), g.normal(0, 0.1, cin), g.normal(0, 1 / np.sqrt(cin), (cout, cin)),
            g.normal(0, 0.1, cout))


@pytest.mark.parametrize("n,h,w,cin,cout,dil,leaky", LAYER_CASES)
def test_sepconv_fp32_matches_oracle(n, h, w, cin, cout, dil, leaky):
    g = synth.rng(130 + cin)
    x = g.normal(size=(n, cin, h, w)).astype(np.float32)
    dw, db, pw, pb = _layer(g, cin, cout)
    got = nhwc_to_nchw(to_np(tc.op_sepconv(to_dev(nchw_to_nhwc(x)), dw, db, pw, pb, dil, leaky, "fp32")))
    for i in range(n):
        d = oracle.depthwise3x3(x[i], dw.astype(np.float32), db.astype(np.float32), dil)
        want = oracle.pointwise(d, pw.astype(np.float32), pb.astype(np.float32), leaky)
        scale = np.abs(pw.astype(np.float32)) @ np.abs(d).reshape(cin, -1)
        err = np.abs(got[i] - want).reshape(cout, -1)
        assert (err <= 1e-5 * (scale + 1.0)).all(), err.max()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n,h,w,cin,cout,dil,leaky", LAYER_CASES)
def test_sepconv_16bit_matches_oracle(prec, n, h, w, cin, cout, dil, leaky):
    """BF16 / FP16: the input is rounded on the host, the depthwise output is stored in the
    16-bit type and so are the pointwise weights; the oracle follows the same roundings in
    FP64, so a difference is at most one 16-bit step of each depthwise output it sums over
    (where FP32 and FP64 round a value on either side of a midpoint) plus the output's own
    rounding."""
    g = synth.rng(140 + cin)
    x = round16(prec, g.normal(size=(n, cin, h, w)).astype(np.float32))
    dw, db, pw, pb = _layer(g, cin, cout)
    got = nhwc_to_nchw(to_np(tc.op_sepconv(to_dev(nchw_to_nhwc(x)), dw, db, pw, pb, dil, leaky, prec)))
    assert tc.op_last_used_tensor_cores()
    pw16 = round16(prec, pw.astype(np.float32))
    step = REL16[prec]
    for i in range(n):
        d = round16(prec, oracle.depthwise3x3(x[i], dw.astype(np.float32), db.astype(np.float32), dil).astype(np.float32))
        want = oracle.pointwise(d, pw16, pb.astype(np.float32), leaky)
        scale = np.abs(pw16) @ np.abs(d).reshape(cin, -1)
        err = np.abs(got[i] - want).reshape(cout, -1)
        bound = step * scale + (step * np.abs(want).reshape(cout, -1) if cout != 2 else 0) + 1e-6
        assert (err <= bound).all(), (err - bound).max()


def _frames(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


def _stream_flows(path, frames, styl, prec):
    import torch
    _, H, W = frames[0].shape
    s = tc.Stream(W, H, prec, weights_path=path)
    out = []
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, H, W), device="cuda")
        s.process_frame(to_dev(I), to_dev(P), O)
        if t > 0:
            Fb = torch.empty((2, H, W), device="cuda")
            Ff = torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            s.synchronize()
            out.append((to_np(Fb), to_np(Ff)))
    layers = s.tensor_core_layers
    s.destroy()
    return out, layers


@pytest.mark.parametrize("chans,radius,W,H", [((16, 32, 48), 3, 64, 64), ((16, 32, 64, 96, 128), 4, 200, 136)])
def test_refined_stream_flows_fp32(chans, radius, W, H):
    path, net = weights_file(chans, radius, refine=True)
    assert len(net.ref) == 7
    frames, styl = _frames(W, H, seed=2, n=3)
    got, _ = _stream_flows(path, frames, styl, "fp32")
    ref = oracle.Stream(net)
    want = [ref.step(I, P) for I, P in zip(frames, styl)][1:]
    # the refinement changes the flow: compare with the net without it
    _, plain = weights_file(chans, radius)
    r0 = oracle.Stream(plain)
    base = [r0.step(I, P) for I, P in zip(frames, styl)][1:]
    assert oracle.epe(want[0]["Fb"], base[0]["Fb"]) > 1e-2
    for (Fb, Ff), r in zip(got, want):
        eb, ef = oracle.epe(Fb, r["Fb"]), oracle.epe(Ff, r["Ff"])
        assert eb <= 1e-3 and ef <= 1e-3, (eb, ef)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_refined_stream_flows_16bit(prec):
    """FP16 meets the fixed 0.05 px bar; BF16 its representation bound 2 u sqrt(n) of the mean
    flow (u = 2^-9, with the 14 refinement convs counted in n)."""
    chans, radius = (16, 32, 64, 96, 128), 4
    path, net = weights_file(chans, radius, refine=True)
    frames, styl = _frames(200, 136, seed=3, n=2)
    got, layers = _stream_flows(path, frames, styl, prec)
    assert layers == 34 + 7  # every pointwise refinement conv on the tensor cores too
    ref = oracle.Stream(net)
    r = [ref.step(I, P) for I, P in zip(frames, styl)][1]
    mag = float(np.sqrt((r["Fb"] ** 2).sum(0)).mean())
    n_layers = 3 * len(chans) + 5 * (len(chans) - 1) + 2 * 7
    bound = 0.05 if prec == "fp16" else max(0.05, 2 * 2.0 ** -9 * np.sqrt(n_layers) * mag)
    eb, ef = oracle.epe(got[0][0], r["Fb"]), oracle.epe(got[0][1], r["Ff"])
    print(f"refined {prec} EPE vs FP64: Fb {eb:.4f} Ff {ef:.4f} (mean |F| {mag:.2f}, bound {bound:.4f})")
    assert eb <= bound and ef <= bound


def test_refined_graph_replay_matches_eager():
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4, refine=True)
    frames, styl = _frames(200, 136, seed=5, n=5)
    runs = []
    for graphs in (False, True):
        s = tc.Stream(200, 136, "bf16", weights_path=path)
        s.set_graphs(graphs)
        outs = []
        for I, P in zip(frames, styl):
            O = torch.empty((3, 136, 200), device="cuda")
            s.process_frame(to_dev(I), to_dev(P), O)
            s.synchronize()
            outs.append(to_np(O))
        s.destroy()
        runs.append(outs)
    for t in range(len(frames)):
        assert np.array_equal(runs[0][t], runs[1][t]), t


def test_refinement_precision_checks():
    path, _ = weights_file((16, 32, 64, 96, 128), 4, refine=True)
    with pytest.raises(tc.TcError) as e:
        tc.Stream(64, 64, "fp8", weights_path=path)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
