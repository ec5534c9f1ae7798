"""The E4M3 path: the tensor-core conv against an FP64 conv of the same E4M3 operands, the
amax recorder against the oracle's, and whole streams against the FP64 oracle of the
quantised network (oracle.quant) and of the exact one.

E4M3 keeps 4 significant bits, so the E4M3 network's flow differs from the exact
network's by the quantisation itself (about 10-15 % of the mean flow for the He-init
networks used here, whose random flows are large).  Each E4M3 kernel is held element by
element to an FP64 evaluation of the same codes: it may differ only where float32
arithmetic (instead of FP64) moves a value across an E4M3 rounding midpoint, and then by
one step.  Whole streams are held statistically (see the stream test for why)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import nchw_to_nhwc, nhwc_to_nchw, to_dev, to_np, weight_scales_e4m3, weights_file
from oracle import quant

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _pair(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


# --------------------------------------------------------------------------------- stages

def _check_e4m3(got, pre, S, rel=1e-5):
    """got: E4M3 outputs of a kernel; pre: the FP64 value before the output rounding; S: the
    scale of the kernel's float32 arithmetic error (sum of |terms|).  Outputs equal
    e4m3(pre) except where pre lies within rel * S of a rounding midpoint, and there they are
    the other neighbour.  Returns (disagreements, outputs)."""
    ref = quant.e4m3(pre)
    got = np.asarray(got, np.float64)
    d = got != ref
    if d.any():
        lo, hi = np.minimum(got[d], ref[d]), np.maximum(got[d], ref[d])
        assert np.array_equal(quant.e4m3((lo + hi) / 2 + (hi - lo) * 1e-9), hi)   # neighbours
        assert np.array_equal(quant.e4m3((lo + hi) / 2 - (hi - lo) * 1e-9), lo)
        assert (np.abs(pre[d] - (lo + hi) / 2) <= rel * S[d]).all()
    return int(d.sum()), d.size


@pytest.mark.parametrize("n,h,w,c,r", [(2, 19, 21, 32, 4), (1, 34, 60, 128, 4), (2, 8, 8, 48, 3), (2, 33, 47, 16, 2),
                                       (3, 68, 120, 96, 4), (2, 136, 240, 64, 4)])
def test_correlation_e4m3_matches_fp64_of_the_same_codes(n, h, w, c, r):
    g = synth.rng(32)
    f1 = quant.e4m3(2.0 * g.normal(size=(n, c, h, w))).astype(np.float32)
    f2 = quant.e4m3(2.0 * g.normal(size=(n, c, h, w))).astype(np.float32)
    got = to_np(tc.op_correlation(to_dev(nchw_to_nhwc(f1)), to_dev(nchw_to_nhwc(f2)), r, precision="fp8"))
    assert tc.op_last_used_tensor_cores()
    flips = total = 0
    for i in range(n):
        pre = oracle.correlation(f1[i], f2[i], r)
        S = oracle.correlation(np.abs(f1[i]), np.abs(f2[i]), r)
        k, t = _check_e4m3(nhwc_to_nchw(got[i:i + 1])[0], pre, S)
        flips, total = flips + k, total + t
    assert flips <= max(2, 1e-3 * total), (flips, total)


def test_correlation_e4m3_rejects_ragged_channels():
    import torch
    x = torch.zeros((1, 8, 8, 24), device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.op_correlation(x, x, 2, precision="fp8")
    assert e.value.status == tc.TC_ERR_UNSUPPORTED


@pytest.mark.parametrize("n,h,w,c,mag", [(2, 17, 23, 16, 3.0), (1, 34, 60, 128, 6.0), (2, 136, 240, 64, 2.0)])
def test_warp_e4m3_matches_fp64_of_the_same_codes(n, h, w, c, mag):
    g = synth.rng(33)
    f = quant.e4m3(2.0 * g.normal(size=(n, c, h, w))).astype(np.float32)
    flow = g.uniform(-mag, mag, (n, 2, h, w)).astype(np.float32)
    got = to_np(tc.op_warp_features(to_dev(nchw_to_nhwc(f)), to_dev(np.moveaxis(flow, 1, -1)), precision="fp8"))
    flips = total = 0
    for i in range(n):
        pre, _ = oracle.warp(f[i], flow[i], 1)
        S, _ = oracle.warp(np.abs(f[i]), flow[i], 1)
        k, t = _check_e4m3(nhwc_to_nchw(got[i:i + 1])[0], pre, S)
        flips, total = flips + k, total + t
    assert flips <= max(2, 1e-3 * total), (flips, total)


# ---------------------------------------------------------------------------- stage: conv

CONV_CASES = [
    # n, h, w, cin, cout, stride: 128-pixel tiles with ragged tails, channel tails, stride 2
    (1, 9, 13, 16, 16, 1), (2, 17, 30, 32, 32, 2), (2, 34, 60, 128, 128, 1), (1, 33, 47, 120, 128, 1),
    (2, 20, 36, 160, 32, 1), (1, 68, 120, 96, 64, 1), (1, 11, 7, 8, 2, 1), (2, 64, 72, 64, 96, 2),
    (1, 5, 6, 6, 10, 1), (2, 3, 130, 216, 128, 1), (1, 7, 300, 16, 16, 2), (1, 40, 260, 48, 48, 1),
]


@pytest.mark.parametrize("n,h,w,cin,cout,stride", CONV_CASES)
def test_conv3x3_e4m3_matches_fp64_of_the_same_codes(n, h, w, cin, cout, stride):
    g = synth.rng(31)
    x = (2.0 * g.normal(size=(n, cin, h, w))).astype(np.float32)
    wt = (g.normal(size=(cout, cin, 3, 3)) / np.sqrt(9 * cin)).astype(np.float32)
    b = g.normal(0, 0.1, cout).astype(np.float32)
    got = to_np(tc.op_conv3x3(to_dev(nchw_to_nhwc(x)), wt, b, stride=stride, leaky=True, precision="fp8"))
    assert tc.op_last_used_tensor_cores()
    # the operands the tensor cores multiply: e4m3(x) (scale 1) and e4m3(w / s_w) s_w
    sw = weight_scales_e4m3(wt)
    wq = quant.e4m3((wt / sw[:, None, None, None]).astype(np.float32)) * sw[:, None, None, None].astype(np.float64)
    xq = quant.e4m3(x)
    flips = total = 0
    for i in range(n):
        pre = oracle.conv3x3(xq[i], wq, b, stride=stride, leaky=True)   # before the output rounding
        # scale of the float32 accumulation error: sum of |products| (+ |bias|)
        S = oracle.conv3x3(np.abs(xq[i]), np.abs(wq), np.abs(b), stride=stride, leaky=False)
        ref = quant.e4m3(pre)
        g_ = nhwc_to_nchw(got[i:i + 1])[0].astype(np.float64)
        d = g_ != ref
        total += d.size
        flips += int(d.sum())
        if d.any():
            # a disagreement is one E4M3 step, at a value within float32 accumulation error of
            # the midpoint between the two neighbours
            lo, hi = np.minimum(g_[d], ref[d]), np.maximum(g_[d], ref[d])
            assert np.array_equal(quant.e4m3((lo + hi) / 2 + (hi - lo) * 1e-9), hi)
            assert np.array_equal(quant.e4m3((lo + hi) / 2 - (hi - lo) * 1e-9), lo)
            mid = (lo + hi) / 2
            assert (np.abs(pre[d] - mid) <= 1e-5 * S[d]).all()
    assert flips <= max(2, 1e-3 * total), (flips, total)


def test_conv_e4m3_rejects_wide_layers():
    import torch
    x = torch.zeros((1, 8, 8, 16), device="cuda")
    with pytest.raises(tc.TcError) as e:
        tc.op_conv3x3(x, np.zeros((144, 16, 3, 3), np.float32), np.zeros(144, np.float32), precision="fp8")
    assert e.value.status == tc.TC_ERR_UNSUPPORTED


# ------------------------------------------------------------------------- calibration

NETS = [((16, 32, 48), 3, 18), ((16, 32, 64, 96, 128), 4, 34)]


@pytest.mark.parametrize("chans,radius,want", NETS)
def test_fp8_stream_needs_scales_then_plans_everything_on_tensor_cores(chans, radius, want):
    import torch
    path, net = weights_file(chans, radius)
    s = tc.Stream(96, 64, "fp8", weights_path=path)
    n = s.activation_segments
    assert n == quant.segments(net) == 3 * len(chans) + 6 * (len(chans) - 1)
    assert s.tensor_core_layers == 0
    I = torch.zeros((3, 64, 96), device="cuda")
    with pytest.raises(tc.TcError) as e:
        s.process_frame(I, I, torch.empty_like(I))
    assert e.value.status == tc.TC_ERR_STATE
    for bad in (np.ones(n - 1), -np.ones(n), np.full(n, np.nan)):
        with pytest.raises(tc.TcError) as e:
            s.set_fp8_scales(bad)
        assert e.value.status == tc.TC_ERR_INVALID_ARG
    with pytest.raises(tc.TcError) as e:
        s.set_amax_recording(True)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    s.set_fp8_scales(np.ones(n))
    assert s.tensor_core_layers == want
    assert s.tensor_core_correlation_levels == len(chans) - 1
    s.set_fp8_scales(np.full(n, 0.5))                  # re-calibration re-plans, same counts
    assert s.tensor_core_layers == want
    s.process_frame(I, I, torch.empty_like(I))
    s.synchronize()
    s.destroy()
    b = tc.Stream(96, 64, "bf16", weights_path=path)
    with pytest.raises(tc.TcError) as e:
        b.set_fp8_scales(np.ones(n))
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    b.destroy()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_amax_recording_matches_oracle(prec):
    import torch
    chans, radius = (16, 32, 64, 96, 128), 4
    path, net = weights_file(chans, radius)
    W, H = 200, 136
    frames, styl = _pair(W, H, seed=5, n=3)
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_amax_recording(True)
    for I, P in zip(frames, styl):
        s.process_frame(to_dev(I), to_dev(P), torch.empty((3, H, W), device="cuda"))
    got = s.get_amax().astype(np.float64)
    s.destroy()
    want = quant.calibrate(net, frames)
    assert (got == 0).tolist() == (want == 0).tolist()
    # float32: activations within ~1e-5 relative of FP64.  bfloat16: each of the n layers
    # on a value's path adds a relative error of about u = 2^-9, independent ones adding up
    # to about u sqrt(n); the bound allows twice that for the deepest segment.
    n_layers = 3 * len(chans) + 5 * (len(chans) - 1)
    rtol = 1e-4 if prec == "fp32" else 2 * 2.0 ** -9 * np.sqrt(n_layers)
    nz = want > 0
    rel = np.abs(got[nz] - want[nz]) / want[nz]
    print(f"{prec} amax: max relative deviation {rel.max():.2e} over {nz.sum()} segments")
    assert rel.max() <= rtol, rel.max()


# ----------------------------------------------------------------------------- streams

STREAMS = [
    ("64x48 3-level r3", (16, 32, 48), 3, 64, 48),
    ("200x136 5-level r4", (16, 32, 64, 96, 128), 4, 200, 136),
]


def _fp8_stream_flows(path, scales, frames, styl):
    import torch
    _, H, W = frames[0].shape
    s = tc.Stream(W, H, "fp8", weights_path=path)
    s.set_fp8_scales(scales)
    flows = []
    for t, (I, P) in enumerate(zip(frames, styl)):
        s.process_frame(to_dev(I), to_dev(P), torch.empty((3, H, W), device="cuda"))
        if t > 0:
            Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            flows.append((to_np(Fb), to_np(Ff)))
    s.synchronize()
    s.destroy()
    return flows


@pytest.mark.parametrize("name,chans,radius,W,H", STREAMS)
def test_fp8_stream_error_is_the_quantisation_error(name, chans, radius, W, H):
    """The E4M3 network is chaotic on its grid: one code moved by one step at the coarsest
    features moves the oracle's quantised flow by ~0.07 px, a quarter of the whole
    quantisation error, so float32-vs-FP64 rounding flips make the GPU and the quantised
    oracle two draws of the same quantisation noise rather than close copies.  Element-wise
    parity of the E4M3 kernels is held by the stage tests above; here the stream's error
    against the exact FP64 network must be the quantisation error itself, on average over
    3 frame pairs x 2 directions: within 0.7-1.3x of the quantised oracle's."""
    path, net = weights_file(chans, radius)
    calib, _ = _pair(W, H, seed=40, n=3)             # calibration frames: another sequence
    sc = quant.scales_from_amax(quant.calibrate(net, calib)).astype(np.float32)
    frames, styl = _pair(W, H, seed=1, n=4)
    got = _fp8_stream_flows(path, sc, frames, styl)
    e_q, e_x, e_qx, mag = [], [], [], []
    for t in range(1, len(frames)):
        q = quant.flow_pair_q(net, frames[t], frames[t - 1], scales=sc.astype(np.float64))
        x = oracle.flow_pair(net, frames[t], frames[t - 1])
        for k in range(2):
            e_q.append(oracle.epe(got[t - 1][k], q[k]))         # GPU vs quantised oracle
            e_x.append(oracle.epe(got[t - 1][k], x[k]))         # GPU vs exact oracle
            e_qx.append(oracle.epe(q[k], x[k]))                 # what quantising costs
            mag.append(float(np.sqrt((x[k] ** 2).sum(0)).mean()))
    E_q, E_x, E_qx = np.mean(e_q), np.mean(e_x), np.mean(e_qx)
    print(f"{name}: e4m3 EPE vs exact FP64 oracle {E_x:.4f} px, quantised oracle vs exact {E_qx:.4f} px, "
          f"GPU vs quantised oracle {E_q:.4f} px (mean |F| {np.mean(mag):.2f} px)")
    assert 0.7 * E_qx <= E_x <= 1.3 * E_qx, (E_x, E_qx)
    assert E_q <= 1.5 * E_qx, (E_q, E_qx)


def test_fp8_graph_replay_matches_eager_launches():
    import torch
    chans, radius = (16, 32, 64, 96, 128), 4
    path, net = weights_file(chans, radius)
    W, H = 200, 136
    calib, _ = _pair(W, H, seed=40, n=2)
    sc = quant.scales_from_amax(quant.calibrate(net, calib)).astype(np.float32)
    frames, styl = _pair(W, H, seed=4, n=5)
    runs = []
    for graphs in (False, True):
        s = tc.Stream(W, H, "fp8", weights_path=path)
        s.set_fp8_scales(sc)
        s.set_graphs(graphs)
        outs = []
        for t, (I, P) in enumerate(zip(frames, styl)):
            O = torch.empty((3, H, W), device="cuda")
            m = torch.empty((H, W), device="cuda", dtype=torch.uint8)
            s.process_frame(to_dev(I), to_dev(P), O, None, m)
            Fb = torch.empty((2, H, W), device="cuda")
            if t > 0:
                s.get_flows(Fb, None)
            s.synchronize()
            outs.append((to_np(O), to_np(m), to_np(Fb) if t > 0 else None))
        s.destroy()
        runs.append(outs)
    for t in range(len(frames)):
        assert np.array_equal(runs[0][t][0], runs[1][t][0]) and np.array_equal(runs[0][t][1], runs[1][t][1])
        if t > 0:
            assert np.array_equal(runs[0][t][2], runs[1][t][2])
