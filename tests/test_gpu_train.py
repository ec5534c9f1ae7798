"""Training (tc_trainer_*, the stage backward passes, the brute-force flow) against the FP64
oracle.

Gradients are checked against central finite differences of the ORACLE's forward (FP64, so
the difference quotient is accurate to ~1e-9): for random directions V and cotangents U,
<grad, V> from the CUDA backward must match (L(p + hV) - L(p - hV)) / 2h with
L = <oracle forward, U>.  The functions are piecewise smooth (LeakyReLU, bilinear cells,
the EPE norm); with h = 1e-7 (1e-6 where no kink is near) a kink is crossed only by values
within ~h of it, which the random inputs avoid (warp flows keep their fractional parts inside (0.1, 0.9)).  The CUDA
side accumulates in float32, so agreement is held to 1e-4 relative (1e-3 for the whole
network, whose gradient sums over ~1e5 products per weight).
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from gpu_common import nchw_to_nhwc, nhwc_to_nchw, to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _train():
    import paper_2301_00750_b300.train as tr
    return tr


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-12)


# ------------------------------------------------------------------- stage backward

@pytest.mark.parametrize("n,h,w,cin,cout,stride,leaky", [
    (2, 9, 13, 8, 16, 1, True), (1, 12, 10, 16, 32, 2, True), (2, 7, 11, 3, 10, 2, True),
    (1, 16, 16, 24, 2, 1, False), (1, 9, 20, 115, 32, 1, True),
])
def test_conv_backward_matches_oracle_finite_differences(n, h, w, cin, cout, stride, leaky):
    import torch
    g = synth.rng(50)
    x = g.normal(size=(n, cin, h, w))
    wt = g.normal(size=(cout, cin, 3, 3)) / np.sqrt(9 * cin)
    b = g.normal(0, 0.1, cout)
    ho, wo = (h - 1) // stride + 1, (w - 1) // stride + 1
    U = g.normal(size=(n, cout, ho, wo))
    xd = to_dev(nchw_to_nhwc(x.astype(np.float32)))
    y = tc.op_conv3x3(xd, wt.astype(np.float32), b.astype(np.float32), stride=stride, leaky=leaky)
    dy = to_dev(nchw_to_nhwc(U.astype(np.float32)))
    dx = torch.empty_like(xd)
    dw = torch.empty((cout, cin, 3, 3), device="cuda")
    db = torch.empty((cout,), device="cuda")
    tr = _train()
    tc._check(tr._lib.tc_op_conv3x3_backward(xd.data_ptr(), n, h, w, cin, to_dev(wt).data_ptr(), cout, stride,
                                             int(leaky), y.data_ptr(), dy.data_ptr(), dx.data_ptr(), dw.data_ptr(),
                                             db.data_ptr(), None))
    torch.cuda.synchronize()
    gx, gw, gb = nhwc_to_nchw(to_np(dx)), to_np(dw), to_np(db)
    xq, wq, bq = x.astype(np.float32).astype(np.float64), wt.astype(np.float32).astype(np.float64), \
        b.astype(np.float32).astype(np.float64)

    def L(xx, ww, bb):
        return sum(float((oracle.conv3x3(xx[i], ww, bb, stride=stride, leaky=leaky) * U[i]).sum()) for i in range(n))

    # directions on the scale of each operand, so a step moves every pre-activation by ~h
    hstep = 1e-7
    for k in range(3):
        Vx, Vw, Vb = g.normal(size=x.shape), g.normal(size=wt.shape) / np.sqrt(9 * cin), g.normal(size=b.shape)
        fd = (L(xq + hstep * Vx, wq + hstep * Vw, bq + hstep * Vb) - L(xq - hstep * Vx, wq - hstep * Vw,
                                                                        bq - hstep * Vb)) / (2 * hstep)
        an = float((gx * Vx).sum() + (gw * Vw).sum() + (gb * Vb).sum())
        assert _rel(an, fd) <= 1e-4, (k, an, fd)
    # each part on its own
    Vx = g.normal(size=x.shape)
    fd = (L(xq + hstep * Vx, wq, bq) - L(xq - hstep * Vx, wq, bq)) / (2 * hstep)
    assert _rel(float((gx * Vx).sum()), fd) <= 1e-4


@pytest.mark.parametrize("n,h,w,c,r", [(2, 9, 11, 8, 2), (1, 14, 12, 32, 4), (1, 6, 7, 4, 3)])
def test_correlation_backward_matches_oracle_finite_differences(n, h, w, c, r):
    import torch
    g = synth.rng(51)
    f1, f2 = g.normal(size=(n, c, h, w)), g.normal(size=(n, c, h, w))
    D = (2 * r + 1) ** 2
    U = g.normal(size=(n, D, h, w))
    d1, d2 = to_dev(nchw_to_nhwc(f1.astype(np.float32))), to_dev(nchw_to_nhwc(f2.astype(np.float32)))
    cost = tc.op_correlation(d1, d2, r)
    dcost = to_dev(nchw_to_nhwc(U.astype(np.float32)))
    g1, g2 = torch.empty_like(d1), torch.empty_like(d2)
    tr = _train()
    tc._check(tr._lib.tc_op_correlation_backward(d1.data_ptr(), d2.data_ptr(), n, h, w, c, r, cost.data_ptr(),
                                                 dcost.data_ptr(), g1.data_ptr(), g2.data_ptr(), None))
    g1, g2 = nhwc_to_nchw(to_np(g1)), nhwc_to_nchw(to_np(g2))
    a1, a2 = f1.astype(np.float32).astype(np.float64), f2.astype(np.float32).astype(np.float64)

    def L(x1, x2):
        return sum(float((oracle.correlation(x1[i], x2[i], r) * U[i]).sum()) for i in range(n))

    for k in range(3):
        V1, V2 = g.normal(size=f1.shape), g.normal(size=f2.shape)
        hs = 1e-6
        fd = (L(a1 + hs * V1, a2 + hs * V2) - L(a1 - hs * V1, a2 - hs * V2)) / (2 * hs)
        an = float((g1 * V1).sum() + (g2 * V2).sum())
        assert _rel(an, fd) <= 1e-4, (k, an, fd)


@pytest.mark.parametrize("n,h,w,c,mag", [(2, 9, 12, 8, 3.0), (1, 16, 14, 32, 6.0)])
def test_warp_backward_matches_oracle_finite_differences(n, h, w, c, mag):
    import torch
    g = synth.rng(52)
    f = g.normal(size=(n, c, h, w))
    # integer part anywhere in [-mag, mag], fractional part inside (0.1, 0.9): no cell edge
    # within the difference step
    flow = np.floor(g.uniform(-mag, mag, (n, 2, h, w))) + g.uniform(0.1, 0.9, (n, 2, h, w))
    U = g.normal(size=(n, c, h, w))
    fd_, fl_ = to_dev(nchw_to_nhwc(f.astype(np.float32))), to_dev(np.moveaxis(flow, 1, -1).astype(np.float32))
    dout = to_dev(nchw_to_nhwc(U.astype(np.float32)))
    gf, gfl = torch.empty_like(fd_), torch.empty_like(fl_)
    tr = _train()
    tc._check(tr._lib.tc_op_warp_features_backward(fd_.data_ptr(), fl_.data_ptr(), n, h, w, c, dout.data_ptr(),
                                                   gf.data_ptr(), gfl.data_ptr(), None))
    gf, gfl = nhwc_to_nchw(to_np(gf)), np.moveaxis(to_np(gfl), -1, 1)
    a, fl = f.astype(np.float32).astype(np.float64), flow.astype(np.float32).astype(np.float64)

    def L(ff, ffl):
        return sum(float((oracle.warp(ff[i], ffl[i], True)[0] * U[i]).sum()) for i in range(n))

    for k in range(3):
        Vf, Vl = g.normal(size=f.shape), g.normal(size=flow.shape)
        hs = 1e-6
        fd = (L(a + hs * Vf, fl + hs * Vl) - L(a - hs * Vf, fl - hs * Vl)) / (2 * hs)
        an = float((gf * Vf).sum() + (gfl * Vl).sum())
        assert _rel(an, fd) <= 1e-4, (k, an, fd)


@pytest.mark.parametrize("n,h,w,s", [(2, 5, 7, 2), (1, 8, 6, 4)])
def test_upsample_backward_is_the_adjoint(n, h, w, s):
    """Upsampling is linear: <up(x), U> = <x, up^T(U)> exactly up to float32 rounding, with
    up evaluated by the oracle."""
    import torch
    g = synth.rng(53)
    x = g.normal(size=(n, 2, h, w))
    U = g.normal(size=(n, 2, h * s, w * s))
    dfine = to_dev(np.moveaxis(U, 1, -1).astype(np.float32))
    dc = torch.empty((n, h, w, 2), device="cuda")
    tr = _train()
    tc._check(tr._lib.tc_op_upsample_flow_backward(dfine.data_ptr(), n, h, w, s, dc.data_ptr(), None))
    torch.cuda.synchronize()
    gx = np.moveaxis(to_np(dc), -1, 1)
    lhs = sum(float((oracle.upsample_flow(x[i], s) * U[i]).sum()) for i in range(n))
    rhs = float((gx * x).sum())
    assert _rel(lhs, rhs) <= 1e-5


def test_autograd_functions_chain():
    """The autograd wrappers compose: d/dx of sum(conv(warp(x, flow))) through torch's
    engine equals the chained stage backward passes (both on the GPU)."""
    import torch
    tr = _train()
    g = synth.rng(54)
    x = to_dev(g.normal(size=(1, 10, 12, 8))).requires_grad_(True)
    flow = to_dev(np.floor(g.uniform(-2, 2, (1, 10, 12, 2))) + 0.5).requires_grad_(True)
    w = torch.tensor(g.normal(size=(16, 8, 3, 3)) / 8, dtype=torch.float32, requires_grad=True)
    b = torch.zeros(16, requires_grad=True)
    y = tr.Conv3x3.apply(tr.WarpFeatures.apply(x, flow), w, b, 1, True)
    y.sum().backward()
    assert x.grad is not None and flow.grad is not None and w.grad is not None and b.grad is not None
    assert torch.isfinite(x.grad).all() and float(b.grad.abs().sum()) > 0


# ---------------------------------------------------------------------- the trainer

def _oracle_loss(net, Ia, Ib, gt):
    """Sum over estimator levels of the batch-mean EPE against the block-averaged truth."""
    B, _, H, W = Ia.shape
    total = 0.0
    for i in range(B):
        pa, pb = oracle.pyramid(net, Ia[i]), oracle.pyramid(net, Ib[i])
        _, lf = oracle.flow_from_pyramids(net, pa, pb, H, W, level_flows=True)
        for l in range(2, net.levels + 1):
            s = 1 << l
            gl = gt[i].reshape(2, H // s, s, W // s, s).mean((2, 4)) / s
            total += oracle.epe(lf[l - 2], gl) / B
    return total


def _perturbed(net, vec):
    out = oracle.Net(net.levels, net.radius, net.chans, net.decoder, [])
    off = 0
    for L in net.layers:
        nw, nb = L["w"].size, L["b"].size
        out.layers.append(dict(L, w=L["w"] + vec[off:off + nw].reshape(L["w"].shape),
                               b=L["b"] + vec[off + nw:off + nw + nb]))
        off += nw + nb
    return out


def _batch(B, size, seed, max_flow):
    a, b, f = synth.training_batch(seed, B, size=size, max_flow=max_flow)
    return a, b, f


def test_trainer_forward_and_gradient_match_oracle():
    tr = _train()
    chans, radius = (16, 32, 48), 3
    path, net = weights_file(chans, radius)
    B, S = 2, 64
    a, b, f = _batch(B, S, 100, 4.0)
    t = tr.Trainer(B, S, S, "fp32", weights_path=path)
    loss = t.run(to_dev(a), to_dev(b), to_dev(f), mode="backward", wait=True)
    want = _oracle_loss(net, a.astype(np.float64), b.astype(np.float64), f.astype(np.float64))
    assert _rel(loss, want) <= 1e-5, (loss, want)
    # level flows (a -> b) vs the oracle's
    for i in range(B):
        pa, pb = oracle.pyramid(net, a[i]), oracle.pyramid(net, b[i])
        _, lf = oracle.flow_from_pyramids(net, pa, pb, S, S, level_flows=True)
        for l in range(2, net.levels + 1):
            got = np.moveaxis(to_np(t.level_flow(l))[i], -1, 0)
            assert oracle.epe(got, lf[l - 2]) <= 1e-4
    grad = t.get_grads().astype(np.float64)
    p0 = t.get_params()
    assert grad.shape == p0.shape and np.isfinite(grad).all()
    g = synth.rng(55)
    hs = 1e-6
    for k in range(3):
        V = g.normal(size=grad.shape)
        V /= np.linalg.norm(V)
        fd = (_oracle_loss(_perturbed(net, hs * V), a, b, f) - _oracle_loss(_perturbed(net, -hs * V), a, b, f)) / (2 * hs)
        an = float(grad @ V)
        print(f"direction {k}: analytic {an:.6e}, finite difference {fd:.6e}")
        assert _rel(an, fd) <= 1e-3, (k, an, fd)
    t.destroy()


def test_bf16_trainer_tracks_fp32():
    tr = _train()
    path, net = weights_file((16, 32, 64, 96, 128), 4)
    B, S = 4, 128
    a, b, f = _batch(B, S, 200, 8.0)
    res = {}
    for prec in ("fp32", "bf16"):
        t = tr.Trainer(B, S, S, prec, weights_path=path)
        loss = t.run(to_dev(a), to_dev(b), to_dev(f), mode="backward", wait=True)
        res[prec] = (loss, t.get_grads().astype(np.float64))
        t.destroy()
    (l32, g32), (l16, g16) = res["fp32"], res["bf16"]
    cos = float(g32 @ g16 / (np.linalg.norm(g32) * np.linalg.norm(g16)))
    print(f"loss fp32 {l32:.5f} bf16 {l16:.5f}; gradient cosine {cos:.5f}")
    # bfloat16 activations: ~2^-9 relative per layer, ~2 u sqrt(n) on the loss (n = 35)
    assert _rel(l32, l16) <= 2 * 2.0 ** -9 * np.sqrt(35)
    assert cos >= 0.99


def test_training_reduces_the_loss_and_checkpoints_resume():
    import torch
    tr = _train()
    chans, radius = (16, 32, 48), 3
    path, net = weights_file(chans, radius)
    B, S = 8, 64
    batches = [tuple(to_dev(x) for x in _batch(B, S, 1000 + 10 * k, 4.0)) for k in range(8)]
    t = tr.Trainer(B, S, S, "fp32", weights_path=path, lr=1e-3)
    first = np.mean([t.run(*bt, mode="forward", wait=True) for bt in batches])
    for it in range(150):
        t.run(*batches[it % len(batches)], mode="step")
    after = np.mean([t.run(*bt, mode="forward", wait=True) for bt in batches])
    print(f"loss over the 8 training batches: {first:.4f} -> {after:.4f} after 150 steps")
    assert t.steps == 150
    assert after < 0.7 * first
    d = tempfile.mkdtemp(prefix="tck")
    ck = os.path.join(d, "ck.bin")
    t.save(ck)
    t2 = tr.Trainer(B, S, S, "fp32", weights_path=path, lr=1e-3)
    t2.load(ck)
    assert t2.steps == 150 and np.array_equal(t2.get_params(), t.get_params())
    t.run(*batches[0], mode="step")
    t2.run(*batches[0], mode="step")
    p1, p2 = t.get_params(), t2.get_params()
    # same state, same batch: the same update up to the order of float atomics
    assert np.abs(p1 - p2).max() <= 1e-6 * max(1.0, np.abs(p1).max())
    # exported weights drive an inference stream: its level-2 flow, upsampled, is the
    # stream's full-resolution flow
    wpath = os.path.join(d, "trained.tcw")
    t.export_weights(wpath)
    s = tc.Stream(S, S, "fp32", weights_path=wpath)
    Ia, Ib, _ = batches[0]
    O = torch.empty((3, S, S), device="cuda")
    s.process_frame(Ib[0].contiguous(), Ib[0].contiguous(), O)
    s.process_frame(Ia[0].contiguous(), Ia[0].contiguous(), O)
    Fb = torch.empty((2, S, S), device="cuda")
    s.get_flows(Fb, None)                     # F_{t -> t-1} = F_{a -> b}
    t.run(*batches[0], mode="forward", wait=True)
    lf2 = t.level_flow(2)[0:1].contiguous()
    up = tc.op_upsample_flow(lf2, 4)[0]
    torch.cuda.synchronize()
    # same layers, different float32 summation orders (the stream permutes x0's channels)
    assert oracle.epe(to_np(Fb), np.moveaxis(to_np(up), -1, 0)) <= 1e-3
    s.destroy()
    t.destroy()
    t2.destroy()


def test_bruteforce_flow_matches_oracle_exactly():
    """8-bit images: every SSD is exact in float32 and in FP64, so the argmin (with the
    same tie rule) must be the same index on both sides."""
    import torch
    tr = _train()
    g = synth.rng(56)
    for (c, h, w, r) in [(3, 24, 31, 3), (1, 17, 20, 2), (3, 40, 40, 4)]:
        a = np.round(g.random((c, h, w)) * 255) / 256
        b = np.roll(a, (1, -2), axis=(1, 2)) if c == 3 else np.round(g.random((c, h, w)) * 255) / 256
        got = to_np(tr.bruteforce_flow(to_dev(a), to_dev(b), r))
        want = oracle.bruteforce_flow(a, b, r)
        assert np.array_equal(got, want), (c, h, w, r)


def test_trained_network_against_brute_force_flow():
    """The yardsticks: on held-out pairs the network's EPE before and after training is set
    beside the brute-force integer flow's (radius 16, which covers the |F| <= 16 px of these
    128x128 pairs) and the zero flow's.  Training on 512 pairs must lower the held-out EPE
    and beat the zero flow."""
    import torch
    tr = _train()
    chans, radius = (16, 32, 48), 3
    path, net = weights_file(chans, radius)
    B, S, R = 8, 128, 16
    train_b = [tuple(to_dev(x) for x in _batch(B, S, 5000 + 10 * k, 16.0)) for k in range(64)]
    a, b, f = _batch(B, S, 90000, 16.0)
    t = tr.Trainer(B, S, S, "fp32", weights_path=path, lr=5e-4)

    def held_out_epe():
        t.run(to_dev(a), to_dev(b), to_dev(f), mode="forward", wait=True)
        lf2 = t.level_flow(2)
        out = []
        for i in range(B):
            full = np.moveaxis(to_np(tc.op_upsample_flow(lf2[i:i + 1].contiguous(), 4)[0]), -1, 0)
            out.append(oracle.epe(full, f[i]))
        return float(np.mean(out))

    before = held_out_epe()
    for it in range(1000):
        t.run(*train_b[it % len(train_b)], mode="step")
    after = held_out_epe()
    bf_epe, zero_epe = [], []
    for i in range(B):
        k = tr.bruteforce_flow(to_dev(a[i]), to_dev(b[i]), R)
        bf_epe.append(oracle.epe(to_np(tr.index_to_flow(k, R)), f[i]))
        zero_epe.append(oracle.epe(np.zeros_like(f[i]), f[i]))
    print(f"held-out EPE: network {before:.3f} px untrained -> {after:.3f} px after 1000 steps; "
          f"brute force {np.mean(bf_epe):.3f} px, zero flow {np.mean(zero_epe):.3f} px")
    assert after < before and after < np.mean(zero_epe)
    t.destroy()
