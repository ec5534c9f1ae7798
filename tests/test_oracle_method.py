"""Pins of the oracle's composite steps: the flow network's coarse-to-fine chain (Sec. 3.2)
and the consistency step (Sec. 3.1, Eqs. 2-7), against closed forms, endpoints and
invariants.  CPU only."""
import json
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _net(chans=(16, 32, 48), radius=3, seed=0, **kw):
    spec = synth.NetSpec(chans=chans, radius=radius)
    layers = synth.he_weights(spec, seed=seed, **kw)
    return spec, oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)


def test_paper_parameter_presets_match_golden():
    g = json.load(open(os.path.join(GOLDEN, "paper_params.json")))
    f = g["final"]
    assert oracle.PAPER_FINAL == dict(k1=f["k1"], k2=f["k2"], alpha=f["alpha"], lam=f["lambda"])
    o = g["objective"]
    assert oracle.PAPER_OBJECTIVE == dict(k1=o["k1"], k2=o["k2"], alpha=o["alpha"], lam=o["lambda"])


# ------------------------------------------------------------------------ network chain

def test_pyramid_shapes_and_first_level_matches_torch():
    spec, net = _net()
    img = synth.rng(1).random((3, 64, 64))
    feats = oracle.pyramid(net, img)
    assert [f.shape for f in feats] == [(16, 32, 32), (32, 16, 16), (48, 8, 8)]
    L = net.layers
    x = torch.from_numpy(img)[None]
    for j in range(3):
        x = Fnn.leaky_relu(Fnn.conv2d(x, torch.from_numpy(L[j]["w"]), torch.from_numpy(L[j]["b"]),
                                      stride=2 if j == 0 else 1, padding=1), 0.1)
    np.testing.assert_allclose(feats[0], x[0].numpy(), rtol=0, atol=1e-12)


def test_zero_estimators_give_zero_flow():
    spec, net = _net()
    for L in net.layers[3 * net.levels:]:
        L["w"][:] = 0
        L["b"][:] = 0
    d = synth.pair64()
    fab, fba = oracle.flow_pair(net, d["I1"], d["I0"])
    assert not fab.any() and not fba.any()


@pytest.mark.parametrize("levels_chans", [(16, 32, 48), (16, 32, 64, 96, 128)])
def test_head_bias_only_closed_form(levels_chans):
    """With every estimator weight zero and head bias b, flow^L = b and
    flow^l = 2 flow^{l+1} + b, so the output is 4 (2^{L-1} - 1) b everywhere."""
    spec, net = _net(chans=levels_chans, radius=2)
    b = np.array([0.25, -0.125])
    for i, L in enumerate(net.layers[3 * net.levels:]):
        L["w"][:] = 0
        L["b"][:] = 0
        if i % 5 == 4:
            L["b"][:] = b
    h = w = 1 << (net.levels + 1)
    img = synth.rng(2).random((3, h, w))
    f = oracle.flow_from_pyramids(net, oracle.pyramid(net, img), oracle.pyramid(net, img), h, w)
    want = 4 * (2 ** (net.levels - 1) - 1) * b
    np.testing.assert_array_equal(f[0], want[0])
    np.testing.assert_array_equal(f[1], want[1])


def _torch_flow(net, fs, fo, h, w):
    """Independent composition of the coarse-to-fine chain from torch library routines
    (conv2d, grid_sample with zero padding, interpolate), with the correlation written as
    unfold of the shifted map."""
    r = net.radius
    n = 2 * r + 1
    E = net.layers[3 * net.levels:]
    prev = None
    for l in range(net.levels, 1, -1):
        s = torch.from_numpy(fs[l - 1])[None]
        o = torch.from_numpy(fo[l - 1])[None]
        c, lh, lw = fs[l - 1].shape
        if prev is None:
            up = torch.zeros(1, 2, lh, lw, dtype=torch.float64)
            o2 = o
        else:
            up = Fnn.interpolate(prev, scale_factor=2, mode="bilinear", align_corners=False) * 2
            yy, xx = torch.meshgrid(torch.arange(lh, dtype=torch.float64),
                                    torch.arange(lw, dtype=torch.float64), indexing="ij")
            gx = 2 * (xx + up[0, 0]) / (lw - 1) - 1
            gy = 2 * (yy + up[0, 1]) / (lh - 1) - 1
            o2 = Fnn.grid_sample(o, torch.stack([gx, gy], -1)[None], mode="bilinear",
                                 padding_mode="zeros", align_corners=True)
        patches = Fnn.unfold(o2, n, padding=r).view(1, c, n * n, lh, lw)
        cv = Fnn.leaky_relu((s[:, :, None] * patches).sum(1) / c, 0.1)
        x0 = torch.cat([cv, s, up], 1)
        conv = lambda x, L, act: (lambda y: Fnn.leaky_relu(y, 0.1) if act else y)(
            Fnn.conv2d(x, torch.from_numpy(L["w"]), torch.from_numpy(L["b"]), padding=1))
        e = E[5 * (net.levels - l):]
        x1 = conv(x0, e[0], 1); x2 = conv(x1, e[1], 1); x3 = conv(x2, e[2], 1)
        x4 = conv(torch.cat([x3, x2], 1), e[3], 1)
        res = conv(torch.cat([x4, x3], 1), e[4], 0)
        prev = up + res
    return (Fnn.interpolate(prev, scale_factor=4, mode="bilinear", align_corners=False) * 4)[0].numpy()


@pytest.mark.parametrize("chans,radius,h,w", [((16, 32, 48), 3, 64, 64), ((8, 12, 16, 20, 24), 4, 64, 96)])
def test_flow_matches_library_composition(chans, radius, h, w):
    spec, net = _net(chans=chans, radius=radius, seed=5)
    g = synth.rng(6)
    a, b = g.random((3, h, w)), g.random((3, h, w))
    pa, pb = oracle.pyramid(net, a), oracle.pyramid(net, b)
    got = oracle.flow_from_pyramids(net, pa, pb, h, w)
    ref = _torch_flow(net, pa, pb, h, w)
    assert np.abs(got).max() > 0.1
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)


# ------------------------------------------------------------------------ consistency step

def _frames(h=24, w=28, seed=0):
    g = synth.rng(seed)
    return [g.random((3, h, w)) for _ in range(5)]


def test_k1_zero_returns_processed_frame_exactly():
    It, Pt, Ip, Pp, Op = _frames()
    Fb = synth.rng(1).uniform(-3, 3, (2, 24, 28))
    r = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, -Fb, k1=0.0)
    assert np.array_equal(r["O"], Pt)
    assert (r["wp"] == 0).all() and (r["wc"] == 2.0).all()


def test_zero_flows_give_all_valid_mask():
    It, Pt, Ip, Pp, Op = _frames()
    z = np.zeros((2, 24, 28))
    r = oracle.consistency(It, Pt, Ip, Pp, Op, z, z)
    assert r["mask"].all()


def test_static_scene_weight_is_k1():
    It, Pt, _, Pp, Op = _frames()
    z = np.zeros((2, 24, 28))
    r = oracle.consistency(It, Pt, It, Pp, Op, z, z, k1=0.37)
    assert (r["wp"] == 0.37).all()


def test_constant_content_is_preserved():
    """A is a convex combination of P_t, Gamma P_{t-1}, Gamma O_{t-1} (Eqs. 2, 5)."""
    It, _, Ip, _, _ = _frames()
    c = np.full((3, 24, 28), 0.625)
    Fb = synth.rng(2).uniform(-4, 4, (2, 24, 28))
    Ff = synth.rng(3).uniform(-4, 4, (2, 24, 28))
    r = oracle.consistency(It, c, Ip, c, c, Fb, Ff, k1=0.9, alpha=3.0)
    np.testing.assert_allclose(r["O"], c, rtol=0, atol=1e-15)
    assert 0 < r["mask"].mean() < 1


@pytest.mark.parametrize("du,dv", [(2, -1), (-1, 3)])
def test_full_weight_returns_warped_previous_output(du, dv):
    """k1 = 1 and I_{t-1} moved consistently with an integer flow: w_p = 1 in bounds, so
    O_t = Gamma(O_{t-1}) (Eq. 4/5) and A^I = Gamma I_{t-1} = I_t, hence w_c = lambda (Eq. 7)."""
    h, w = 20, 22
    g = synth.rng(4)
    big = g.random((3, h + 8, w + 8))
    It = big[:, 4:4 + h, 4:4 + w]
    Ip = big[:, 4 - dv:4 - dv + h, 4 - du:4 - du + w]          # Ip(x + F) = It(x)
    Pt, Pp, Op = g.random((3, h, w)), g.random((3, h, w)), g.random((3, h, w))
    Fb = np.stack([np.full((h, w), float(du)), np.full((h, w), float(dv))])
    r = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, -Fb, k1=1.0, lam=2.0)
    ys, xs = slice(max(0, -dv), min(h, h - dv)), slice(max(0, -du), min(w, w - du))
    ysrc, xsrc = slice(ys.start + dv, ys.stop + dv), slice(xs.start + du, xs.stop + du)
    assert r["mask"][ys, xs].all()
    assert np.array_equal(r["O"][:, ys, xs], Op[:, ysrc, xsrc])
    assert (r["wc"][ys, xs] == 2.0).all()
    out = r["mask"] == 0
    assert out.any() and np.array_equal(r["O"][:, out], Pt[:, out])


def test_fb_test_consistent_and_inconsistent_flows():
    It, Pt, Ip, Pp, Op = _frames()
    h, w = 24, 28
    Fb = np.stack([np.full((h, w), 3.0), np.full((h, w), -2.0)])
    r = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, -Fb)
    _, inb = oracle.warp(It, Fb, 0)
    assert np.array_equal(r["mask"], inb)
    big = np.stack([np.full((h, w), 8.0), np.full((h, w), 0.0)])
    r2 = oracle.consistency(It, Pt, Ip, Pp, Op, big, big)
    assert not r2["mask"].any()
    r3 = oracle.consistency(It, Pt, Ip, Pp, Op, big, big, fb_check=False)
    assert np.array_equal(r3["mask"], oracle.warp(It, big, 0)[1])


def test_wc_closed_form_through_warped_input():
    """I_t - A^I_t = w_p (I_t - Gamma I_{t-1}) (Eq. 6), so w_c = lambda exp(-alpha w_p^2 d_p)
    where exp(-alpha d_p) = w_p whenever w_p < k1 and the mask is set."""
    It, Pt, Ip, Pp, Op = _frames()
    Ip = It + 0.004 * synth.rng(5).normal(size=It.shape)
    z = np.zeros((2, 24, 28))
    r = oracle.consistency(It, Pt, Ip, Pp, Op, z, z, k1=0.99, alpha=2000.0, lam=1.5)
    wp = r["wp"]
    sel = (wp < 0.99) & (wp > 1e-6)
    assert sel.sum() > 50
    d = -np.log(wp[sel]) / 2000.0
    np.testing.assert_allclose(r["wc"][sel], 1.5 * np.exp(-2000.0 * wp[sel] ** 2 * d), rtol=1e-10)


def test_stream_first_frame_is_processed_frame():
    spec, net = _net()
    d = synth.pair64()
    s = oracle.Stream(net, k1=0.5)
    r0 = s.step(d["I0"], d["P0"])
    assert np.array_equal(r0["O"], d["P0"].astype(np.float64))
    r1 = s.step(d["I1"], d["P1"])
    assert r1["O"].shape == (3, 64, 64) and r1["Fb"].shape == (2, 64, 64)


def test_generator_flow_is_ground_truth():
    """The rendered sequence moves along its analytic flows: bilinear warping frame t-1 by the
    backward flow reproduces frame t away from square edges (cubic vs bilinear resampling
    differ by the interpolation error only)."""
    seq = synth.Sequence(width=160, height=96, seed=3, side_range=(20, 30), max_vel=4.0)
    f0, f1 = seq.frame(0), seq.frame(1)
    Fb, Ff = seq.flow_backward(1), seq.flow_forward(1)
    wI, inb = oracle.warp(f0, Fb, 0)
    err = np.abs(wI - f1).max(0)
    r = oracle.consistency(f1, f1, f0, f0, f0, Fb, Ff, k1=1.0, alpha=0.0)
    ok = (r["mask"] == 1) & (inb == 1)
    assert ok.mean() > 0.8
    assert np.median(err[ok]) < 0.02


def test_photometric_weight_uses_squared_norm_over_channels():
    """||x||^2 of a colour difference in one channel only is that difference squared (Eq. 3):
    zero flow, I_t = I_{t-1} + delta in the red channel -> w_p = exp(-alpha delta^2)."""
    It, Pt, _, Pp, Op = _frames()
    Ip = It.copy()
    Ip[0] -= 0.01
    z = np.zeros((2, 24, 28))
    r = oracle.consistency(It, Pt, Ip, Pp, Op, z, z, k1=1.0, alpha=6500.0)
    np.testing.assert_allclose(r["wp"], np.exp(-6500.0 * 1e-4), rtol=1e-12)


def test_blend_decomposes_into_eq2_and_eq5_weights():
    """A = w_p G + (1 - w_p) L, L = (1 - w_p) P_t + w_p Gamma P_{t-1}: with one of
    P_t, P_{t-1}, O_{t-1} set to one and the others zero (zero flow), O equals (1 - w_p)^2,
    w_p (1 - w_p) and w_p respectively."""
    It, _, _, _, _ = _frames()
    Ip = It + 0.005 * synth.rng(7).normal(size=It.shape)
    z = np.zeros((2, 24, 28))
    one, zero = np.ones((3, 24, 28)), np.zeros((3, 24, 28))
    kw = dict(k1=0.8, alpha=1500.0)
    wp = oracle.consistency(It, zero, Ip, zero, one, z, z, **kw)["O"]
    np.testing.assert_allclose(oracle.consistency(It, one, Ip, zero, zero, z, z, **kw)["O"], (1 - wp) ** 2, atol=1e-15)
    np.testing.assert_allclose(oracle.consistency(It, zero, Ip, one, zero, z, z, **kw)["O"], wp * (1 - wp), atol=1e-15)
    assert 0.05 < wp.mean() < 0.8


@pytest.mark.parametrize("fb_u,ff_cols,ff_u,want_valid", [
    # integer F_b = (+2, 0): F_f~(x) = F_f(x + 2); F_f = -2 on columns 3..5, so exactly the
    # columns x with x + 2 in 3..5 pass the test (|F_b + F_f~|^2 = 0); elsewhere
    # |2 + 0|^2 = 4 > 0.01 * 4 + 0.5.  Sampling F_f at x would give 3..5, at x - 2 5..7.
    (2.0, (3, 4, 5), -2.0, (1, 2, 3)),
    # fractional F_b = (+1.5, 0): F_f~(x) = (F_f(x + 1) + F_f(x + 2)) / 2; F_f = -1.5 on
    # columns 4..6: x = 3, 4 see -1.5 (lhs 0, valid); x = 2, 5 see -0.75 (lhs 0.5625 >
    # 0.01 * (2.25 + 0.5625) + 0.5 = 0.528, occluded); the rest see 0 (lhs 2.25, occluded).
    (1.5, (4, 5, 6), -1.5, (3, 4)),
])
def test_fb_test_samples_forward_flow_at_backward_target(fb_u, ff_cols, ff_u, want_valid):
    """The forward-backward test reads F_f where F_b points (F_f~ = Gamma_{F_b}(F_f), C6),
    on a spatially varying F_f whose decision changes if it is read anywhere else; the mask
    is hand-computed (columns past W - 1 - u are out of bounds either way)."""
    h, w = 4, 10
    It, Pt, Ip, Pp, Op = [np.full((3, h, w), 0.5) for _ in range(5)]
    Fb = np.zeros((2, h, w))
    Fb[0] = fb_u
    Ff = np.zeros((2, h, w))
    Ff[0][:, list(ff_cols)] = ff_u
    r = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, Ff, k1=0.5)
    want = np.zeros((h, w), np.uint8)
    want[:, list(want_valid)] = 1
    assert np.array_equal(r["mask"], want), r["mask"][0]
