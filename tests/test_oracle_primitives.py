"""Pins of the oracle's primitives against things other than the oracle itself: library
routines on tiny inputs (FP64 torch conv2d / grid_sample / interpolate), closed forms and
invariants.  CPU only."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle
import synth


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64))


# ------------------------------------------------------------------------ conv (Sec. 3.2)

@pytest.mark.parametrize("cin,cout,h,w,stride,leaky", [
    (3, 5, 7, 9, 1, True), (4, 2, 8, 6, 2, True), (3, 4, 9, 7, 2, False), (6, 3, 5, 11, 1, False),
])
def test_conv_matches_torch(cin, cout, h, w, stride, leaky):
    g = synth.rng(3)
    x = g.normal(size=(cin, h, w))
    wt = g.normal(size=(cout, cin, 3, 3))
    b = g.normal(size=cout)
    ref = Fnn.conv2d(_t(x)[None], _t(wt), _t(b), stride=stride, padding=1)[0]
    if leaky:
        ref = Fnn.leaky_relu(ref, 0.1)
    got = oracle.conv3x3(x, wt, b, stride=stride, leaky=leaky)
    assert got.shape == tuple(ref.shape)
    np.testing.assert_allclose(got, ref.numpy(), rtol=0, atol=1e-12)


def test_conv_delta_kernel_is_identity():
    g = synth.rng(4)
    x = g.normal(size=(3, 6, 7))
    wt = np.zeros((3, 3, 3, 3))
    for c in range(3):
        wt[c, c, 1, 1] = 1.0
    assert np.array_equal(oracle.conv3x3(x, wt, None, 1, False), x)


# ------------------------------------------------------------------------ warp (Sec. 3.1, Gamma)

@pytest.mark.parametrize("zero", [0, 1])
def test_warp_zero_flow_is_identity(zero):
    x = synth.rng(5).random((3, 9, 13))
    out, inb = oracle.warp(x, np.zeros((2, 9, 13)), zero)
    assert np.array_equal(out, x) and inb.all()


@pytest.mark.parametrize("zero", [0, 1])
@pytest.mark.parametrize("du,dv", [(2, -1), (-3, 2), (0, 1)])
def test_warp_integer_shift_exact_on_interior(zero, du, dv):
    h, w = 12, 14
    x = synth.rng(6).random((2, h, w))
    flow = np.stack([np.full((h, w), float(du)), np.full((h, w), float(dv))])
    out, inb = oracle.warp(x, flow, zero)
    ys, xs = slice(max(0, -dv), min(h, h - dv)), slice(max(0, -du), min(w, w - du))
    ysrc, xsrc = slice(ys.start + dv, ys.stop + dv), slice(xs.start + du, xs.stop + du)
    assert np.array_equal(out[:, ys, xs], x[:, ysrc, xsrc])
    assert inb[ys, xs].all()
    assert inb.sum() == (ys.stop - ys.start) * (xs.stop - xs.start)


@pytest.mark.parametrize("zero,mode", [(0, "border"), (1, "zeros")])
def test_warp_matches_grid_sample(zero, mode):
    h, w = 16, 16
    g = synth.rng(7)
    x = g.random((3, h, w))
    flow = g.uniform(-6, 6, (2, h, w))
    out, inb = oracle.warp(x, flow, zero)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    sx, sy = xx + flow[0], yy + flow[1]
    grid = np.stack([2 * sx / (w - 1) - 1, 2 * sy / (h - 1) - 1], -1)[None]
    ref = Fnn.grid_sample(_t(x)[None], _t(grid), mode="bilinear", padding_mode=mode,
                          align_corners=True)[0].numpy()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)
    assert not inb.all() and inb.any()


# ------------------------------------------------------------------------ correlation (Sec. 3.2)

def _unit_features(c, h, w, seed):
    f = synth.rng(seed).normal(size=(c, h, w))
    return f / np.sqrt((f ** 2).sum(0, keepdims=True))


@pytest.mark.parametrize("du,dv", [(2, -1), (-3, 3), (0, 0), (1, 2)])
def test_correlation_argmax_finds_integer_shift(du, dv):
    r, c, h, w = 3, 32, 14, 15
    f1 = _unit_features(c, h + 8, w + 8, 8)
    f2 = np.roll(f1, (dv, du), axis=(1, 2))            # f2(x + d) = f1(x)
    cv = oracle.correlation(f1, f2, r)
    k = cv.argmax(0)
    want = (dv + r) * (2 * r + 1) + (du + r)
    assert (k[4:-4, 4:-4] == want).all()


def test_correlation_constant_features_mean_and_leaky():
    r, c, h, w = 2, 6, 7, 8
    a = 0.7
    cv = oracle.correlation(np.full((c, h, w), a), np.full((c, h, w), a), r)
    n = 2 * r + 1
    for k in range(n * n):
        dy, dx = k // n - r, k % n - r
        inside = np.zeros((h, w), bool)
        inside[max(0, -dy):min(h, h - dy), max(0, -dx):min(w, w - dx)] = True
        np.testing.assert_allclose(cv[k][inside], a * a, rtol=1e-15)
        assert (cv[k][~inside] == 0).all()
    neg = oracle.correlation(np.full((c, h, w), a), np.full((c, h, w), -a), r)
    np.testing.assert_allclose(neg[(n * n) // 2], -0.1 * a * a, rtol=1e-15)


def test_correlation_swap_symmetry():
    r, c, h, w = 2, 5, 9, 10
    g = synth.rng(9)
    f1, f2 = g.normal(size=(c, h, w)), g.normal(size=(c, h, w))
    a, b = oracle.correlation(f1, f2, r), oracle.correlation(f2, f1, r)
    n = 2 * r + 1
    for k in range(n * n):
        dy, dx = k // n - r, k % n - r
        kk = (-dy + r) * n + (-dx + r)
        for y in range(max(0, -dy), min(h, h - dy)):
            for x in range(max(0, -dx), min(w, w - dx)):
                assert abs(a[k, y, x] - b[kk, y + dy, x + dx]) < 1e-13


# ------------------------------------------------------------------------ flow upsampling

@pytest.mark.parametrize("s,h,w", [(2, 5, 7), (4, 3, 6), (2, 1, 4)])
def test_upsample_matches_interpolate(s, h, w):
    f = synth.rng(10).normal(size=(2, h, w))
    ref = Fnn.interpolate(_t(f)[None], scale_factor=s, mode="bilinear", align_corners=False)[0] * s
    np.testing.assert_allclose(oracle.upsample_flow(f, s), ref.numpy(), rtol=0, atol=1e-12)


def test_upsample_constant_flow_scales():
    f = np.stack([np.full((4, 5), 1.25), np.full((4, 5), -0.5)])
    up = oracle.upsample_flow(f, 2)
    assert (up[0] == 2.5).all() and (up[1] == -1.0).all()


def test_pad_replicate():
    x = synth.rng(11).random((3, 5, 6))
    p = oracle.pad_replicate(x, 8, 8)
    ref = np.pad(x, ((0, 0), (0, 3), (0, 2)), mode="edge")
    assert np.array_equal(p, ref)


# ------------------------------------------------------------------------ brute-force flow

@pytest.mark.parametrize("du,dv", [(2, -1), (-3, 0), (1, 3)])
def test_bruteforce_flow_finds_translation(du, dv):
    r = 3
    base = synth.blurred_noise(40, 40, 3, 1.0, synth.rng(12))
    a = base[:, 8:32, 8:32]
    b = base[:, 8 - dv:32 - dv, 8 - du:32 - du]      # b(x + d) = a(x)
    k = oracle.bruteforce_flow(a, b, r)
    want = (dv + r) * (2 * r + 1) + (du + r)
    assert (k[4:-4, 4:-4] == want).all()


def test_epe_definition():
    f = np.zeros((2, 3, 4))
    g = np.zeros((2, 3, 4))
    g[0] = 3.0
    g[1] = 4.0
    assert oracle.epe(f, g) == 5.0


@pytest.mark.parametrize("r", [1, 2, 3])
def test_bruteforce_tie_rule_smallest_norm_then_smallest_index(r):
    """C12: a's vertical stripes are b's shifted by one column, so every odd horizontal
    displacement (and any vertical one) gives SSD 0 in the interior.  The smallest |d| among
    them is 1, at d = (-1, 0) and (+1, 0); the smaller index k = (dy + r)(2r + 1) + (dx + r)
    wins, i.e. d = (-1, 0).  A rule by index alone, by the largest index, or by |d| then the
    largest index each gives another k."""
    h, w = 16, 18
    cols = np.arange(w) % 2
    b = np.broadcast_to(cols.astype(np.float64), (3, h, w)).copy()
    a = 1.0 - b
    k = oracle.bruteforce_flow(a, b, r)
    want = r * (2 * r + 1) + (r - 1)
    assert (k[r + 1:-(r + 1), r + 1:-(r + 1)] == want).all()
    # flat images: every displacement ties at SSD 0 and the zero displacement wins
    flat = np.full((1, h, w), 0.3)
    assert (oracle.bruteforce_flow(flat, flat, r) == r * (2 * r + 1) + r).all()
