"""Stage-by-stage parity of the CUDA kernels against the FP64 oracle, through the C ABI.

Inputs are seeded (synth); expected values come from the oracle only.  Tolerances follow
from float32 arithmetic: a sum of K products of O(1) terms carries an error of about
K * 2^-24 relative to the sum of magnitudes, so conv outputs (K <= 9 * 211) are held to
2e-5 of the output scale, the correlation (a mean over <= 128 channels) to 1e-5, the
bilinear warps (4 taps) to 2e-6.  BF16 / FP16 operands are rounded on the host first, so
both sides see the same values; BF16 outputs are rounded to 8 significant bits (2^-9
relative), FP16 outputs to 11 (2^-11).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import REL16, nchw_to_nhwc, nhwc_to_nchw, planar_to_hw2, round16, to_dev, to_np

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


@pytest.mark.parametrize("n,h,w,s", [(2, 5, 7, 2), (1, 3, 9, 4), (2, 68, 120, 2), (1, 272, 480, 4)])
def test_upsample_flow(n, h, w, s):
    f = synth.rng(20).normal(0, 3, (n, 2, h, w))
    got = to_np(tc.op_upsample_flow(to_dev(np.moveaxis(f, 1, -1)), s))
    for i in range(n):
        ref = oracle.upsample_flow(f[i].astype(np.float32), s)
        np.testing.assert_allclose(np.moveaxis(got[i], -1, 0), ref, rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,h,w,c,mag", [(2, 17, 23, 8, 3.0), (1, 34, 60, 128, 6.0), (2, 136, 240, 64, 2.0)])
def test_warp_features(prec, n, h, w, c, mag):
    g = synth.rng(21)
    f = round16(prec, g.normal(size=(n, c, h, w)).astype(np.float32))
    flow = g.uniform(-mag, mag, (n, 2, h, w)).astype(np.float32)
    got = to_np(tc.op_warp_features(to_dev(nchw_to_nhwc(f)), to_dev(np.moveaxis(flow, 1, -1)), precision=prec))
    tol = 2e-6 if prec == "fp32" else REL16[prec]
    for i in range(n):
        ref, _ = oracle.warp(f[i], flow[i], 1)
        np.testing.assert_allclose(nhwc_to_nchw(got[i:i + 1])[0], ref, rtol=tol, atol=tol * 4)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,h,w,c,r", [(2, 19, 21, 32, 4), (1, 34, 60, 128, 4), (2, 8, 8, 48, 3), (2, 33, 47, 16, 2),
                                       (1, 21, 37, 24, 1), (3, 68, 120, 96, 4), (2, 136, 240, 64, 4)])
def test_correlation(prec, n, h, w, c, r):
    g = synth.rng(22)
    f1 = round16(prec, g.normal(size=(n, c, h, w)).astype(np.float32))
    f2 = round16(prec, g.normal(size=(n, c, h, w)).astype(np.float32))
    got = to_np(tc.op_correlation(to_dev(nchw_to_nhwc(f1)), to_dev(nchw_to_nhwc(f2)), r, precision=prec))
    # BF16 / FP16 cost volumes with c a multiple of 8 up to 128 run on the tensor cores
    # (banded GEMM)
    assert tc.op_last_used_tensor_cores() == (prec != "fp32" and c % 8 == 0 and c <= 128)
    for i in range(n):
        ref = oracle.correlation(f1[i], f2[i], r)
        g_ = nhwc_to_nchw(got[i:i + 1])[0]
        if prec == "fp32":
            np.testing.assert_allclose(g_, ref, rtol=1e-5, atol=1e-5)
        else:
            np.testing.assert_allclose(g_, ref, rtol=REL16[prec], atol=1e-4)


def test_correlation_finds_integer_shift():
    """Unit-norm features shifted by an integer displacement: argmax over the cost volume
    is the shift (bit-exact index), as for the oracle."""
    g = synth.rng(23)
    f1 = g.normal(size=(32, 40, 44))
    f1 /= np.sqrt((f1 ** 2).sum(0, keepdims=True))
    du, dv, r = 3, -2, 4
    f2 = np.roll(f1, (dv, du), axis=(1, 2))
    got = to_np(tc.op_correlation(to_dev(nchw_to_nhwc(f1[None])), to_dev(nchw_to_nhwc(f2[None])), r))[0]
    k = got.argmax(-1)
    assert (k[5:-5, 5:-5] == (dv + r) * 9 + (du + r)).all()
    ref = oracle.correlation(f1.astype(np.float32), f2.astype(np.float32), r).argmax(0)
    assert np.array_equal(k[5:-5, 5:-5], ref[5:-5, 5:-5])


CONV_CASES = [
    # n, h, w, cin, cout, stride   (bf16 cases with cin % 8 == 0 and cout % 16 == 0 run on
    # the tensor cores: several 128-pixel tiles, ragged row tails, channel tails, stride 2)
    (1, 9, 13, 16, 16, 1), (2, 17, 30, 32, 32, 2), (2, 34, 60, 128, 128, 1), (1, 33, 47, 120, 128, 1),
    (2, 20, 36, 160, 32, 1), (1, 68, 120, 96, 64, 1), (1, 11, 7, 8, 2, 1), (2, 64, 72, 64, 96, 2),
    (1, 5, 6, 6, 10, 1), (1, 136, 240, 64, 64, 1), (2, 272, 480, 32, 32, 1), (1, 7, 300, 16, 16, 2),
    (2, 3, 130, 216, 128, 1), (1, 8, 8, 48, 48, 1),
    # wide rows: two tiles with a ragged second one, a one-pixel last tile, three K steps
    (1, 20, 300, 128, 128, 1), (2, 9, 480, 120, 96, 1), (1, 6, 257, 64, 128, 1), (1, 3, 192, 192, 128, 1),
    # one K step and <= 32 outputs: row tails of 3 and 1, a one-pixel last tile, a
    # 24-channel input, three images
    (2, 23, 200, 64, 32, 1), (1, 1, 129, 16, 16, 1), (3, 17, 128, 24, 16, 1),
    # a single 120-pixel tile per row over 50 rows and two images, two K steps, 96 outputs
    (2, 50, 120, 128, 96, 1),
    # enough tiles for the persistent stride-1 kernel to take several rows per tile: 2 rows
    # of 128 outputs with streamed weights (odd row count: a one-row last group), rows of 64
    # outputs behind a 32-channel tail step, rows of 32 outputs over three K steps
    (1, 299, 130, 120, 128, 1), (2, 150, 260, 96, 64, 1), (2, 300, 130, 160, 32, 1),
    # rows of exactly one and two 126-pixel tiles of that kernel
    (1, 5, 126, 64, 64, 1), (2, 4, 252, 128, 128, 1),
]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("n,h,w,cin,cout,stride", CONV_CASES)
def test_conv3x3(prec, n, h, w, cin, cout, stride):
    g = synth.rng(24)
    x = g.normal(size=(n, cin, h, w)).astype(np.float32)
    wt = (g.normal(size=(cout, cin, 3, 3)) / np.sqrt(9 * cin)).astype(np.float32)
    b = g.normal(0, 0.1, cout).astype(np.float32)
    x, wt = round16(prec, x), round16(prec, wt)
    got = to_np(tc.op_conv3x3(to_dev(nchw_to_nhwc(x)), wt, b, stride=stride, leaky=True, precision=prec))
    eligible = prec != "fp32" and cin % 8 == 0 and cout % 16 == 0 and cout <= 128
    assert tc.op_last_used_tensor_cores() == eligible
    for i in range(n):
        ref = oracle.conv3x3(x[i], wt, b, stride=stride, leaky=True)
        g_ = nhwc_to_nchw(got[i:i + 1])[0]
        scale = max(1.0, np.abs(ref).max())
        if prec == "fp32":
            np.testing.assert_allclose(g_, ref, rtol=0, atol=2e-5 * scale)
        else:
            # the output's own rounding (relative) plus float32 accumulation order
            np.testing.assert_allclose(g_, ref, rtol=REL16[prec], atol=(1e-3 if prec == "bf16" else 2.5e-4) * scale)


# --------------------------------------------------------------------- consistency (K7)

def _k7_inputs(W, H, seed=0):
    seq = synth.Sequence(width=W, height=H, seed=seed)
    I0, I1 = seq.frame(0), seq.frame(1)
    P0, P1 = seq.stylized(0, I0), seq.stylized(1, I1)
    O0 = P0 + synth.rng(seed + 7).normal(0, 0.01, P0.shape).astype(np.float32)
    return I1, P1, I0, P0, O0, seq.flow_backward(1), seq.flow_forward(1)


def _check_k7(got, ref, wc_tol=2e-4):
    O, wc, mask = got
    band = ref["band"] == 1
    assert band.mean() < 1e-3
    ok = ~band
    mism = (mask != ref["mask"]) & ok
    assert mism.sum() == 0, f"{mism.sum()} mask mismatches outside the band"
    err = np.abs(O - ref["O"]).max(0)
    assert err[ok].max() <= 1e-4, err[ok].max()
    lam = max(1.0, np.abs(ref["wc"]).max())
    assert np.abs(wc - ref["wc"])[ok].max() <= wc_tol * lam


@pytest.mark.parametrize("W,H", [(1920, 1080), (333, 197)])
@pytest.mark.parametrize("alpha,k1", [(6.5e3, 0.5), (0.0, 0.75), (6.5e3, 1.0)])
def test_consistency_given_flows(W, H, alpha, k1):
    It, Pt, Ip, Pp, Op, Fb, Ff = _k7_inputs(W, H)
    params = dict(k1=k1, alpha=alpha, lam=2.0)
    O, wc, mask = tc.op_consistency(*[to_dev(a) for a in (It, Pt, Ip, Pp, Op)], to_dev(planar_to_hw2(Fb)),
                                    to_dev(planar_to_hw2(Ff)), scale=1, **params)
    ref = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, Ff, **params)
    assert 0.3 < ref["mask"].mean() < 1.0
    _check_k7((to_np(O), to_np(wc), to_np(mask)), ref)


@pytest.mark.parametrize("W,H,scale", [(1920, 1080, 4), (250, 130, 4), (64, 64, 2)])
def test_consistency_upsampled_flows(W, H, scale):
    """Flows given at 1/scale resolution and upsampled inside the kernel (the final flow
    upsampling of the network fused into the consistency pass)."""
    It, Pt, Ip, Pp, Op, _, _ = _k7_inputs(W, H, seed=3)
    fh, fw = -(-H // scale), -(-W // scale)
    fb = synth.random_lowres_flow(fh, fw, 6.0 / scale, 31)
    ff = -fb + synth.random_lowres_flow(fh, fw, 0.6 / scale, 32)
    Fb = oracle.upsample_flow(fb, scale)[:, :H, :W]
    Ff = oracle.upsample_flow(ff, scale)[:, :H, :W]
    params = dict(k1=0.6, alpha=6.5e3, lam=2.0)
    O, wc, mask = tc.op_consistency(*[to_dev(a) for a in (It, Pt, Ip, Pp, Op)], to_dev(planar_to_hw2(fb)),
                                    to_dev(planar_to_hw2(ff)), scale=scale, **params)
    ref = oracle.consistency(It, Pt, Ip, Pp, Op, Fb, Ff, **params)
    # The in-bounds test compares x + u with the frame edge; the oracle's upsampled u is
    # FP64, so exclude pixels within 1e-4 px of an edge.
    yy, xx = np.mgrid[0:H, 0:W]
    sx, sy = xx + Fb[0], yy + Fb[1]
    edge = np.minimum.reduce([np.abs(sx), np.abs(sx - (W - 1)), np.abs(sy), np.abs(sy - (H - 1))]) < 1e-4
    ref["band"] = (ref["band"] | edge).astype(np.uint8)
    assert 0.2 < ref["mask"].mean()
    _check_k7((to_np(O), to_np(wc), to_np(mask)), ref)


def test_consistency_k1_zero_is_identity_on_processed_frame():
    It, Pt, Ip, Pp, Op, Fb, Ff = _k7_inputs(160, 96)
    O, wc, _ = tc.op_consistency(*[to_dev(a) for a in (It, Pt, Ip, Pp, Op)], to_dev(planar_to_hw2(Fb)),
                                 to_dev(planar_to_hw2(Ff)), scale=1, k1=0.0, alpha=6.5e3, lam=2.0)
    assert np.array_equal(to_np(O), Pt)
    assert (to_np(wc) == 2.0).all()
