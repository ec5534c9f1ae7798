"""Pins of the E4M3 oracle (oracle.quant) against things other than itself: PyTorch's
float8_e4m3fn conversion, hand-worked E4M3 values, the unquantised C oracle, and the
properties a quantiser must have (idempotence, the 2^-4 relative error bound)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import quant


def test_every_e4m3_code_is_a_fixed_point():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8).view(torch.float8_e4m3fn)
    v = codes.to(torch.float64).numpy()
    v = v[np.isfinite(v)]
    assert len(v) == 254                                   # 0x7f and 0xff are NaN
    assert np.array_equal(quant.e4m3(v), v)
    assert v.max() == 448.0 and np.min(v[v > 0]) == 2.0 ** -9


def test_rounding_matches_pytorch_float8_e4m3fn():
    g = synth.rng(3)
    x = np.concatenate([g.normal(size=20000) * s for s in (1e-3, 0.05, 1.0, 30.0)])
    x = x[np.abs(x) < 440].astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(quant.e4m3(x), want)


@pytest.mark.parametrize("x,want", [
    (448.0, 448.0), (500.0, 448.0), (-1e6, -448.0),        # saturation
    (1.0625, 1.0), (1.1875, 1.25), (-1.0625, -1.0),        # ties to even (step 1/8 in [1, 2))
    (2.0 ** -10, 0.0), (3 * 2.0 ** -10, 2.0 ** -8),        # subnormal ties (step 2^-9)
    (2.0 ** -6 + 2.0 ** -10, 2.0 ** -6), (240.0, 240.0), (232.0, 224.0), (248.0, 256.0),
])
def test_worked_values(x, want):
    assert quant.e4m3(np.array([x]))[0] == want


def test_qdq_idempotent_and_within_relative_bound():
    g = synth.rng(4)
    x = g.normal(size=50000) * 3.0
    s = float(np.abs(x).max()) / quant.E4M3_MAX
    y = quant.qdq(x, s)
    assert np.array_equal(quant.qdq(y, s), y)
    normal = np.abs(x) >= s * 2.0 ** -6
    rel = np.abs(y - x)[normal] / np.abs(x)[normal]
    assert rel.max() <= 2.0 ** -4 + 1e-15
    assert np.abs(y - x)[~normal].max() <= s * 2.0 ** -10 + 1e-18


def test_weight_qdq_per_output_channel():
    g = synth.rng(5)
    w = g.normal(size=(8, 6, 3, 3)) * np.arange(1, 9)[:, None, None, None]
    s_in = np.array([1.0, 0.5, 2.0, 0.25, 4.0, 1.0])
    wq = quant.weight_qdq(w, s_in)
    # each output channel's largest folded weight is exactly representable at 448 s_w
    for o in range(8):
        f = np.abs(w[o] * s_in[:, None, None]).max()
        k = np.argmax(np.abs(w[o] * s_in[:, None, None]))
        assert np.isclose(np.abs((wq[o] * s_in[:, None, None]).ravel()[k]), f, rtol=1e-15)
        err = np.abs((wq[o] - w[o]) * s_in[:, None, None])
        # half a quantum of the top binade [256, 448] of the codes (quantum 32), in weight units
        assert err.max() <= f * 16 / 448 * (1 + 1e-12)
    assert np.allclose(quant.weight_qdq(wq, s_in), wq, rtol=1e-14, atol=0)


def _net_and_frames(chans=(16, 32, 48), radius=3, W=64, H=48):
    spec = synth.NetSpec(chans=chans, radius=radius)
    layers = synth.he_weights(spec, seed=0)
    net = oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)
    seq = synth.Sequence(width=W, height=H, seed=2, side_range=(6, 12), max_vel=2.0)
    return net, [seq.frame(t) for t in range(3)]


def test_unquantised_composition_equals_c_oracle():
    net, fr = _net_and_frames()
    fab, fba = oracle.flow_pair(net, fr[0], fr[1])
    qab, qba = quant.flow_pair_q(net, fr[0], fr[1], scales=None)
    assert np.abs(qab - fab).max() <= 1e-10 and np.abs(qba - fba).max() <= 1e-10


def test_calibration_records_pyramid_amax():
    net, fr = _net_and_frames()
    amax = quant.calibrate(net, fr)
    assert amax.shape == (quant.segments(net),)
    hp, wp = oracle.padded_size(48, 64, net.levels)
    for l in range(1, net.levels + 1):
        m = max(np.abs(oracle.pyramid(net, oracle.pad_replicate(f, hp, wp))[l - 1]).max() for f in fr)
        assert np.isclose(amax[quant.seg_pyr(net, l, 2)], m, rtol=1e-12)
    # the coarsest level has no up-sampled flow
    assert amax[quant.seg_est(net, net.levels, 1)] == 0.0
    assert (amax[[quant.seg_est(net, l, k) for l in range(2, net.levels + 1) for k in (0, 2, 3, 4, 5)]] > 0).all()


def test_quantised_flow_close_to_exact_flow():
    """E4M3 activations and weights move the flow, but by a fraction of its size."""
    net, fr = _net_and_frames()
    sc = quant.scales_from_amax(quant.calibrate(net, fr))
    fab, _ = oracle.flow_pair(net, fr[0], fr[1])
    qab, _ = quant.flow_pair_q(net, fr[0], fr[1], scales=sc)
    mag = float(np.sqrt((fab ** 2).sum(0)).mean())
    e = oracle.epe(qab, fab)
    assert 0 < e < 0.5 * mag, (e, mag)
