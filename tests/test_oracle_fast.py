"""Pins of the oracle's fast preset (Table 3: the flow computed on frames downscaled by 2):

* downscale2 equals torch's 2x2 average pooling of the edge-replicated frame (odd sizes too);
* the x8 flow upsampling equals torch's bilinear interpolation (align_corners=False) x 8;
* with every estimator weight zero and head bias b the level-2 flow is (2^{L-1} - 1) b, so
  the fast preset's frame flow is 8 (2^{L-1} - 1) b (4 (2^{L-1} - 1) b at full size);
* a static pair gives the same zero-motion blend as the full-size network's stream
  (identical frames: every flow is the same constant for both).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle
import synth
from gpu_common import weights_file


@pytest.mark.parametrize("h,w", [(6, 8), (7, 9), (1, 5), (5, 1)])
def test_downscale2_is_average_pooling(h, w):
    x = synth.rng(90).random((3, h, w))
    t = torch.from_numpy(x)[None]
    t = Fnn.pad(t, (0, w % 2, 0, h % 2), mode="replicate") if (h % 2 or w % 2) else t
    ref = Fnn.avg_pool2d(t, 2)[0].numpy()
    np.testing.assert_allclose(oracle.downscale2(x), ref, rtol=0, atol=1e-15)


def test_upsample_by_8_matches_interpolate():
    f = synth.rng(91).normal(size=(2, 5, 7))
    ref = Fnn.interpolate(torch.from_numpy(f)[None], scale_factor=8, mode="bilinear", align_corners=False)[0] * 8
    np.testing.assert_allclose(oracle.upsample_flow(f, 8), ref.numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("fs", [1, 2])
def test_head_bias_only_flow_of_the_stream(fs):
    _, net0 = weights_file((16, 32, 48), 3)
    net = oracle.net_from_layers(net0.levels, net0.radius, net0.chans, net0.decoder,
                                 [dict(L, w=L["w"].copy(), b=L["b"].copy()) for L in net0.layers])
    b = np.array([0.25, -0.125])
    for i, L in enumerate(net.layers[3 * net.levels:]):
        L["w"][:] = 0
        L["b"][:] = 0
        if i % 5 == 4:
            L["b"][:] = b
    seq = synth.Sequence(width=70, height=50, seed=1, side_range=(8, 12), max_vel=2.0)
    frames = [seq.frame(t) for t in range(2)]
    st = oracle.Stream(net, flow_downscale=fs)
    st.step(frames[0], frames[0])
    r = st.step(frames[1], frames[1])
    want = 4 * fs * (2 ** (net.levels - 1) - 1) * b
    assert r["Fb"].shape == (2, 50, 70)
    np.testing.assert_array_equal(r["Fb"][0], np.full((50, 70), want[0]))
    np.testing.assert_array_equal(r["Ff"][1], np.full((50, 70), want[1]))


def test_fast_preset_flows_are_the_half_size_network_upsampled():
    """The fast preset's flow on a 64x48 frame equals the full-size oracle network's level-2
    flow on the 32x24 downscaled pair, upsampled x8 (pixels of the frame)."""
    _, net = weights_file((16, 32, 48), 3)
    seq = synth.Sequence(width=64, height=48, seed=2, side_range=(8, 12), max_vel=2.0)
    a, b = seq.frame(0), seq.frame(1)
    st = oracle.Stream(net, flow_downscale=2)
    st.step(a, a)
    r = st.step(b, b)
    ha, hb = oracle.downscale2(a), oracle.downscale2(b)
    pa, pb = oracle.pyramid(net, ha), oracle.pyramid(net, hb)
    _, lf = oracle.flow_from_pyramids(net, pb, pa, 24, 32, level_flows=True)
    np.testing.assert_array_equal(r["Fb"], oracle.upsample_flow(lf[0], 8)[:, :48, :64])
