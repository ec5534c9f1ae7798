"""Pins of the oracle's refinement network with depthwise-separable convs ("-sepref",
Sec. 3.2):

* the depthwise dilated 3x3 conv equals torch's grouped conv2d (groups = channels,
  dilation d, zero padding d), dilations larger than the map included;
* the pointwise conv equals an einsum over channels (+ LeakyReLU);
* the refinement chain equals an independent torch composition of cat(flow, x4, x3),
  grouped dilated convs, 1x1 convs and LeakyReLU, plus the flow;
* in the network: all-zero refinement weights leave the flow unchanged; with every
  estimator weight zero, head bias b and the last refinement bias c, the frame's flow is the
  closed form 4 ((2^{L-1} - 1) b + c) (the refinement acts on level 2, before the x4);
* TCW2 files round-trip through the writer and the oracle's parser.
"""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle
import synth
from gpu_common import weights_file


@pytest.mark.parametrize("dil", [1, 2, 5, 16])
def test_depthwise_matches_grouped_conv(dil):
    g = synth.rng(100 + dil)
    c, h, w = 5, 9, 13
    x = g.normal(size=(c, h, w))
    dw = g.normal(size=(c, 3, 3))
    db = g.normal(size=c)
    ref = Fnn.conv2d(torch.from_numpy(x)[None], torch.from_numpy(dw)[:, None], torch.from_numpy(db), padding=dil,
                     dilation=dil, groups=c)[0].numpy()
    np.testing.assert_allclose(oracle.depthwise3x3(x, dw, db, dil), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("leaky", [True, False])
def test_pointwise_matches_einsum(leaky):
    g = synth.rng(110)
    x = g.normal(size=(7, 6, 5))
    pw = g.normal(size=(4, 7))
    pb = g.normal(size=4)
    ref = np.einsum("oc,chw->ohw", pw, x) + pb[:, None, None]
    if leaky:
        ref = np.where(ref < 0, 0.1 * ref, ref)
    np.testing.assert_allclose(oracle.pointwise(x, pw, pb, leaky), ref, rtol=0, atol=1e-12)


def _rand_ref(g, cin, spec):
    ref = []
    for k, (cout, dil) in enumerate(spec):
        ref.append(dict(cin=cin, cout=cout, dil=dil, leaky=0 if k == len(spec) - 1 else 1,
                        dw=g.normal(size=(cin, 3, 3)), db=g.normal(size=cin), pw=g.normal(size=(cout, cin)) / cin,
                        pb=g.normal(size=cout)))
        cin = cout
    return ref


def test_refine_matches_torch_composition():
    g = synth.rng(120)
    h, w = 11, 14
    flow, x4, x3 = g.normal(size=(2, h, w)), g.normal(size=(4, h, w)), g.normal(size=(6, h, w))
    ref = _rand_ref(g, 12, [(8, 1), (8, 2), (5, 4), (2, 1)])
    t = torch.cat([torch.from_numpy(a) for a in (flow, x4, x3)])[None]
    for L in ref:
        t = Fnn.conv2d(t, torch.from_numpy(L["dw"])[:, None], torch.from_numpy(L["db"]), padding=L["dil"],
                       dilation=L["dil"], groups=L["cin"])
        t = Fnn.conv2d(t, torch.from_numpy(L["pw"])[:, :, None, None], torch.from_numpy(L["pb"]))
        if L["leaky"]:
            t = Fnn.leaky_relu(t, 0.1)
    want = flow + t[0].numpy()
    np.testing.assert_allclose(oracle.refine(flow, x4, x3, ref), want, rtol=0, atol=1e-11)


def _net_with_refine(chans=(16, 32, 48)):
    _, net = weights_file(chans, 3, refine=True)
    return oracle.Net(net.levels, net.radius, net.chans, net.decoder,
                      [dict(L, w=L["w"].copy(), b=L["b"].copy()) for L in net.layers],
                      [{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in L.items()} for L in net.ref])


def test_zero_refinement_leaves_the_flow():
    net = _net_with_refine()
    assert len(net.ref) == 7 and net.ref[0]["cin"] == 2 + 32 + 64
    plain = oracle.Net(net.levels, net.radius, net.chans, net.decoder, net.layers, [])
    for L in net.ref:
        for k in ("dw", "db", "pw", "pb"):
            L[k][:] = 0
    d = synth.pair64()
    a = oracle.flow_pair(net, d["I1"], d["I0"])
    b = oracle.flow_pair(plain, d["I1"], d["I0"])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_refinement_bias_closed_form():
    net = _net_with_refine()
    b = np.array([0.25, -0.125])
    c = np.array([0.5, 0.375])
    for i, L in enumerate(net.layers[3 * net.levels:]):
        L["w"][:] = 0
        L["b"][:] = b if i % 5 == 4 else 0
    for L in net.ref:
        for k in ("dw", "db", "pw", "pb"):
            L[k][:] = 0
    net.ref[-1]["pb"][:] = c
    h = w = 1 << (net.levels + 1)
    img = synth.rng(2).random((3, h, w))
    f = oracle.flow_from_pyramids(net, oracle.pyramid(net, img), oracle.pyramid(net, img), h, w)
    want = 4 * ((2 ** (net.levels - 1) - 1) * b + c)
    np.testing.assert_array_equal(f[0], want[0])
    np.testing.assert_array_equal(f[1], want[1])


def test_tcw2_round_trip():
    spec = synth.NetSpec(chans=(16, 32, 48), radius=3, refine=synth.REFINE_CHANS, refine_dil=synth.REFINE_DIL)
    layers = synth.he_weights(spec, seed=5)
    path = os.path.join(tempfile.mkdtemp(prefix="tcw2"), "net.tcw")
    synth.write_weights(path, spec, layers)
    with open(path, "rb") as f:
        assert f.read(4) == b"TCW2"
    net = oracle.load_weights(path)
    want = oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)
    assert len(net.ref) == len(want.ref) == 7
    for a, b in zip(net.ref, want.ref):
        assert (a["cin"], a["cout"], a["dil"], a["leaky"]) == (b["cin"], b["cout"], b["dil"], b["leaky"])
        for k in ("dw", "db", "pw", "pb"):
            assert np.array_equal(a[k], b[k])
    assert [L["cout"] for L in net.ref] == list(synth.REFINE_CHANS)
    assert [L["dil"] for L in net.ref] == list(synth.REFINE_DIL)
