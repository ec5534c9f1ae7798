"""FP64 oracle of the E4M3-quantised flow network (test infrastructure only).

The paper deploys its flow network with 8-bit linear weight quantisation and low-precision
accumulation (supplement, "Quantization and Mobile Deployment"); it gives no formula.  The
reading implemented here, and checked against the library's E4M3 path by the tests:

* E4M3 is the 8-bit float with 4 exponent bits (bias 7), 3 mantissa bits, subnormals, no
  infinities, largest finite value 448.  Rounding is to nearest, ties to even; values past
  448 saturate to +-448.
* An activation segment (a group of channels written by one producer; see ``segments``)
  has one scale s: a value x is held as e4m3(x / s), i.e. it is replaced by
  ``qdq(x, s) = e4m3(x / s) * s``.  Calibration takes s = amax / 448 over calibration frames.
* A convolution's weights are quantised per output channel o *after* folding the scale of
  each input channel in: w'[o, c] = w[o, c] s_in[c], s_w[o] = max |w'[o]| / 448, and the
  layer computes with w_eff[o, c] = e4m3(w'[o, c] / s_w[o]) s_w[o] / s_in[c].
* The first pyramid convolution (3 input channels) is not quantised; its output is.  Flows,
  the up-sampled flow used as the residual base, and the flow head's output stay exact.
* The feature warp and the cost volume requantise their outputs: the warped features with
  the scale of the features they warp, the cost volume with its own scale.

The 16-bit operand formats are modelled too (``round16``, ``flow_pair_16``): the weights
and/or every stored activation (pyramid outputs, warped features, cost volume, up-flow,
x1..x4) rounded to bfloat16 or IEEE half, the rest in FP64.  This is an attribution tool
for the precision variants (which rounding moves the flows how far), not a model of a
kernel's exact arithmetic.

Everything else is the network of ``oracle.flow_from_pyramids`` (Sec. 3.2), composed here
in Python from the same C primitives; with ``scales=None`` the composition reproduces
``oracle.flow_from_pyramids`` (a test pins that), and it can record the amax of every
segment instead of quantising.
"""
from __future__ import annotations

import numpy as np

from . import Net, conv3x3, correlation, pad_replicate, padded_size, upsample_flow, warp

E4M3_MAX = 448.0


def e4m3(a):
    """Nearest E4M3 value (ties to even, saturating at +-448), as float64."""
    a = np.asarray(a, np.float64)
    m = np.abs(a)
    _, ex = np.frexp(np.maximum(m, 2.0 ** -6))      # m = f 2^ex, f in [0.5, 1)
    q = np.ldexp(1.0, ex - 4)                         # quantum: 2^(e - 3) with e = ex - 1
    r = np.minimum(np.round(m / q) * q, E4M3_MAX)     # np.round: ties to even
    return np.where(a < 0, -r, r)


def qdq(x, s):
    """Quantise-dequantise with scale s (> 0)."""
    return e4m3(np.asarray(x, np.float64) / s) * s


def segments(net: Net) -> int:
    """Number of activation segments: 3 per pyramid level, 6 per estimator level."""
    return 3 * net.levels + 6 * (net.levels - 1)


def seg_pyr(net: Net, l: int, j: int) -> int:
    """Output of pyramid conv j (0, 1, 2) of level l (1..L)."""
    return 3 * (l - 1) + j


def seg_est(net: Net, l: int, k: int) -> int:
    """Estimator input group k of level l (L..2): 0 cost volume, 1 up-sampled flow, 2 x1,
    3 x2, 4 x3, 5 x4."""
    return 3 * net.levels + 6 * (net.levels - l) + k


def weight_qdq(w, s_in):
    """Per-output-channel E4M3 weights with the input-channel scales s_in (cin,) folded in."""
    w = np.asarray(w, np.float64)
    s_in = np.asarray(s_in, np.float64)
    wf = w * s_in[None, :, None, None]
    amax = np.abs(wf).reshape(w.shape[0], -1).max(1)
    sw = np.where(amax > 0, amax / E4M3_MAX, 1.0)
    return e4m3(wf / sw[:, None, None, None]) * sw[:, None, None, None] / s_in[None, :, None, None]


class _Q:
    """Quantises (scales given) or records amax (amax array given) or does nothing."""

    def __init__(self, scales=None, amax=None):
        self.scales = None if scales is None else np.where(np.asarray(scales, np.float64) > 0,
                                                           np.asarray(scales, np.float64), 1.0)
        self.amax = amax

    def act(self, x, seg):
        if self.amax is not None:
            self.amax[seg] = max(self.amax[seg], float(np.abs(x).max()) if x.size else 0.0)
        return x if self.scales is None else qdq(x, self.scales[seg])

    def conv(self, x, L, segs, stride=1):
        w = L["w"]
        if self.scales is not None and segs is not None:
            w = weight_qdq(w, self.scales[np.asarray(segs)])
        return conv3x3(x, w, L["b"], stride=stride, leaky=bool(L["leaky"]))


def pyramid_q(net: Net, img_padded, q: _Q):
    """Feature pyramid (Sec. 3.2) with the activations of every level passed through q."""
    feats = []
    cur = np.asarray(img_padded, np.float64)
    for l in range(1, net.levels + 1):
        La, Lb, Lc = net.layers[3 * (l - 1):3 * l]
        in_segs = None if l == 1 else [seg_pyr(net, l - 1, 2)] * La["cin"]
        t0 = q.act(q.conv(cur, La, in_segs, stride=2), seg_pyr(net, l, 0))
        t1 = q.act(q.conv(t0, Lb, [seg_pyr(net, l, 0)] * Lb["cin"]), seg_pyr(net, l, 1))
        cur = q.act(q.conv(t1, Lc, [seg_pyr(net, l, 1)] * Lc["cin"]), seg_pyr(net, l, 2))
        feats.append(cur)
    return feats


def flow_q(net: Net, feat_self, feat_other, hp, wp, q: _Q):
    """Coarse-to-fine flow F_{self->other} (Sec. 3.2) with the estimator inputs passed
    through q; same steps as ``oracle.flow_from_pyramids``."""
    nd = (2 * net.radius + 1) ** 2
    prev = None
    for l in range(net.levels, 1, -1):
        lh, lw, cl = hp >> l, wp >> l, net.chans[l - 1]
        E = net.layers[3 * net.levels + 5 * (net.levels - l):][:5]
        fs, fo = feat_self[l - 1], feat_other[l - 1]
        if prev is None:
            up = np.zeros((2, lh, lw))
            f2w = fo
        else:
            up = upsample_flow(prev, 2)
            f2w, _ = warp(fo, up, zero_outside=True)
            f2w = q.act(f2w, seg_pyr(net, l, 2)) if q.scales is not None else f2w
        cv = q.act(correlation(fs, f2w, net.radius), seg_est(net, l, 0))
        upq = q.act(up, seg_est(net, l, 1))
        x0 = np.concatenate([cv, fs, upq], 0)
        s0 = [seg_est(net, l, 0)] * nd + [seg_pyr(net, l, 2)] * cl + [seg_est(net, l, 1)] * 2
        x1 = q.act(q.conv(x0, E[0], s0), seg_est(net, l, 2))
        x2 = q.act(q.conv(x1, E[1], [seg_est(net, l, 2)] * E[1]["cin"]), seg_est(net, l, 3))
        x3 = q.act(q.conv(x2, E[2], [seg_est(net, l, 3)] * E[2]["cin"]), seg_est(net, l, 4))
        s32 = [seg_est(net, l, 4)] * x3.shape[0] + [seg_est(net, l, 3)] * x2.shape[0]
        x4 = q.act(q.conv(np.concatenate([x3, x2], 0), E[3], s32), seg_est(net, l, 5))
        s43 = [seg_est(net, l, 5)] * x4.shape[0] + [seg_est(net, l, 4)] * x3.shape[0]
        res = q.conv(np.concatenate([x4, x3], 0), E[4], s43)
        prev = up + res
    return upsample_flow(prev, 4)


def flow_pair_q(net: Net, I_a, I_b, scales=None):
    """F_{a->b} and F_{b->a} of two (3, h, w) frames through the quantised network."""
    _, h, w = I_a.shape
    hp, wp = padded_size(h, w, net.levels)
    q = _Q(scales)
    pa = pyramid_q(net, pad_replicate(I_a, hp, wp), q)
    pb = pyramid_q(net, pad_replicate(I_b, hp, wp), q)
    fab = flow_q(net, pa, pb, hp, wp, q)[:, :h, :w]
    fba = flow_q(net, pb, pa, hp, wp, q)[:, :h, :w]
    return np.ascontiguousarray(fab), np.ascontiguousarray(fba)


def calibrate(net: Net, frames):
    """amax of every activation segment over a frame sequence, as a stream sees it: every
    frame's pyramid, and both flow directions between consecutive frames."""
    amax = np.zeros(segments(net))
    q = _Q(amax=amax)
    _, h, w = frames[0].shape
    hp, wp = padded_size(h, w, net.levels)
    pyrs = [pyramid_q(net, pad_replicate(f, hp, wp), q) for f in frames]
    for a, b in zip(pyrs[1:], pyrs[:-1]):
        flow_q(net, a, b, hp, wp, q)
        flow_q(net, b, a, hp, wp, q)
    return amax


def scales_from_amax(amax):
    """E4M3 scales amax / 448 (1 for a segment that stayed zero)."""
    amax = np.asarray(amax, np.float64)
    return np.where(amax > 0, amax / E4M3_MAX, 1.0)


# ----------------------------------------------------------------------------- 16-bit formats

def round16(a, fmt):
    """Nearest value of the 16-bit format ("bf16": 8 significant bits, "fp16": IEEE half with
    subnormals), ties to even, as float64.  Values are first rounded to float32 (the
    library's storage of a float), then to the format."""
    a32 = np.ascontiguousarray(a, np.float32)
    if fmt == "fp16":
        with np.errstate(over="ignore"):  # beyond 65504 -> inf, as the conversion defines
            return a32.astype(np.float16).astype(np.float64)
    if fmt != "bf16":
        raise ValueError(fmt)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


class _R16(_Q):
    """Rounds weights and/or activations to a 16-bit format (see round16)."""

    def __init__(self, fmt, weights=True, activations=True):
        super().__init__()
        self.fmt, self.w, self.a = fmt, weights, activations

    def act(self, x, seg):
        return round16(x, self.fmt) if self.a else x

    def conv(self, x, L, segs, stride=1):
        w = round16(L["w"], self.fmt) if self.w else L["w"]
        return conv3x3(x, w, L["b"], stride=stride, leaky=bool(L["leaky"]))


def _flow_r16(net: Net, feat_self, feat_other, hp, wp, q: _R16):
    """flow_q with the warped features, cost volume and up-flow rounded by q as well."""
    prev = None
    for l in range(net.levels, 1, -1):
        lh, lw = hp >> l, wp >> l
        E = net.layers[3 * net.levels + 5 * (net.levels - l):][:5]
        fs, fo = feat_self[l - 1], feat_other[l - 1]
        if prev is None:
            up = np.zeros((2, lh, lw))
            f2w = fo
        else:
            up = upsample_flow(prev, 2)
            f2w = q.act(warp(fo, up, zero_outside=True)[0], None)
        x0 = np.concatenate([q.act(correlation(fs, f2w, net.radius), None), fs, q.act(up, None)], 0)
        x1 = q.act(q.conv(x0, E[0], None), None)
        x2 = q.act(q.conv(x1, E[1], None), None)
        x3 = q.act(q.conv(x2, E[2], None), None)
        x4 = q.act(q.conv(np.concatenate([x3, x2], 0), E[3], None), None)
        prev = up + q.conv(np.concatenate([x4, x3], 0), E[4], None)
    return upsample_flow(prev, 4)


def flow_pair_16(net: Net, I_a, I_b, fmt, weights=True, activations=True):
    """F_{a->b} and F_{b->a} with the weights and/or the stored activations rounded to the
    16-bit format fmt; flows, the residual base and the head's output stay FP64."""
    _, h, w = I_a.shape
    hp, wp = padded_size(h, w, net.levels)
    q = _R16(fmt, weights, activations)
    pa = pyramid_q(net, pad_replicate(I_a, hp, wp), q)
    pb = pyramid_q(net, pad_replicate(I_b, hp, wp), q)
    fab = _flow_r16(net, pa, pb, hp, wp, q)[:, :h, :w]
    fba = _flow_r16(net, pb, pa, hp, wp, q)[:, :h, :w]
    return np.ascontiguousarray(fab), np.ascontiguousarray(fba)
