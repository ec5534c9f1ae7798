"""8-bit video frames through tc_process_frame_host_rgb8_async.

The entry point decodes interleaved RGB8 codes q to q / 255 (float32 division), runs the
frame as tc_process_frame would on those values, and quantises O as floor(255 clamp(O, 0, 1)
+ 0.5) with the product and the sum rounded separately.  Checked here:
  * against the float32 host entry point given the decoded frames (the same kernels):
    O equal bit for bit after the same quantisation computed in float32 on the host, w_c and
    the mask equal bit for bit, on the eager first frames and the replayed graphs;
  * against the FP64 oracle's stream on the decoded frames with alpha = 0 (where O depends on
    the flows only through bilinear taps): every code within one step of the oracle's O
    quantised in float64, and equal wherever the oracle's value is not within 1e-3 of a code
    boundary;
  * the round trip of every code through the first frame (O_1 = P_1).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


def _frames8(W, H, seed, n):
    """Seeded sequence of the synthetic frames, clipped to [0, 1] and rounded to 8-bit codes,
    as interleaved (H, W, 3) uint8."""
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    out_i, out_p = [], []
    for t in range(n):
        f = seq.frame(t)
        p = seq.stylized(t, f)
        for a, dst in ((f, out_i), (p, out_p)):
            q = np.floor(np.clip(np.asarray(a, np.float64), 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)
            dst.append(np.ascontiguousarray(np.moveaxis(q, 0, -1)))
    return out_i, out_p


def _decode(q):
    """(H, W, 3) codes -> planar (3, H, W) float32 q / 255."""
    return np.ascontiguousarray(np.moveaxis(q, -1, 0).astype(np.float32) / np.float32(255.0))


def _quantise32(O):
    """Planar float32 O -> (H, W, 3) codes, in float32 as the entry point defines it."""
    v = np.clip(np.nan_to_num(O.astype(np.float32), nan=0.0), np.float32(0), np.float32(1))
    q = np.floor(v * np.float32(255.0) + np.float32(0.5)).astype(np.uint8)
    return np.ascontiguousarray(np.moveaxis(q, 0, -1))


def _run_rgb8(path, I8, P8, prec, **params):
    import torch
    H, W, _ = I8[0].shape
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_consistency(**params)
    pin = lambda a: torch.from_numpy(a).pin_memory()
    hI, hP = [pin(a) for a in I8], [pin(a) for a in P8]
    outs = [(torch.empty((H, W, 3), dtype=torch.uint8).pin_memory(), torch.empty((H, W)).pin_memory(),
             torch.empty((H, W), dtype=torch.uint8).pin_memory()) for _ in I8]
    for t in range(len(I8)):
        s.process_frame_host_rgb8_async(hI[t], hP[t], *outs[t])
    s.synchronize()
    s.destroy()
    return [tuple(o.numpy().copy() for o in out) for out in outs]


def _run_float(path, I8, P8, prec, **params):
    import torch
    H, W, _ = I8[0].shape
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_consistency(**params)
    res = []
    for I, P in zip(I8, P8):
        O = np.empty((3, H, W), np.float32)
        wc = np.empty((H, W), np.float32)
        m = np.empty((H, W), np.uint8)
        s.process_frame_host(_decode(I), _decode(P), O, wc, m)
        res.append((O, wc, m))
    s.destroy()
    torch.cuda.synchronize()
    return res


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_rgb8_entry_point_matches_float_entry_point(prec):
    path, _ = weights_file()
    I8, P8 = _frames8(64, 64, seed=11, n=5)
    got = _run_rgb8(path, I8, P8, prec, k1=0.4)
    want = _run_float(path, I8, P8, prec, k1=0.4)
    for t, ((O8, wc, m), (O, wcf, mf)) in enumerate(zip(got, want)):
        assert np.array_equal(O8, _quantise32(O)), t
        assert np.array_equal(wc, wcf) and np.array_equal(m, mf), t


def test_rgb8_ragged_size_matches_float_entry_point():
    path, _ = weights_file(chans=(16, 32, 64, 96, 128), radius=4)
    I8, P8 = _frames8(200, 136, seed=12, n=3)
    got = _run_rgb8(path, I8, P8, "fp16", k1=0.6)
    want = _run_float(path, I8, P8, "fp16", k1=0.6)
    for t, ((O8, wc, m), (O, wcf, mf)) in enumerate(zip(got, want)):
        assert np.array_equal(O8, _quantise32(O)) and np.array_equal(m, mf) and np.array_equal(wc, wcf), t


def test_rgb8_against_oracle_alpha0():
    path, net = weights_file()
    I8, P8 = _frames8(64, 64, seed=13, n=3)
    got = _run_rgb8(path, I8, P8, "fp32", k1=0.5, alpha=0.0)
    st = oracle.Stream(net, k1=0.5, alpha=0.0)
    for t in range(len(I8)):
        r = st.step(_decode(I8[t]).astype(np.float64), _decode(P8[t]).astype(np.float64))
        x = np.clip(np.asarray(r["O"], np.float64), 0.0, 1.0) * 255.0 + 0.5
        want = np.moveaxis(np.floor(x), 0, -1)
        near = np.moveaxis(np.abs(x - np.round(x)) < 1e-3 * 255.0, 0, -1)
        d = np.abs(got[t][0].astype(np.int32) - want.astype(np.int32))
        assert d.max() <= 1, t
        assert (d[~near] == 0).all(), t


def test_rgb8_first_frame_round_trip():
    """The first output is P_1 itself: every code, decoded and re-quantised, comes back
    unchanged (the decode and the quantisation are exact inverses on the codes)."""
    import torch
    path, _ = weights_file()
    W, H = 64, 64
    I8 = np.zeros((H, W, 3), np.uint8)
    P8 = (np.arange(H * W * 3) % 256).astype(np.uint8).reshape(H, W, 3)
    s = tc.Stream(W, H, "fp32", weights_path=path)
    O8 = torch.empty((H, W, 3), dtype=torch.uint8).pin_memory()
    s.process_frame_host_rgb8_async(torch.from_numpy(I8).pin_memory(), torch.from_numpy(P8).pin_memory(), O8)
    s.synchronize()
    s.destroy()
    assert np.array_equal(O8.numpy(), P8)
