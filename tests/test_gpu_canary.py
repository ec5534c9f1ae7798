"""Canary padding around the output buffers of every stage op and of a stream's outputs:
guard regions on both sides of each output must be intact after the call (no write out of
bounds) and every output element must have been written.  This stands in for a device
memory checker, which is not available here.  Sizes are ragged (partial 128-pixel tiles,
odd widths, channel counts off the 64-channel step)."""
import numpy as np
import pytest

import synth
from gpu_common import check_guarded, guarded, nchw_to_nhwc, planar_to_hw2, round16, to_dev, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("n,h,w,cin,cout,stride", [(2, 9, 131, 40, 48, 1), (1, 17, 30, 32, 32, 2),
                                                   (1, 5, 257, 120, 128, 1), (2, 23, 200, 16, 16, 1)])
def test_conv3x3_canary(prec, n, h, w, cin, cout, stride):
    import torch
    g = synth.rng(60)
    x = to_dev(nchw_to_nhwc(round16(prec, g.normal(size=(n, cin, h, w)).astype(np.float32))))
    wt = (g.normal(size=(cout, cin, 3, 3)) / np.sqrt(9 * cin)).astype(np.float32)
    b = g.normal(0, 0.1, cout).astype(np.float32)
    shape = (n, (h - 1) // stride + 1, (w - 1) // stride + 1, cout)
    buf, out = guarded(shape)
    tc.op_conv3x3(x, wt, b, stride=stride, precision=prec, out=out)
    torch.cuda.synchronize()
    check_guarded(buf, shape)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("n,h,w,c,r", [(2, 19, 21, 32, 4), (1, 9, 37, 24, 2), (3, 17, 33, 128, 3)])
def test_correlation_and_warp_canary(prec, n, h, w, c, r):
    import torch
    g = synth.rng(61)
    f1 = to_dev(nchw_to_nhwc(round16(prec, g.normal(size=(n, c, h, w)).astype(np.float32))))
    f2 = to_dev(nchw_to_nhwc(round16(prec, g.normal(size=(n, c, h, w)).astype(np.float32))))
    shape = (n, h, w, (2 * r + 1) ** 2)
    buf, out = guarded(shape)
    tc.op_correlation(f1, f2, r, precision=prec, out=out)
    flow = to_dev(np.moveaxis(g.uniform(-5, 5, (n, 2, h, w)).astype(np.float32), 1, -1))
    wbuf, wout = guarded((n, h, w, c))
    tc.op_warp_features(f1, flow, precision=prec, out=wout)
    ubuf, uout = guarded((n, 4 * h, 4 * w, 2))
    tc.op_upsample_flow(flow, 4, out=uout)
    torch.cuda.synchronize()
    check_guarded(buf, shape)
    check_guarded(wbuf, (n, h, w, c))
    check_guarded(ubuf, (n, 4 * h, 4 * w, 2))


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_sepconv_downscale_solver_canary(prec):
    import torch
    g = synth.rng(62)
    n, h, w, cin, cout = 2, 13, 70, 40, 24
    x = to_dev(nchw_to_nhwc(round16(prec, g.normal(size=(n, cin, h, w)).astype(np.float32))))
    dw, db = g.normal(0, 0.3, (cin, 3, 3)), g.normal(0, 0.1, cin)
    pw, pb = g.normal(0, 0.2, (cout, cin)), g.normal(0, 0.1, cout)
    buf, out = guarded((n, h, w, cout))
    tc.op_sepconv(x, dw, db, pw, pb, dil=2, precision=prec, out=out)
    img = to_dev(g.random((3, 37, 51)).astype(np.float32))
    dbuf, dout = guarded((3, 19, 26))
    tc.op_downscale2(img, out=dout)
    P, A = img, to_dev(g.random((3, 37, 51)).astype(np.float32))
    wc = to_dev(g.random((37, 51)).astype(np.float32))
    sbuf, sout = guarded((3, 37, 51))
    tc.op_poisson_solve(P, A, wc, iters=20, out=sout)
    torch.cuda.synchronize()
    check_guarded(buf, (n, h, w, cout))
    check_guarded(dbuf, (3, 19, 26))
    check_guarded(sbuf, (3, 37, 51))


def test_consistency_canary():
    import torch
    W, H = 133, 71
    seq = synth.Sequence(width=W, height=H, seed=3, side_range=(10, 20), max_vel=3.0)
    I0, I1 = seq.frame(0), seq.frame(1)
    P0, P1 = seq.stylized(0, I0), seq.stylized(1, I1)
    fb = to_dev(planar_to_hw2(seq.flow_backward(1)))
    ff = to_dev(planar_to_hw2(seq.flow_forward(1)))
    ob, O = guarded((3, H, W))
    wb, wc = guarded((H, W))
    mb, m = guarded((H, W), "uint8")
    tc.op_consistency(to_dev(I1), to_dev(P1), to_dev(I0), to_dev(P0), to_dev(P0), fb, ff, scale=1, O=O, wc=wc, mask=m,
                      k1=0.5)
    torch.cuda.synchronize()
    check_guarded(ob, (3, H, W))
    check_guarded(wb, (H, W))
    check_guarded(mb, (H, W), "uint8")  # mask bytes are 0 or 1, never the marker
    assert set(np.unique(m.cpu().numpy())) <= {0, 1}


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_stream_outputs_canary(prec):
    """Four frames of a 5-level stream at a ragged size (graphs captured and replayed from
    the third frame): O_t, w_c, the mask and the flows stay inside their buffers."""
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    W, H = 200, 136
    seq = synth.Sequence(width=W, height=H, seed=8, side_range=(16, 30), max_vel=2.0)
    s = tc.Stream(W, H, prec, weights_path=path)
    for t in range(4):
        I = seq.frame(t)
        P = seq.stylized(t, I)
        ob, O = guarded((3, H, W))
        wb, wc = guarded((H, W))
        mb, m = guarded((H, W), "uint8")
        s.process_frame(to_dev(I), to_dev(P), O, wc, m)
        fbb, Fb = guarded((2, H, W))
        ffb, Ff = guarded((2, H, W))
        if t > 0:
            s.get_flows(Fb, Ff)
        s.synchronize()
        check_guarded(ob, (3, H, W))
        check_guarded(wb, (H, W))
        check_guarded(mb, (H, W), "uint8")
        assert set(np.unique(m.cpu().numpy())) <= {0, 1}
        check_guarded(fbb, (2, H, W), written=t > 0)
        check_guarded(ffb, (2, H, W), written=t > 0)
    s.destroy()
