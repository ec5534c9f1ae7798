"""End-to-end check over a 30-frame 1920x1080 sequence (the full-size staging of the
oracle's tolerances): the FP32 stream against the FP64 oracle's stream frame by frame.

With alpha = 0 (w_p = k1 M) O_t depends on the flows only through bilinear taps, so it must
stay within 1e-4 of the oracle's wherever no mask decision differed along the pixel's
history: a pixel is tainted when its mask differs from the oracle's (the flows differ by
~1e-5 px, which can flip a forward-backward decision lying that close to its threshold) or
lies in the oracle's rounding band, and at the next frame every pixel whose warp taps touch
a tainted pixel is tainted too (the previous output feeds every blend).  Over all 30 frames
the untainted pixels stay within 1e-4 and the tainted ones are a small fraction; the flow
EPE is held to 1e-3 px on every frame pair."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

N = 30


def test_30_frame_1080p_stream_matches_oracle_at_alpha_zero():
    import torch
    path, net = weights_file((16, 32, 64, 96, 128), 4)
    seq = synth.Sequence(seed=0)
    params = dict(k1=0.75, alpha=0.0, lam=2.0)
    s = tc.Stream(1920, 1080, "fp32", weights_path=path)
    s.set_consistency(**params)
    ref = oracle.Stream(net, **params)
    O = torch.empty((3, 1080, 1920), device="cuda")
    m = torch.empty((1080, 1920), device="cuda", dtype=torch.uint8)
    Fb = torch.empty((2, 1080, 1920), device="cuda")
    Ff = torch.empty((2, 1080, 1920), device="cuda")
    worst_o, worst_epe, worst_taint = 0.0, 0.0, 0.0
    taint = np.zeros((1080, 1920), bool)
    for t in range(N):
        I = seq.frame(t)
        P = seq.stylized(t, I)
        s.process_frame(to_dev(I), to_dev(P), O, None, m)
        if t > 0:
            s.get_flows(Fb, Ff)
        torch.cuda.synchronize()
        r = ref.step(I, P)
        got = to_np(O)
        if t == 0:
            assert np.array_equal(got, P)
            continue
        eb, ef = oracle.epe(to_np(Fb), r["Fb"]), oracle.epe(to_np(Ff), r["Ff"])
        worst_epe = max(worst_epe, eb, ef)
        assert eb <= 1e-3 and ef <= 1e-3, (t, eb, ef)
        # taps of this frame's warp that touch a pixel tainted at the previous frame
        touched = oracle.warp(taint[None].astype(np.float64), r["Fb"], zero_outside=False)[0][0] > 0
        taint = (to_np(m) != r["mask"]) | (r["band"] != 0) | touched
        worst_taint = max(worst_taint, float(taint.mean()))
        assert taint.mean() < 0.02, (t, taint.mean())
        err = np.abs(got - r["O"]).max(0)[~taint].max()
        worst_o = max(worst_o, float(err))
        assert err <= 1e-4, (t, err)
    s.destroy()
    print(f"30 frames at 1080p: worst O max-abs {worst_o:.2e} on untainted pixels (alpha = 0), worst tainted "
          f"fraction {worst_taint:.2e}, worst flow EPE {worst_epe:.2e} px")
