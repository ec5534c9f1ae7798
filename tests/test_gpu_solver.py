"""The screened-Poisson solver (Eq. 1 by Eq. 8) on the GPU against the FP64 oracle: the
stage entry point, and streams with the solver on (tc_consistency.solver_iters).

Tolerance: for the paper's settings the iteration contracts (eta (8 + w_c) < 2 (1 + kappa)
for w_c <= 2), so float32 rounding does not grow through the 150 iterations: each update
rounds a handful of values of the iterate's scale (~1), about 2^-24 each, and the damped sum
over the iterations stays a few 1e-7 x the iteration count; the bound 5e-5 is about 10x
the 150-iteration figure."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import to_dev, to_np, weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

TOL = 5e-5


@pytest.mark.parametrize("c,h,w,iters", [(3, 37, 53, 150), (1, 70, 33, 7), (3, 96, 128, 17), (3, 16, 16, 1),
                                         (3, 200, 130, 150), (1, 1, 40, 9), (3, 33, 1, 16)])
def test_poisson_solve_matches_oracle(c, h, w, iters):
    g = synth.rng(70 + h)
    P = g.random((c, h, w)).astype(np.float32)
    A = g.random((c, h, w)).astype(np.float32)
    wc = (2.0 * g.random((h, w))).astype(np.float32)
    got = to_np(tc.op_poisson_solve(to_dev(P), to_dev(A), to_dev(wc), iters=iters, eta=0.15, kappa=0.2))
    want = oracle.poisson_solve(P, A, wc, eta=0.15, kappa=0.2, iters=iters)
    err = np.abs(got - want).max()
    assert err <= TOL, err


def test_poisson_solve_misaligned_buffers_match_aligned():
    """Buffers offset by one float (not 8-byte aligned) take the scalar load path; the
    result is the same bit for bit."""
    import torch
    g = synth.rng(73)
    c, h, w = 3, 150, 256
    P = g.random((c, h, w)).astype(np.float32)
    A = g.random((c, h, w)).astype(np.float32)
    wc = (2.0 * g.random((h, w))).astype(np.float32)
    ref = to_np(tc.op_poisson_solve(to_dev(P), to_dev(A), to_dev(wc), iters=20))

    def shifted(a):
        big = torch.zeros(a.size + 1, device="cuda")
        big[1:] = torch.from_numpy(a.ravel()).cuda()
        return big[1:].view(a.shape)
    got = to_np(tc.op_poisson_solve(shifted(P), shifted(A), shifted(wc), iters=20))
    assert np.array_equal(got, ref)
    want = oracle.poisson_solve(P, A, wc, iters=20)
    assert np.abs(got - want).max() <= TOL


def test_poisson_zero_iterations_and_fixed_point():
    g = synth.rng(71)
    P = g.random((3, 20, 30)).astype(np.float32)
    wc = g.random((20, 30)).astype(np.float32)
    A = g.random((3, 20, 30)).astype(np.float32)
    assert np.array_equal(to_np(tc.op_poisson_solve(to_dev(P), to_dev(A), to_dev(wc), iters=0)), A)
    # O = P = A is a fixed point: the gradient vanishes there
    out = to_np(tc.op_poisson_solve(to_dev(P), to_dev(P), to_dev(wc), iters=40))
    assert np.abs(out - P).max() <= 1e-6


def test_poisson_solve_at_1080p_matches_oracle_on_a_window():
    """Full-frame solve: away from the frame border a pixel's iterate depends only on inputs
    within 150 pixels, so a 400 x 400 window solved by the oracle (with the window's own
    Neumann border) agrees with the frame's solve on its centre 100 x 100."""
    import torch
    H, W = 1080, 1920
    P = torch.rand((3, H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    A = torch.rand((3, H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    wc = 2 * torch.rand((H, W), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    O = to_np(tc.op_poisson_solve(P, A, wc, iters=150))
    y0, x0 = 300, 700
    sl = (slice(None), slice(y0, y0 + 400), slice(x0, x0 + 400))
    want = oracle.poisson_solve(to_np(P)[sl], to_np(A)[sl], to_np(wc)[sl[1:]], iters=150)
    err = np.abs(O[:, y0 + 150:y0 + 250, x0 + 150:x0 + 250] - want[:, 150:250, 150:250]).max()
    assert err <= TOL, err
    # and the top-left corner, where the frame's own Neumann border applies
    want = oracle.poisson_solve(to_np(P)[:, :300, :300], to_np(A)[:, :300, :300], to_np(wc)[:300, :300], iters=150)
    err = np.abs(O[:, :140, :140] - want[:, :140, :140]).max()
    assert err <= TOL, err


def _frames(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_stream_solver_stage_by_stage(prec):
    """Each frame of a stream with the solver on: the stream's own flows and previous output
    give A_t and w_c through the consistency stage; the stream's output must be the FP64
    solve of Eq. 1 from that A_t, and the stream's w_c the stage's w_c bit for bit."""
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    W, H = 200, 136
    frames, styl = _frames(W, H, seed=5, n=4)
    params = dict(k1=0.5, alpha=6.5e3, lam=2.0)
    s = tc.Stream(W, H, prec, weights_path=path)
    s.set_consistency(solver_iters=150, eta=0.15, kappa=0.2, **params)
    prev = None
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, H, W), device="cuda")
        wc = torch.empty((H, W), device="cuda")
        s.process_frame(to_dev(I), to_dev(P), O, wc)
        if t == 0:
            s.synchronize()
            assert np.array_equal(to_np(O), P)
        else:
            Fb = torch.empty((2, H, W), device="cuda")
            Ff = torch.empty((2, H, W), device="cuda")
            s.get_flows(Fb, Ff)
            s.synchronize()
            hw2 = lambda f: f.permute(1, 2, 0).contiguous()
            A, wc_ref, _ = tc.op_consistency(to_dev(I), to_dev(P), to_dev(prev[0]), to_dev(prev[1]), prev[2],
                                             hw2(Fb), hw2(Ff), scale=1, **params)
            torch.cuda.synchronize()
            assert np.array_equal(to_np(wc), to_np(wc_ref)), t
            want = oracle.poisson_solve(P, to_np(A), to_np(wc_ref), eta=0.15, kappa=0.2, iters=150)
            err = np.abs(to_np(O) - want).max()
            assert err <= TOL, (t, err)
        prev = (I, P, O)
    s.destroy()


def test_stream_solver_matches_oracle_stream():
    """Whole streams, GPU FP32 against the FP64 oracle stream with the solver: alpha = 0
    makes the blend depend on the flow only through the bilinear taps and the mask, so the
    outputs agree to the flow deviation except around the pixels whose mask decision flips;
    the solve spreads those few differences without amplifying them."""
    import torch
    path, net = weights_file((16, 32, 48), 3)
    d = synth.pair64()
    frames = [d["I0"], d["I1"], d["I1"][:, ::-1].copy()]
    styl = [d["P0"], d["P1"], d["P1"][:, ::-1].copy()]
    params = dict(k1=0.5, alpha=0.0, lam=2.0)
    s = tc.Stream(64, 64, "fp32", weights_path=path)
    s.set_consistency(solver_iters=150, **params)
    ref = oracle.Stream(net, solver_iters=150, **params)
    for t, (I, P) in enumerate(zip(frames, styl)):
        O = torch.empty((3, 64, 64), device="cuda")
        wc = torch.empty((64, 64), device="cuda")
        m = torch.empty((64, 64), device="cuda", dtype=torch.uint8)
        s.process_frame(to_dev(I), to_dev(P), O, wc, m)
        r = ref.step(I, P)
        s.synchronize()
        err = np.abs(to_np(O) - r["O"])
        same = (to_np(m) == r["mask"]).mean()
        print(f"frame {t}: mask agreement {same:.4f}, max |dO| {err.max():.2e}, mean |dO| {err.mean():.2e}")
        assert same > 0.97
        assert err.mean() <= 2e-3 and np.quantile(err, 0.9) <= 1e-3, (t, err.mean())
    s.destroy()


def test_solver_graph_replay_matches_eager():
    import torch
    path, _ = weights_file((16, 32, 64, 96, 128), 4)
    frames, styl = _frames(200, 136, seed=9, n=5)
    runs = []
    for graphs in (False, True):
        s = tc.Stream(200, 136, "bf16", weights_path=path)
        s.set_graphs(graphs)
        outs = []
        for t, (I, P) in enumerate(zip(frames, styl)):
            # the iteration count changes mid-stream: graphs are rebuilt
            s.set_consistency(solver_iters=150 if t < 3 else 31)
            O = torch.empty((3, 136, 200), device="cuda")
            wc = torch.empty((136, 200), device="cuda")
            s.process_frame(to_dev(I), to_dev(P), O, wc)
            s.synchronize()
            outs.append((to_np(O), to_np(wc)))
        s.destroy()
        runs.append(outs)
    for t in range(len(frames)):
        assert np.array_equal(runs[0][t][0], runs[1][t][0]) and np.array_equal(runs[0][t][1], runs[1][t][1]), t


def test_solver_off_again_restores_the_causal_output():
    """Turning the solver off mid-stream returns to O_t = A_t."""
    import torch
    path, _ = weights_file((16, 32, 48), 3)
    frames, styl = _frames(64, 64, seed=3, n=3)
    s = tc.Stream(64, 64, "fp32", weights_path=path)
    s.set_consistency(solver_iters=150)
    outs = []
    for t, (I, P) in enumerate(zip(frames, styl)):
        if t == 2:
            s.set_consistency(solver_iters=0)
        O = torch.empty((3, 64, 64), device="cuda")
        s.process_frame(to_dev(I), to_dev(P), O)
        if t == 2:
            Fb = torch.empty((2, 64, 64), device="cuda")
            Ff = torch.empty((2, 64, 64), device="cuda")
            s.get_flows(Fb, Ff)
            hw2 = lambda f: f.permute(1, 2, 0).contiguous()
            A, _, _ = tc.op_consistency(to_dev(I), to_dev(P), to_dev(frames[1]), to_dev(styl[1]), outs[1],
                                        hw2(Fb), hw2(Ff), scale=1)
            s.synchronize()
            assert np.array_equal(to_np(O), to_np(A))
        outs.append(O)
    s.destroy()


@pytest.mark.parametrize("bad", [dict(solver_iters=-1), dict(solver_iters=10001), dict(solver_iters=5, eta=0.0),
                                 dict(solver_iters=5, kappa=1.0), dict(solver_iters=5, kappa=-0.1)])
def test_solver_controls_are_validated(bad):
    path, _ = weights_file((16, 32, 48), 3)
    s = tc.Stream(64, 64, "fp32", weights_path=path)
    with pytest.raises(tc.TcError) as e:
        s.set_consistency(**bad)
    assert e.value.status == tc.TC_ERR_INVALID_ARG
    s.destroy()


def test_server_rejects_the_solver():
    path, _ = weights_file((16, 32, 48), 3)
    srv = tc.Server(path, precision="bf16", workers=1)
    sid = srv.open(64, 64)
    with pytest.raises(tc.TcError) as e:
        srv.set_consistency(sid, solver_iters=150)
    assert e.value.status == tc.TC_ERR_UNSUPPORTED
    srv.destroy()
