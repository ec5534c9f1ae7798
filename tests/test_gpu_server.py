"""The multi-stream server (tc_server_*): results of a stream are the same alone, in a mix
with other streams running concurrently, and batched with streams of its size (frames of
several streams in one step's shared launches), and equal a plain stream's; HBM-budget
admission of shared batches, and cancellation."""
import numpy as np
import pytest

import synth
from gpu_common import weights_file

pytestmark = pytest.mark.gpu
tc = pytest.importorskip("paper_2301_00750_b300")

NET = ((16, 32, 64, 96, 128), 4)


def _frames(W, H, seed, n):
    seq = synth.Sequence(width=W, height=H, seed=seed, side_range=(max(8, W // 12), max(10, W // 6)),
                         max_vel=max(2.0, W / 160))
    I = [seq.frame(t) for t in range(n)]
    return I, [seq.stylized(t, f) for t, f in enumerate(I)]


def _drain(srv, n, timeout_s=60):
    import time
    got, t0 = [], time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        got += srv.poll(timeout_ms=200)
    return got


STREAMS = [(320, 200, 11), (256, 160, 12), (320, 200, 13), (200, 136, 14)]
N_FRAMES = 4


@pytest.mark.parametrize("batch_lanes", [1, 4])
def test_each_stream_alone_equals_in_the_mix(batch_lanes):
    import torch
    path, _ = weights_file(*NET)
    data = {k: _frames(W, H, seed, N_FRAMES) for k, (W, H, seed) in enumerate(STREAMS)}
    # a plain stream (tc_create_stream) per sequence
    plain = {}
    for k, (W, H, _) in enumerate(STREAMS):
        s = tc.Stream(W, H, "bf16", weights_path=path)
        O = torch.empty((3, H, W), device="cuda")
        plain[k] = []
        for t in range(N_FRAMES):
            s.process_frame(torch.from_numpy(data[k][0][t]).cuda(), torch.from_numpy(data[k][1][t]).cuda(), O)
            plain[k].append(O.cpu().numpy())
        s.destroy()
    # alone: one worker, one stream at a time
    alone = {}
    srv = tc.Server(path, precision="bf16", workers=1, batch_lanes=batch_lanes)
    for k, (W, H, _) in enumerate(STREAMS):
        sid = srv.open(W, H)
        outs = [np.zeros((3, H, W), np.float32) for _ in range(N_FRAMES)]
        for t in range(N_FRAMES):
            srv.submit(sid, data[k][0][t], data[k][1][t], outs[t], tag=t)
        done = _drain(srv, N_FRAMES)
        assert len(done) == N_FRAMES and all(c["status"] == 0 for c in done)
        assert [c["frame"] for c in done] == list(range(N_FRAMES))
        alone[k] = outs
        srv.close(sid)
    srv.destroy()
    # mix: four workers, all streams open, frames submitted interleaved (with batch_lanes 4
    # the two 320x200 streams share a batch, and their queued frames share steps)
    srv = tc.Server(path, precision="bf16", workers=4, batch_lanes=batch_lanes)
    sids = {k: srv.open(W, H) for k, (W, H, _) in enumerate(STREAMS)}
    mixed = {k: [np.zeros((3, H, W), np.float32) for _ in range(N_FRAMES)] for k, (W, H, _) in enumerate(STREAMS)}
    for t in range(N_FRAMES):
        for k in range(len(STREAMS)):
            srv.submit(sids[k], data[k][0][t], data[k][1][t], mixed[k][t], tag=100 * k + t)
    done = _drain(srv, N_FRAMES * len(STREAMS))
    assert len(done) == N_FRAMES * len(STREAMS) and all(c["status"] == 0 for c in done)
    for k in range(len(STREAMS)):
        frames = [c["frame"] for c in done if c["stream_id"] == sids[k]]
        assert frames == sorted(frames)            # per-stream order kept
    if batch_lanes > 1:
        assert max(c["batch"] for c in done) >= 2  # frames of two streams ran in one step
    else:
        assert all(c["batch"] == 1 for c in done)
    srv.destroy()
    for k in range(len(STREAMS)):
        for t in range(N_FRAMES):
            # same kernels, same inputs: bit-identical whatever else runs on the GPU
            assert np.array_equal(alone[k][t], mixed[k][t]), (k, t)
            assert np.array_equal(alone[k][t], plain[k][t]), (k, t)


def test_budget_admission_and_release():
    path, _ = weights_file(*NET)
    srv = tc.Server(path, precision="bf16", workers=2)
    per = srv.stream_bytes(320, 200)
    srv.destroy()
    srv = tc.Server(path, precision="bf16", workers=2, hbm_budget_bytes=2 * per + per // 2)
    a = srv.open(320, 200)
    b = srv.open(320, 200)
    with pytest.raises(tc.TcError) as e:
        srv.open(320, 200)
    assert e.value.status == tc.TC_ERR_BUSY
    assert srv.bytes_in_use == 2 * per
    srv.close(a)
    c = srv.open(320, 200)                          # the freed memory admits a new stream
    assert c not in (a, b) and srv.bytes_in_use == 2 * per
    srv.destroy()
    # shared batches: two streams of a size take two lanes of one batch, a third a new one
    srv = tc.Server(path, precision="bf16", workers=2, batch_lanes=2)
    per2 = srv.stream_bytes(320, 200)
    assert per < per2 < 2 * per
    a, b = srv.open(320, 200), srv.open(320, 200)
    assert srv.bytes_in_use == per2
    c = srv.open(320, 200)
    assert srv.bytes_in_use == 2 * per2
    srv.close(a)
    assert srv.bytes_in_use == 2 * per2             # its batch still holds b
    srv.close(b)
    assert srv.bytes_in_use == per2                 # the batch's last stream closed
    srv.close(c)
    assert srv.bytes_in_use == 0
    srv.destroy()


@pytest.mark.parametrize("lanes", [1, 3])
def test_admission_charge_covers_what_a_batch_allocates(lanes):
    path, _ = weights_file(*NET)
    for prec in ("bf16", "fp32", "fp16"):
        srv = tc.Server(path, precision=prec, workers=1, batch_lanes=lanes)
        want = srv.stream_bytes(320, 200)
        srv.destroy()
        b = tc.Batch(320, 200, lanes, prec, weights_path=path)
        got = tc.stream_device_bytes(b) + 3 * lanes * 3 * 200 * 320 * 4  # + the server's I, P, O staging
        b.destroy()
        assert got <= want <= 1.05 * got + (1 << 20), (prec, got, want)


def test_cancel_drops_queued_frames_in_order():
    path, _ = weights_file(*NET)
    srv = tc.Server(path, precision="bf16", workers=1)
    sid = srv.open(256, 160)
    I, P = _frames(256, 160, 21, 2)
    outs = [np.zeros((3, 160, 256), np.float32) for _ in range(12)]
    for t in range(12):
        srv.submit(sid, I[t % 2], P[t % 2], outs[t], tag=t)
    srv.cancel(sid)
    done = _drain(srv, 12)
    assert len(done) == 12
    ok = [c for c in done if c["status"] == 0]
    dropped = [c for c in done if c["status"] == tc.TC_ERR_STATE]
    assert len(ok) + len(dropped) == 12 and len(dropped) >= 1
    # what ran ran in order and first; the rest was dropped
    assert sorted(c["frame"] for c in ok) == list(range(len(ok)))
    assert sorted(c["frame"] for c in dropped) == list(range(len(ok), 12))
    srv.close(sid)
    srv.destroy()


def test_rgb8_submissions_equal_a_plain_stream_quantised():
    """8-bit submissions (tc_server_submit_rgb8), batched with a stream of the same size that
    submits float32 frames: each 8-bit stream's outputs equal a plain stream's float32
    outputs on the decoded frames, quantised (floor(255 clamp(O, 0, 1) + 0.5) in float32), and
    the float32 stream in the same batch is unchanged."""
    import torch
    path, _ = weights_file(*NET)
    W, H = 320, 200
    q8 = lambda a: np.ascontiguousarray(np.moveaxis(
        np.floor(np.clip(np.asarray(a, np.float64), 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8), 0, -1))
    dec = lambda q: np.ascontiguousarray(np.moveaxis(q, -1, 0).astype(np.float32) / np.float32(255.0))
    quant = lambda O: np.ascontiguousarray(np.moveaxis(np.floor(
        np.clip(O, np.float32(0), np.float32(1)) * np.float32(255.0) + np.float32(0.5)).astype(np.uint8), 0, -1))
    seqs = {k: _frames(W, H, 40 + k, N_FRAMES) for k in range(3)}
    rgb = {k: ([q8(a) for a in seqs[k][0]], [q8(a) for a in seqs[k][1]]) for k in (0, 1)}

    def plain(I, P):
        s = tc.Stream(W, H, "bf16", weights_path=path)
        O = torch.empty((3, H, W), device="cuda")
        out = []
        for a, b in zip(I, P):
            s.process_frame(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), O)
            out.append(O.cpu().numpy())
        s.destroy()
        return out

    want8 = {k: [quant(O) for O in plain([dec(q) for q in rgb[k][0]], [dec(q) for q in rgb[k][1]])] for k in (0, 1)}
    want32 = plain(*seqs[2])
    srv = tc.Server(path, precision="bf16", workers=2, batch_lanes=4)
    sids = {k: srv.open(W, H) for k in range(3)}
    got8 = {k: [np.zeros((H, W, 3), np.uint8) for _ in range(N_FRAMES)] for k in (0, 1)}
    got32 = [np.zeros((3, H, W), np.float32) for _ in range(N_FRAMES)]
    for t in range(N_FRAMES):
        for k in (0, 1):
            srv.submit_rgb8(sids[k], rgb[k][0][t], rgb[k][1][t], got8[k][t], tag=10 * k + t)
        srv.submit(sids[2], seqs[2][0][t], seqs[2][1][t], got32[t], tag=100 + t)
    done = _drain(srv, 3 * N_FRAMES)
    srv.destroy()
    assert len(done) == 3 * N_FRAMES and all(c["status"] == 0 for c in done)
    for k in (0, 1):
        for t in range(N_FRAMES):
            assert np.array_equal(got8[k][t], want8[k][t]), (k, t)
    for t in range(N_FRAMES):
        assert np.array_equal(got32[t], want32[t]), t
