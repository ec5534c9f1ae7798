"""Trains the lite flow network on seeded synthetic pairs with known flow (Sec. 3.2
"Training"; supplement "Training Settings") and scores the result.

    python -m paper_2301_00750_b300.train_synthetic [--pairs 20000] [--batch 32] [--epochs 60]
        [--lr 1e-4] [--out learned.tcw] [--precision bf16]

* Data: ``--pairs`` 256x256 pairs of ``synth.training_pair`` (blurred-noise texture, smooth
  random flow |F| <= 16 px, 0-3 occluding rectangles; seeds 1,000,000 + i), generated on
  the host by a process pool and kept on the device for the whole run; 256 held-out pairs
  (seeds 9,000,000 + i).
* Training: the library's native trainer (tc_trainer_run): forward, multi-scale EPE loss
  with equal level weights, the hand-written backward passes, AdamW on float32 master
  weights; batch ``--batch`` drawn without replacement, reshuffled every epoch (seeded).
* Score: held-out EPE (Eq. 10) of the network's final flow (level-2 flow upsampled x4)
  against the ground truth, beside the brute-force SSD-argmin flow (tc_op_bruteforce_flow,
  radius 16) and the zero flow.
* Precision check on the learned weights: a 1920x1080 pair of the seeded sequence through
  FP32, FP16, BF16 and E4M3 streams; each variant's EPE against the FP32 flows, and the FP32
  flows' EPE against the sequence's analytic flow.

Prints one JSON line; writes the learned weights (TCW1) to ``--out``.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

import synth

TRAIN_SEED, HELD_SEED = 1_000_000, 9_000_000
SIZE, MAX_FLOW = 256, 16.0
BRUTE_RADIUS = 16


def _chunk(args):
    seed0, n = args
    ps = [synth.training_pair(seed0 + i, SIZE, MAX_FLOW) for i in range(n)]
    return (np.stack([p[0] for p in ps]), np.stack([p[1] for p in ps]), np.stack([p[2] for p in ps]))


def generate(pool, seed0, n, chunk=64):
    """Yields (a, b, flow) host chunks of the pairs seed0 .. seed0 + n - 1, in order."""
    jobs = [(seed0 + k, min(chunk, n - k)) for k in range(0, n, chunk)]
    yield from pool.imap(_chunk, jobs)


def upsampled_epe(torch, tc, lf2, gt):
    """Mean EPE of the level-2 flows (B, h/4, w/4, 2) upsampled x4 against (B, 2, h, w)."""
    full = tc.op_upsample_flow(lf2.contiguous(), 4)  # (B, h, w, 2)
    d = full.permute(0, 3, 1, 2) - gt
    return d.square().sum(1).sqrt().mean(dim=(1, 2))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--held-out", type=int, default=256)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--workers", type=int, default=0, help="host processes generating pairs (0: all CPUs)")
    ap.add_argument("--out", default="learned.tcw")
    ap.add_argument("--eval-every", type=int, default=10, help="epochs between held-out evaluations")
    ap.add_argument("--skip-precision-check", action="store_true")
    args = ap.parse_args()

    # The pool is started (spawn) before the first GPU call.
    workers = args.workers or len(os.sched_getaffinity(0))
    pool = mp.get_context("spawn").Pool(workers)

    import torch

    import paper_2301_00750_b300 as tc
    import paper_2301_00750_b300.train as tr

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    A = torch.empty((args.pairs, 3, SIZE, SIZE), device="cuda")
    B = torch.empty_like(A)
    F = torch.empty((args.pairs, 2, SIZE, SIZE), device="cuda")
    k = 0
    for a, b, f in generate(pool, TRAIN_SEED, args.pairs):
        n = a.shape[0]
        A[k:k + n].copy_(torch.from_numpy(a))
        B[k:k + n].copy_(torch.from_numpy(b))
        F[k:k + n].copy_(torch.from_numpy(f))
        k += n
    held = [tuple(torch.from_numpy(x).cuda() for x in c) for c in generate(pool, HELD_SEED, args.held_out,
                                                                             chunk=args.batch)]
    pool.close()
    pool.join()
    t_data = time.perf_counter() - t0

    spec = synth.NetSpec()
    init = args.out + ".init"
    synth.write_weights(init, spec, synth.he_weights(spec, seed=0))
    t = tr.Trainer(args.batch, SIZE, SIZE, args.precision, weights_path=init, lr=args.lr)

    def held_out_epe():
        e = []
        for a, b, f in held:
            if a.shape[0] != args.batch:
                continue
            t.run(a, b, f, mode="forward", wait=True)
            e.append(upsampled_epe(torch, tc, t.level_flow(2), f))
        return float(torch.cat(e).mean().item())

    curve = [dict(epoch=0, steps=0, held_out_epe=round(held_out_epe(), 4))]
    g = torch.Generator(device="cpu")
    g.manual_seed(12345)
    nb = args.pairs // args.batch
    t1 = time.perf_counter()
    for ep in range(1, args.epochs + 1):
        perm = torch.randperm(args.pairs, generator=g).cuda()
        for i in range(nb):
            idx = perm[i * args.batch:(i + 1) * args.batch]
            t.run(A.index_select(0, idx), B.index_select(0, idx), F.index_select(0, idx), mode="step")
        if ep % args.eval_every == 0 or ep == args.epochs:
            torch.cuda.synchronize()
            curve.append(dict(epoch=ep, steps=t.steps, train_loss=round(t.loss(), 4),
                              held_out_epe=round(held_out_epe(), 4),
                              seconds=round(time.perf_counter() - t1, 1)))
            print(json.dumps(curve[-1]), flush=True)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    t.export_weights(args.out)
    steps = t.steps
    t.destroy()
    del A, B, F

    # Yardsticks: brute-force SSD-argmin flow and the zero flow on the same held-out pairs.
    bf, zero = [], []
    for a, b, f in held:
        for i in range(a.shape[0]):
            kk = tr.bruteforce_flow(a[i].contiguous(), b[i].contiguous(), BRUTE_RADIUS)
            bf.append((tr.index_to_flow(kk, BRUTE_RADIUS) - f[i]).square().sum(0).sqrt().mean().item())
            zero.append(f[i].square().sum(0).sqrt().mean().item())

    line = {
        "what": "config-3 training: lite flow net 5 levels 16/32/64/96/128, radius 4, on seeded 256x256 pairs",
        "pairs": args.pairs, "held_out": args.held_out, "batch": args.batch, "epochs": args.epochs,
        "steps": steps, "lr": args.lr, "precision": args.precision,
        "seconds": {"data": round(t_data, 1), "train": round(t_train, 1)},
        "pairs_per_s": round(steps * args.batch / t_train, 1),
        "held_out_epe_px": {"network": curve[-1]["held_out_epe"], "untrained": curve[0]["held_out_epe"],
                            "brute_force_r16": round(float(np.mean(bf)), 4), "zero_flow": round(float(np.mean(zero)), 4)},
        "curve": curve, "weights": args.out,
    }
    if not args.skip_precision_check:
        line["precision_check_1080p"] = precision_check(torch, tc, args.out)
    print(json.dumps(line), flush=True)


def precision_check(torch, tc, path):
    """The learned net on the pair (frames 2, 1) of the seeded 1080p sequence: every variant's
    flows against the FP32 flows, and the FP32 flows against the analytic flow."""
    seq = synth.Sequence(seed=0)
    frames = [seq.frame(t) for t in range(3)]
    styl = [seq.stylized(t, f) for t, f in enumerate(frames)]
    dI = [torch.from_numpy(f).cuda() for f in frames]
    dP = [torch.from_numpy(p).cuda() for p in styl]
    H, W = frames[0].shape[1:]

    def flows(prec, scales=None):
        s = tc.Stream(W, H, prec, weights_path=path)
        if scales is not None:
            s.set_fp8_scales(scales)
        O = torch.empty((3, H, W), device="cuda")
        for t in (1, 2):
            s.process_frame(dI[t], dP[t], O)
        Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
        s.get_flows(Fb, Ff)
        s.synchronize()
        s.destroy()
        return Fb, Ff

    def epe(a, b):
        return round(float((a - b).square().sum(0).sqrt().mean().item()), 5)

    ref = flows("fp32")
    gt = torch.from_numpy(seq.flow_backward(2)).cuda()
    out = {"fp32_vs_analytic_flow_px": epe(ref[0], gt), "mean_flow_px": round(float(gt.square().sum(0).sqrt().mean()), 3)}
    scales = tc.calibrate_fp8(W, H, list(zip(dI, dP)), weights_path=path)
    for prec in ("fp16", "bf16", "fp8"):
        Fb, Ff = flows(prec, scales if prec == "fp8" else None)
        out[prec] = {"epe_vs_fp32_px": {"Fb": epe(Fb, ref[0]), "Ff": epe(Ff, ref[1])},
                     "at_fixed_epe": bool(max(epe(Fb, ref[0]), epe(Ff, ref[1])) <= 0.05)}
    return out


if __name__ == "__main__":
    main()
