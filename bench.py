"""Benchmark: 1080p frames/s of the per-frame hot path (flow network + consistency step).

One step = one frame of one stream through tc_process_frame: feature pyramid of frame t,
the flow network in both directions (t->t-1, t-1->t), and the fused warp + mask + blend,
on the synthetic 1920x1080 sequence (textured canvas under affine camera motion with 3
occluding squares), 5-level network 16/32/64/96/128, correlation radius 4, He-init
weights, consistency weight k1 swept over {0, .25, .5, .75, 1} frame by frame.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp16|bf16|fp8|fp32] [--impl ours|reference]

The metric is frames/s at a fixed flow error: EPE <= 0.05 px per direction against the
plain FP32 path's flows.  The headline runs the FP16 tensor-core path (half operands,
float32 accumulation), which meets that bar; BF16 and E4M3 are timed beside it with their
EPE against FP32 and marked as not at fixed EPE where they miss it.  E4M3 streams take
their activation scales from a BF16 pass over frames 0-2 of the sequence (amax / 448 per
activation segment), outside the timed region.

Multi-GPU (torchrun, one rank per GPU): every rank runs its own independent stream (the
path shards by stream, no collective on the data path); value = frames of all ranks / the
slowest rank's time (weak scaling).  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "1080p frames/s (flow+consistency) vs FP32 plain at fixed EPE; p99 frame latency"
UNIT = "frames/s"
K1_SWEEP = (0.0, 0.25, 0.5, 0.75, 1.0)
SOLVER_ITERS = 150  # Eq. 8 iterations per frame in the paper's full method
FIXED_EPE_PX = 0.05  # flow error bar of the reduced-precision variants, against FP32
SOLVER_FLOPS_PER_PX_ITER = 9  # per channel: neighbour sum (3 adds) and 3 FMAs
WIDTH, HEIGHT = 1920, 1080
SPEC = dict(chans=(16, 32, 64, 96, 128), radius=4)
N_FRAMES = 8
# DRAM read + write bytes of the FP16 estimator convs (conv1-conv4, levels 5-2, both flow
# directions) for one 1080p frame, from an ncu capture of the current persistent conv kernel.
ESTIMATOR_DRAM_BYTES_PER_FRAME = 662.5e6
# Peak of plain float32 FMA issue: 148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz.
FP32_SIMT_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


# ----------------------------------------------------------------------------- workload

def net_spec(refine=False):
    spec = synth.NetSpec(chans=SPEC["chans"], radius=SPEC["radius"])
    if refine:
        spec.refine, spec.refine_dil = synth.REFINE_CHANS, synth.REFINE_DIL
    return spec


def write_weights(path, refine=False):
    spec = net_spec(refine)
    synth.write_weights(path, spec, synth.he_weights(spec, seed=0))


def make_frames(seed, n=N_FRAMES, width=WIDTH, height=HEIGHT):
    seq = synth.Sequence(width=width, height=height, seed=seed)
    frames = [seq.frame(t) for t in range(n)]
    return frames, [seq.stylized(t, f) for t, f in enumerate(frames)]


def frame_order(step):
    """Ping-pong through the resident frames so consecutive frames stay consecutive."""
    period = 2 * (N_FRAMES - 1)
    k = step % period
    return k if k < N_FRAMES else period - k


def conv_flops_per_frame(spec, width=WIDTH, height=HEIGHT):
    """Algorithmic FLOPs (2 per multiply-add, true channel counts, no padding) per frame:
    pyramid of one frame + estimator convs (conv1..conv4) and the flow head in both
    directions + the correlation (both directions)."""
    L = spec.levels
    m = 1 << L
    hp, wp = -(-height // m) * m, -(-width // m) * m
    pyr = est = head = corr = 0
    for name, cin, cout, stride, _ in spec.layer_table():
        if name.startswith("pyr"):
            l = int(name[3])
            px = (hp >> l) * (wp >> l)
            pyr += 2 * px * cout * cin * 9
        else:
            l = int(name[3])
            px = 2 * (hp >> l) * (wp >> l)
            f = 2 * px * cout * cin * 9
            if name.endswith("c5"):
                head += f
            else:
                est += f
    d = (2 * spec.radius + 1) ** 2
    for l in range(2, L + 1):
        corr += 2 * 2 * (hp >> l) * (wp >> l) * d * spec.chans[l - 1]
    return dict(pyramid_conv=pyr, estimator_conv=est, head=head, correlation=corr)


# Algorithmic bytes per pixel of the fused consistency pass: read I_t, P_t (24 B), gather
# I, P, O of frame t-1 (36 B), write O_t (12 B), the kept copies of I_t, P_t, O_t (36 B),
# w_c (4 B) and the mask (1 B).  The level-2 flows it upsamples are < 1% of this.
CONSISTENCY_BYTES_PER_PX = 24 + 36 + 12 + 36 + 4 + 1


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, maximum SM clock, the throttle reasons seen active at least once,
        and the number of parsed samples, from nvidia-smi's CSV lines (FIELDS, no units)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ----------------------------------------------------------------------------- GPU arm

def dist_setup(backend=None):
    """One process per GPU (torchrun env).  NCCL on GPUs; gloo when no GPU is present (the
    host-side logic is tested that way).  The data path has no collective: every rank runs
    its own independent streams; only barriers and the max over ranks of the timed region
    use the process group."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, seconds_local, world):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds_local, world)


def fp8_scales(tc, path, dev_frames, dev_styl, flow_downscale=1):
    """E4M3 activation scales from a BF16 pass over frames 0-2 (static calibration)."""
    H, W = dev_frames[0].shape[1:]
    return tc.calibrate_fp8(W, H, list(zip(dev_frames[:3], dev_styl[:3])), weights_path=path,
                            flow_downscale=flow_downscale)


def open_stream(tc, path, W, H, precision, scales, flow_downscale=1):
    s = tc.Stream(W, H, precision, weights_path=path, flow_downscale=flow_downscale)
    if precision == "fp8":
        s.set_fp8_scales(scales)
    return s


def consistency_controls(step, solver_iters, latency):
    """k1 swept over K1_SWEEP; with one frame of latency the paper's final k1 = 0.3, k2 = 0.5
    (k1 + k2 must stay below 1)."""
    if latency:
        return dict(k1=0.3, k2=0.5, solver_iters=solver_iters)
    return dict(k1=K1_SWEEP[step % len(K1_SWEEP)], solver_iters=solver_iters)


def time_stream(tc, torch, path, dev_frames, dev_styl, precision, steps, warmup, profile=False, scales=None,
                solver_iters=0, latency=0, flow_downscale=1, pipelined=False, frame_timing=False):
    """Runs warmup + steps frames through one stream; returns timings (device events).
    pipelined: tc_set_pipelined (frame t+1's pyramid overlaps the flow estimation of frames t
    and t-1, each with its own buffer set);
    the timed region then ends with tc_join, and there are no per-frame times."""
    H, W = dev_frames[0].shape[1:]
    s = open_stream(tc, path, W, H, precision, scales, flow_downscale)
    if latency:
        s.set_consistency(**consistency_controls(0, solver_iters, latency))
        s.set_latency(latency)
    if pipelined:
        s.set_pipelined(True)
    O = torch.empty((3, H, W), device="cuda")
    wc = torch.empty((H, W), device="cuda")
    mask = torch.empty((H, W), device="cuda", dtype=torch.uint8)
    step = 0
    for _ in range(warmup):
        s.set_consistency(**consistency_controls(step, solver_iters, latency))
        i = frame_order(step)
        s.process_frame(dev_frames[i], dev_styl[i], O, wc, mask)
        step += 1
    s.synchronize()
    torch.cuda.synchronize()
    if profile:
        s.set_profiling(True)
    if frame_timing:
        s.set_frame_timing(True)  # pipelined: per-frame device latency (pyramid may start -> blend done)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    launches = 0
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(steps):
        s.set_consistency(**consistency_controls(step, solver_iters, latency))
        i = frame_order(step)
        s.process_frame(dev_frames[i], dev_styl[i], O, wc, mask)
        launches += s.launch_count
        if not pipelined:
            ev[k + 1].record(stream)
        step += 1
    if pipelined:
        s.join()
        ev[steps].record(stream)
    torch.cuda.synchronize()
    per = None if pipelined else [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    prof = s.get_profile() if profile else None
    frame_ms = [float(v) for v in s.get_frame_times(steps)] if frame_timing else None
    tc_layers, tc_corr = s.tensor_core_layers, s.tensor_core_correlation_levels
    s.destroy()
    return dict(total_ms=total, per_frame_ms=per, launches=launches, profile=prof, tc_layers=tc_layers,
                tc_corr=tc_corr, frame_ms=frame_ms)


def pair_flows(tc, torch, path, dev_frames, dev_styl, precision, scales=None):
    """F_{t->t-1}, F_{t-1->t} of the pair (frames 2, 1) of the resident sequence through a
    stream of the given precision (device tensors)."""
    H, W = dev_frames[0].shape[1:]
    s = open_stream(tc, path, W, H, precision, scales)
    O = torch.empty((3, H, W), device="cuda")
    for t in (1, 2):
        s.process_frame(dev_frames[t], dev_styl[t], O)
    Fb, Ff = torch.empty((2, H, W), device="cuda"), torch.empty((2, H, W), device="cuda")
    s.get_flows(Fb, Ff)
    s.synchronize()
    s.destroy()
    return Fb, Ff


def epe_px(a, b):
    """Average end-point error (Eq. 10) between two (2, H, W) device flows."""
    return float(((a - b) ** 2).sum(0).sqrt().mean().item())


def pipelined_value(entry, res, n):
    """Adds the pipelined-mode frames/s of a side configuration (the value is the default mode's)."""
    if res is not None:
        entry["pipelined"] = round(n / (res["total_ms"] / 1e3), 3)


def e2e_host(tc, torch, path, frames, styl, precision, steps, warmup, scales=None, solver_iters=0, latency=0,
             flow_downscale=1, pipelined=False, pipe_mode=False):
    """End-to-end through the host-buffer entry points: pinned host I_t, P_t in, O_t out per
    frame.  pipelined: tc_process_frame_host_async for every frame (uploads, kernels and
    downloads of neighbouring frames overlap; four output buffers in rotation) and one
    tc_synchronize inside the timed region; else tc_process_frame_host, which waits for
    each frame.  pipe_mode: the stream in pipelined mode (tc_set_pipelined), with the async
    call only."""
    H, W = frames[0].shape[1:]
    s = open_stream(tc, path, W, H, precision, scales, flow_downscale)
    if latency:
        s.set_consistency(**consistency_controls(0, solver_iters, latency))
        s.set_latency(latency)
    if pipe_mode:
        s.set_pipelined(True)
    hI = [torch.from_numpy(f).pin_memory() for f in frames]
    hP = [torch.from_numpy(p).pin_memory() for p in styl]
    hO = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(4 if pipelined else 1)]
    call = s.process_frame_host_async if pipelined else s.process_frame_host
    step = 0
    for _ in range(warmup):
        i = frame_order(step)
        s.set_consistency(**consistency_controls(step, solver_iters, latency))
        call(hI[i], hP[i], hO[step % len(hO)])
        step += 1
    s.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        i = frame_order(step)
        s.set_consistency(**consistency_controls(step, solver_iters, latency))
        call(hI[i], hP[i], hO[step % len(hO)])
        step += 1
    s.synchronize()
    dt = time.perf_counter() - t0
    s.destroy()
    img = 3 * H * W * 4
    return dict(value=steps / dt, h2d=2 * img, d2h=img)


def e2e_host_rgb8(tc, torch, path, frames, styl, precision, steps, warmup, scales=None, pipe_mode=False):
    """End-to-end with 8-bit video frames (tc_process_frame_host_rgb8_async): the synthetic
    frames clipped to [0, 1] and rounded to interleaved RGB8 codes, uploaded, decoded on the
    device, run, and O_t quantised and downloaded as RGB8; one tc_synchronize inside the timed
    region, as the float32 `e2e`."""
    H, W = frames[0].shape[1:]
    q8 = lambda a: torch.from_numpy(np.ascontiguousarray(np.moveaxis(
        np.floor(np.clip(a, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8), 0, -1))).pin_memory()
    hI, hP = [q8(f) for f in frames], [q8(p) for p in styl]
    hO = [torch.empty((H, W, 3), dtype=torch.uint8).pin_memory() for _ in range(4)]
    s = open_stream(tc, path, W, H, precision, scales)
    if pipe_mode:
        s.set_pipelined(True)
    step = 0
    for _ in range(warmup):
        i = frame_order(step)
        s.set_consistency(**consistency_controls(step, 0, 0))
        s.process_frame_host_rgb8_async(hI[i], hP[i], hO[step % 4])
        step += 1
    s.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        i = frame_order(step)
        s.set_consistency(**consistency_controls(step, 0, 0))
        s.process_frame_host_rgb8_async(hI[i], hP[i], hO[step % 4])
        step += 1
    s.synchronize()
    dt = time.perf_counter() - t0
    s.destroy()
    return dict(value=steps / dt, h2d=2 * 3 * H * W, d2h=3 * H * W)


def host_link(torch, img_bytes, reps=10):
    """The host link's throughput for the end-to-end copy pattern of one frame, measured with
    pinned buffers: H2D of I_t and P_t (2 x img_bytes) alone, D2H of O_t (img_bytes) alone, and
    both at once on two streams.  The link roofline takes the two directions as independent
    (full duplex): 1 / max(H2D time, D2H time) frames/s; the concurrent time is reported beside
    it (it came out above the pipelined entry point's own per-frame time, which overlaps the
    copies of neighbouring frames better than back-to-back bursts do)."""
    n = img_bytes // 4
    hin = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    hout = torch.empty(n, dtype=torch.float32).pin_memory()
    din = [torch.empty(n, device="cuda") for _ in range(2)]
    dout = torch.empty(n, device="cuda")
    up, down = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(h2d, d2h):
        for it in range(reps + 2):
            if it == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            if h2d:
                with torch.cuda.stream(up):
                    for k in range(2):
                        din[k].copy_(hin[k], non_blocking=True)
            if d2h:
                with torch.cuda.stream(down):
                    hout.copy_(dout, non_blocking=True)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t_up, t_down, t_both = timed(True, False), timed(False, True), timed(True, True)
    return dict(h2d_gbs=round(2 * img_bytes / t_up / 1e9, 1), d2h_gbs=round(img_bytes / t_down / 1e9, 1),
                both_ms_per_frame=round(t_both * 1e3, 4), frames_per_s_bound=round(1.0 / max(t_up, t_down), 1))


def oracle_threads():
    """Threads of the oracle's OpenMP loops: OMP_NUM_THREADS when set, else (the OpenMP
    default) the CPUs this process may run on."""
    v = os.environ.get("OMP_NUM_THREADS", "").split(",")[0].strip()
    return int(v) if v.isdigit() and int(v) > 0 else len(os.sched_getaffinity(0))


def cpu_baseline_oracle(seed=0):
    """The FP64 oracle timed on this host's cores on a bounded sample: one full 1080p frame
    step (pyramid of frame t, both flow directions, consistency) after frame t-1."""
    import oracle
    spec = net_spec()
    layers = synth.he_weights(spec, seed=0)
    net = oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)
    seq = synth.Sequence(width=WIDTH, height=HEIGHT, seed=seed)
    f0, f1 = seq.frame(0), seq.frame(1)
    p0, p1 = seq.stylized(0, f0), seq.stylized(1, f1)
    st = oracle.Stream(net, k1=0.5)
    st.step(f0, p0)
    t0 = time.perf_counter()
    st.step(f1, p1)
    dt = time.perf_counter() - t0
    return dict(value=1.0 / dt, unit=UNIT, cores=oracle_threads(), kind="oracle",
                sample=f"one 1920x1080 frame step of the FP64 oracle (pyramid, both flow directions, "
                       f"consistency), {dt:.1f} s")


def run_ours(args):
    import torch
    import paper_2301_00750_b300 as tc

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    tmp = tempfile.mkdtemp(prefix="tcbench")
    path = os.path.join(tmp, "net.tcw")
    write_weights(path)
    frames, styl = make_frames(seed=rank)
    dev_frames = [torch.from_numpy(f).cuda() for f in frames]
    dev_styl = [torch.from_numpy(p).cuda() for p in styl]
    torch.cuda.synchronize()
    scales = fp8_scales(tc, path, dev_frames, dev_styl, args.flow_downscale) \
        if args.precision == "fp8" or not args.skip_fp8 else None

    clocks = ClockSampler(local)
    barrier(world)
    clocks.start()
    time.sleep(0.3)
    main = time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, args.steps, args.warmup,
                       scales=scales, solver_iters=args.solver_iters, latency=args.latency,
                       flow_downscale=args.flow_downscale, pipelined=not args.sequential)
    clk = clocks.stop()
    barrier(world)
    total_s = max_over_ranks(main["total_ms"] / 1e3, world)
    value = weak_scaling_value(args.steps, main["total_ms"] / 1e3, world)
    # the default (sequential) mode: each frame ordered on the caller's stream, per-frame
    # device times for the latency percentiles
    seq = main if args.sequential else time_stream(
        tc, torch, path, dev_frames, dev_styl, args.precision, args.steps, args.warmup, scales=scales,
        solver_iters=args.solver_iters, latency=args.latency, flow_downscale=args.flow_downscale)

    # Pipelined mode's per-frame latency, in a pass of its own (two timing events per frame)
    plat = None if args.sequential else time_stream(
        tc, torch, path, dev_frames, dev_styl, args.precision, args.steps, args.warmup, scales=scales,
        solver_iters=args.solver_iters, latency=args.latency, flow_downscale=args.flow_downscale, pipelined=True,
        frame_timing=True)
    # Per-stage device times over the same number of steps (events around every launch).
    prof = time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, args.steps, 2, profile=True,
                       scales=scales, solver_iters=args.solver_iters, latency=args.latency,
                       flow_downscale=args.flow_downscale)
    fp32 = fp8 = fp8_pipe = None
    if args.precision != "fp32" and not args.skip_fp32:
        fp32 = time_stream(tc, torch, path, dev_frames, dev_styl, "fp32", max(3, args.steps // 4), 2,
                           flow_downscale=args.flow_downscale)
    if args.precision != "fp8" and not args.skip_fp8:
        fp8 = time_stream(tc, torch, path, dev_frames, dev_styl, "fp8", args.steps, 3, scales=scales,
                          flow_downscale=args.flow_downscale)
        fp8_pipe = None if args.sequential else time_stream(
            tc, torch, path, dev_frames, dev_styl, "fp8", args.steps, 3, scales=scales,
            flow_downscale=args.flow_downscale, pipelined=True)
    # Every reduced-precision variant's flows against the FP32 path's on one frame pair, and
    # its frames/s (pipelined and sequential): the metric is frames/s at EPE <= 0.05 px.
    variants = {}
    if not args.skip_variants and args.flow_downscale == 1 and args.latency == 0 and args.solver_iters == 0:
        ref = pair_flows(tc, torch, path, dev_frames, dev_styl, "fp32")
        for prec in ("fp16", "bf16", "fp8"):
            if prec == "fp8" and scales is None:
                continue  # E4M3 not calibrated in this run (--skip-fp8)
            Fb, Ff = pair_flows(tc, torch, path, dev_frames, dev_styl, prec, scales if prec == "fp8" else None)
            eb, ef = epe_px(Fb, ref[0]), epe_px(Ff, ref[1])
            if prec == args.precision:
                vp, vs = (None if args.sequential else main), seq
            elif prec == "fp8" and fp8 is not None:
                vp, vs = fp8_pipe, fp8
            else:
                vs = time_stream(tc, torch, path, dev_frames, dev_styl, prec, args.steps, 3,
                                 scales=scales if prec == "fp8" else None)
                vp = None if args.sequential else time_stream(
                    tc, torch, path, dev_frames, dev_styl, prec, args.steps, 3,
                    scales=scales if prec == "fp8" else None, pipelined=True)
            nv = len(vs["per_frame_ms"])
            pv = sorted(vs["per_frame_ms"])
            variants[prec] = {
                "pipelined": round(args.steps / (vp["total_ms"] / 1e3), 3) if vp is not None else None,
                "sequential": round(nv / (vs["total_ms"] / 1e3), 3),
                "p99_ms_sequential": round(pv[min(nv - 1, int(0.99 * nv))], 4),
                "epe_vs_fp32_px": {"Fb": round(eb, 5), "Ff": round(ef, 5)},
                "at_fixed_epe": bool(max(eb, ef) <= FIXED_EPE_PX)}
        Fm = ref[0].square().sum(0).sqrt().mean().item()
        variants["note"] = (f"flows of the pair (frames 2, 1), mean |F_b| {Fm:.2f} px; fixed EPE: <= "
                            f"{FIXED_EPE_PX} px per direction against the FP32 path")
    solver = None
    if not args.skip_solver and args.solver_iters == 0:
        # the paper's full output: Eq. 1 solved by 150 Eq. 8 iterations after the blend
        n = max(3, args.steps // 4)
        solver = (time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, solver_iters=SOLVER_ITERS,
                              scales=scales),
                  time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 2, profile=True,
                              solver_iters=SOLVER_ITERS, scales=scales),
                  None if args.sequential else
                  time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, solver_iters=SOLVER_ITERS,
                              scales=scales, pipelined=True))
    latency = None
    if not args.skip_latency and args.latency == 0:
        # the paper's one-frame-latency form (next frame in Eqs. 2, 3, 6; k1 0.3, k2 0.5)
        n = max(3, args.steps // 4)
        latency = (time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, scales=scales, latency=1),
                   time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, profile=True,
                               scales=scales, latency=1),
                   None if args.sequential else
                   time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, scales=scales, latency=1,
                               pipelined=True))
    refined = None
    if not args.skip_refine and args.precision != "fp8":
        # the network with the depthwise-separable refinement after the level-2 estimator
        rpath = os.path.join(tmp, "net_ref.tcw")
        write_weights(rpath, refine=True)
        n = max(3, args.steps // 4)
        refined = (time_stream(tc, torch, rpath, dev_frames, dev_styl, args.precision, n, 3,
                               flow_downscale=args.flow_downscale),
                   time_stream(tc, torch, rpath, dev_frames, dev_styl, args.precision, n, 3, profile=True,
                               flow_downscale=args.flow_downscale),
                   None if args.sequential else
                   time_stream(tc, torch, rpath, dev_frames, dev_styl, args.precision, n, 3,
                               flow_downscale=args.flow_downscale, pipelined=True))
    fast = None
    if not args.skip_fast and args.flow_downscale == 1:
        # the paper's fast preset (Table 3): flow on half-size frames, 50 solver iterations
        n = max(3, args.steps // 4)
        fscales = fp8_scales(tc, path, dev_frames, dev_styl, 2) if args.precision == "fp8" else None
        fast = (time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, scales=fscales,
                            solver_iters=50, flow_downscale=2),
                time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, profile=True,
                            scales=fscales, solver_iters=50, flow_downscale=2),
                None if args.sequential else
                time_stream(tc, torch, path, dev_frames, dev_styl, args.precision, n, 3, scales=fscales,
                            solver_iters=50, flow_downscale=2, pipelined=True))
    e2e = e2e_host(tc, torch, path, frames, styl, args.precision, max(3, min(args.steps, 100)), 3, scales=scales,
                   solver_iters=args.solver_iters, latency=args.latency, flow_downscale=args.flow_downscale,
                   pipelined=True, pipe_mode=not args.sequential)
    e2e_sync = e2e_host(tc, torch, path, frames, styl, args.precision, max(3, min(args.steps, 50)), 2,
                        scales=scales, solver_iters=args.solver_iters, latency=args.latency,
                        flow_downscale=args.flow_downscale)
    e2e_v, e2e_sync_v = e2e["value"], e2e_sync["value"]
    H, W = frames[0].shape[1:]
    link = host_link(torch, 3 * H * W * 4)
    e2e8 = None
    if not args.latency and not args.solver_iters and args.flow_downscale == 1:
        e2e8 = e2e_host_rgb8(tc, torch, path, frames, styl, args.precision, max(3, min(args.steps, 100)), 3,
                             scales=scales, pipe_mode=not args.sequential)
    if world > 1:
        e2e_v = world / max_over_ranks(1.0 / e2e["value"], world)
        e2e_sync_v = world / max_over_ranks(1.0 / e2e_sync["value"], world)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    gemm_peaks = measure_gemm_peaks(torch) if not args.skip_peaks else {}
    fp32_peak = gemm_peaks.get("fp32_tflops") or FP32_SIMT_PEAK_TFLOPS
    fp32_peak_source = ("of measured fp32 SGEMM (this run, TF32 off)" if gemm_peaks.get("fp32_tflops")
                        else "derived: 148 SM x 128 FP32 lanes x 2 x 2032 MHz")
    flops = conv_flops_per_frame(net_spec())
    p = prof["profile"]
    steps = args.steps
    dom = max(p, key=lambda k: p[k][0])
    # Convs (and the correlation) of a 16-bit stream run on the tensor cores: roofline against
    # the measured dense bf16 peak (fp16 has the same nominal dense rate), the burst figure:
    # the profiled pass times a few hundred milliseconds, not a seconds-long loop.  FP32
    # streams run on the CUDA cores: derived FP32 FMA peak.
    tensor_path = prof["tc_layers"] > 0 if dom != "correlation" else prof["tc_corr"] > 0
    peaks = measured_peaks()
    if dom == "solver":
        achieved = SOLVER_FLOPS_PER_PX_ITER * 3 * WIDTH * HEIGHT * args.solver_iters * steps / (p[dom][0] / 1e3) / 1e12
        peak, unit, bound = fp32_peak, "TFLOP/s", "alu"
    elif dom in ("estimator_conv", "pyramid_conv", "head", "correlation"):
        achieved = flops[dom] * steps / (p[dom][0] / 1e3) / 1e12
        if tensor_path and args.precision == "fp8":
            # the e4m3 GEMM peak measured in this run, else the bf16 one x the nominal dense
            # fp8 : bf16 ratio (4.5 : 2.25)
            peak, unit, bound = gemm_peaks.get("e4m3_tflops") or 2 * peaks.get("bf16_tflops"), "TFLOP/s", "tensor"
        elif tensor_path:
            peak, unit, bound = peaks.get("bf16_tflops"), "TFLOP/s", "tensor"
        else:
            peak, unit, bound = fp32_peak, "TFLOP/s", "alu"
    else:
        achieved = CONSISTENCY_BYTES_PER_PX * WIDTH * HEIGHT * steps / (p[dom][0] / 1e3) / 1e9
        peak, unit, bound = peaks.get("hbm_gbs"), "GB/s", "hbm"
    if bound == "alu":
        peak_source = fp32_peak_source
    elif bound == "tensor" and args.precision == "fp8":
        peak_source = ("of measured e4m3 cuBLAS GEMM (this run)" if gemm_peaks.get("e4m3_tflops") else
                       "of measured bf16 burst x 2 (nominal dense fp8:bf16), MEASURED_PEAKS.json")
    elif bound == "tensor":
        peak_source = ("of measured bf16 burst (MEASURED_PEAKS.json; fp16 and bf16 have the same nominal "
                       "dense rate)" if args.precision == "fp16" else "of measured bf16 burst (MEASURED_PEAKS.json)")
    else:
        peak_source = "of measured HBM copy (MEASURED_PEAKS.json)"
    per = sorted(seq["per_frame_ms"])
    # DRAM bytes of the dominant class per frame, from one ncu capture of the current kernels
    # (cold reads, writes partly still in L2); known for the default FP16 workload only
    traffic, traffic_note = None, "no ncu capture of this configuration"
    if (dom == "estimator_conv" and args.precision == "fp16" and args.flow_downscale == 1 and
            args.solver_iters == 0 and args.latency == 0):
        traffic = ESTIMATOR_DRAM_BYTES_PER_FRAME
        traffic_note = ("conv1-conv4 of levels 5-2, both directions, one frame: dram__bytes_read.sum + "
                        "dram__bytes_write.sum over the 16 launches (ncu capture of the current kernels)")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(total_s * 1e3 / steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp8": "e4m3", "fp32": "f32", "fp16": "f16"}.get(args.precision, args.precision),
        "data": "synthetic (seeded 1080p sequence, He-init weights)",
        "config": workload_config(args),
        "mode": ("sequential: each frame ordered on the caller's stream" if args.sequential else
                 "pipelined (tc_set_pipelined): frame t+1's feature pyramid runs on its own stream while "
                 "two frames' flow estimations run on two more; inputs resident, one tc_join at the end "
                 "of the timed region"),
        "sequential": {"value": round(args.steps / (seq["total_ms"] / 1e3), 3), "unit": UNIT,
                       "ms_per_step": round(seq["total_ms"] / args.steps, 4)},
        "latency_ms": {"p50": round(per[len(per) // 2], 4), "p99": round(per[min(len(per) - 1, int(0.99 * len(per)))], 4),
                       "mode": "sequential (per-frame device time)"},
        "latency_ms_pipelined": (None if plat is None else {
            "p50": round(sorted(plat["frame_ms"])[len(plat["frame_ms"]) // 2], 4),
            "p99": round(sorted(plat["frame_ms"])[min(len(plat["frame_ms"]) - 1, int(0.99 * len(plat["frame_ms"])))], 4),
            "frames_per_s_while_timed": round(args.steps / (plat["total_ms"] / 1e3), 3),
            "mode": "pipelined: device time from the moment a frame's pyramid may start to the end of its blend"}),
        "stage_ms_per_frame": {k: round(v[0] / steps, 4) for k, v in p.items() if v[1]},
        "roofline": {"kernel": dom, "bound": bound, "achieved": round(achieved, 2), "peak": peak, "unit": unit,
                     "frac": round(achieved / peak, 4) if peak else None,
                     "traffic": traffic,
                     "traffic_note": traffic_note,
                     "peak_source": peak_source},
        "gpu_launches": main["launches"],
        "clocks": clk,
        "e2e": {"value": round(e2e_v * (world if world > 1 else 1), 3), "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                "api": "tc_process_frame_host_async for every frame from pinned host memory, one "
                       "tc_synchronize at the end of the timed region (uploads and downloads overlap the "
                       "neighbouring frames' kernels)" + ("" if args.sequential else "; the stream in pipelined mode"),
                "link": dict(link, frac=round(e2e["value"] / link["frames_per_s_bound"], 4),
                             note="host link roofline of this copy pattern, measured in this run with pinned "
                                  "buffers: 1 / max(H2D time of I_t + P_t, D2H time of O_t), the two directions "
                                  "taken as independent; frac = e2e / that bound")},
        "e2e_sync": {"value": round(e2e_sync_v * (world if world > 1 else 1), 3), "unit": UNIT,
                     "h2d_bytes_per_step": e2e_sync["h2d"], "d2h_bytes_per_step": e2e_sync["d2h"],
                     "api": "tc_process_frame_host, which waits for each frame (its P_t upload overlaps the "
                            "flow network)"},
    }
    if e2e8 is not None:
        line["e2e_rgb8"] = {"value": round(e2e8["value"] * (world if world > 1 else 1), 3), "unit": UNIT,
                            "h2d_bytes_per_step": e2e8["h2d"], "d2h_bytes_per_step": e2e8["d2h"],
                            "api": "tc_process_frame_host_rgb8_async: 8-bit interleaved RGB frames in and out "
                                   "(the synthetic frames clipped to [0, 1] and rounded to codes), decoded and "
                                   "quantised on the device, one tc_synchronize at the end of the timed region"
                                   + ("" if args.sequential else "; the stream in pipelined mode")}
    if gemm_peaks:
        line["measured_gemm_peaks"] = gemm_peaks
    if variants:
        line["variants"] = variants
        if args.precision in variants:
            line["at_fixed_epe"] = variants[args.precision]["at_fixed_epe"]
    if fp32 is not None:
        line["fp32_plain"] = {"value": round(len(fp32["per_frame_ms"]) / (fp32["total_ms"] / 1e3), 3), "unit": UNIT}
    if fp8 is not None:
        p8 = sorted(fp8["per_frame_ms"])
        line["fp8_e4m3"] = {"value": round(len(p8) / (fp8["total_ms"] / 1e3), 3), "unit": UNIT,
                            "p99_ms": round(p8[min(len(p8) - 1, int(0.99 * len(p8)))], 4),
                            "mode": "sequential",
                            "scales": "static, amax/448 from a BF16 pass over frames 0-2"}
        if fp8_pipe is not None:
            line["fp8_e4m3"]["pipelined"] = round(args.steps / (fp8_pipe["total_ms"] / 1e3), 3)
    if solver is not None:
        sv, svp, svq = solver
        n = len(sv["per_frame_ms"])
        ms = svp["profile"]["solver"][0] / n
        line["with_solver"] = {
            "value": round(n / (sv["total_ms"] / 1e3), 3), "unit": UNIT, "iters": SOLVER_ITERS,
            "solver_ms_per_frame": round(ms, 4),
            "pixel_iterations_per_s": round(WIDTH * HEIGHT * SOLVER_ITERS / (ms / 1e3), 1),
            # 9 flops (3 adds, 3 FMAs) per pixel, channel and iteration, on the CUDA cores
            "roofline": {"kernel": "solver", "bound": "alu",
                         "achieved": round(SOLVER_FLOPS_PER_PX_ITER * 3 * WIDTH * HEIGHT * SOLVER_ITERS / (ms / 1e3) / 1e12, 3),
                         "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                         "frac": round(SOLVER_FLOPS_PER_PX_ITER * 3 * WIDTH * HEIGHT * SOLVER_ITERS / (ms / 1e3) / 1e12
                                       / fp32_peak, 4),
                         "peak_source": fp32_peak_source},
            "note": "Eq. 1 by Eq. 8 (eta 0.15, kappa 0.2) after the blend, time-blocked 8 iterations per launch"}
        pipelined_value(line["with_solver"], svq, n)
    if refined is not None:
        rt, rtp, rtq = refined
        n = len(rt["per_frame_ms"])
        line["with_refinement"] = {
            "value": round(n / (rt["total_ms"] / 1e3), 3), "unit": UNIT,
            "refine_ms_per_frame": round(rtp["profile"]["refine"][0] / n, 4),
            "note": "network + depthwise-separable refinement (7 layers 128/128/128/96/64/32/2, dilations "
                    "1/2/4/8/16/1/1) on the level-2 flows of both directions"}
        pipelined_value(line["with_refinement"], rtq, n)
    if fast is not None:
        ft, ftp, ftq = fast
        n = len(ft["per_frame_ms"])
        pf = sorted(ft["per_frame_ms"])
        line["fast_preset"] = {
            "value": round(n / (ft["total_ms"] / 1e3), 3), "unit": UNIT,
            "p99_ms": round(pf[min(n - 1, int(0.99 * n))], 4),
            "stage_ms_per_frame": {k: round(v[0] / n, 4) for k, v in ftp["profile"].items() if v[1]},
            "note": "Table 3's fast preset: flow network on 960x540 2x2-mean frames (flow upsampled x8), "
                    "50 Eq. 8 iterations"}
        pipelined_value(line["fast_preset"], ftq, n)
    if latency is not None:
        lt, ltp, ltq = latency
        n = len(lt["per_frame_ms"])
        line["with_next_frame"] = {
            "value": round(n / (lt["total_ms"] / 1e3), 3), "unit": UNIT, "latency_frames": 1,
            "consistency_ms_per_frame": round(ltp["profile"]["consistency"][0] / n, 4),
            "note": "frame t returned with frame t+1: w_n of Eq. 3 (k2 0.5) in Eqs. 2 and 6, k1 0.3"}
        pipelined_value(line["with_next_frame"], ltq, n)
    if world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline_oracle()
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "_fallback": True}


def measure_gemm_peaks(torch, n=8192, reps=8):
    """Dense peaks the way the bf16 one is measured: the best of `reps` cuBLAS GEMMs of
    n^3 (2 n^3 flop each, CUDA events) -- e4m3 x e4m3 -> bf16 through torch._scaled_mm
    (unit scales) and float32 x float32 with TF32 off (the CUDA cores' FMA path)."""
    out = {}

    def best(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return 2.0 * n ** 3 / min(ts) / 1e12

    try:
        a8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()  # column-major operand
        one = torch.ones((), device="cuda")
        out["e4m3_tflops"] = round(best(lambda: torch._scaled_mm(a8, b8, one, one, out_dtype=torch.bfloat16)), 1)
        del a8, b8
    except Exception as e:  # noqa: BLE001 (reported, not fatal)
        out["e4m3_error"] = str(e)[:200]
    tf32 = torch.backends.cuda.matmul.allow_tf32
    try:
        torch.backends.cuda.matmul.allow_tf32 = False
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        out["fp32_tflops"] = round(best(lambda: torch.matmul(a, b)), 2)
        del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    torch.cuda.empty_cache()
    out["how"] = (f"best of {reps} cuBLAS GEMMs of {n}^3 (2 n^3 flop): torch._scaled_mm e4m3 x e4m3 -> bf16, "
                  f"and torch.matmul float32 with TF32 off (CUDA-core FMA)")
    return out


# ----------------------------------------------------------------------------- reference arm

def workload_config(args):
    """The line's `config`: the workload, named by what it is and its sizes."""
    return {"workload": "1920x1080 RGB stream, lite flow net 5 levels 16/32/64/96/128, radius 4, "
                        "decoder 128/96/64/32/2, both flow directions + fused consistency, "
                        + ("k1 swept {0,.25,.5,.75,1}" if not args.latency else
                           "k1 0.3 and k2 0.5 with the next frame (one frame of latency)")
                        + (f", then {args.solver_iters} Eq. 8 solver iterations" if args.solver_iters else "")
                        + (", flow network on 2x2-mean half-size frames" if args.flow_downscale == 2 else ""),
            "frames_resident": N_FRAMES, "streams_per_gpu": 1,
            "precision": args.precision, "l2": "per-frame working set > 126 MB L2 (no flush needed)"}


def run_reference(args):
    """The FP64 oracle on this host's cores, with the main arm's workload and settings (the
    k1 sweep or one frame of latency, solver iterations, the flow downscale).  Each step is a
    bounded sample: one frame step of a 1920x128 band of the sequence (pyramid, both flows,
    consistency, the solver when on), reported as 1080p-frame equivalents per second.  Under
    torchrun rank 0 alone runs it."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    spec = net_spec()
    layers = synth.he_weights(spec, seed=0)
    net = oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers)
    bh = 128
    seq = synth.Sequence(width=WIDTH, height=bh, seed=0)
    nf = 3 if args.latency else 2
    frames = [seq.frame(t) for t in range(nf)]
    styl = [seq.stylized(t, f) for t, f in enumerate(frames)]

    def one_step(i):
        # the timed call computes one output frame: the flows of its pair and the blend
        c = consistency_controls(i, args.solver_iters, args.latency)
        st = oracle.Stream(net, k1=c["k1"], k2=c.get("k2", 0.5), solver_iters=c["solver_iters"],
                           latency=args.latency, flow_downscale=args.flow_downscale)
        for t in range(nf - 1):
            st.step(frames[t], styl[t])
        t0 = time.perf_counter()
        st.step(frames[nf - 1], styl[nf - 1])
        return time.perf_counter() - t0

    for i in range(args.warmup):
        one_step(i)
    times = [one_step(i) for i in range(args.steps)]
    frac = (WIDTH * bh) / (WIDTH * HEIGHT)
    total = sum(times)
    value = args.steps * frac / total
    sample = f"per step: one frame step of a 1920x{bh} band ({frac:.4f} of a 1080p frame), FP64 oracle"
    config = workload_config(args)
    config["precision"] = "f64 (oracle)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded sequence, He-init weights)", "config": config,
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": sample + "; one host process (rank 0)"},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- serving

SERVE_MIX = [(640, 360, 4), (1280, 720, 4), (1920, 1080, 6), (2560, 1440, 2)]


def serve_load(srv, streams, frames_by_size, rate, seconds, seed, warm=1.0):
    """Poisson frame arrivals at `rate` frames/s per stream for warm + seconds; returns served
    frames/s over the measured window, latency percentiles, batch sizes and drops."""
    g = np.random.Generator(np.random.PCG64(seed))
    latencies, batches, done_n, dropped = [], [], 0, 0
    tag_slot = {}
    for s_ in streams:
        s_["free"] = list(range(len(s_["outs"])))
        s_["next"] = g.exponential(1.0 / rate)
    t0 = time.perf_counter()
    n_tag = 0
    while True:
        now = time.perf_counter() - t0
        if now > seconds + warm:
            break
        for s_ in streams:
            while s_["next"] <= now:
                if not s_["free"]:
                    dropped += s_["next"] >= warm  # client found no free output slot: frame skipped
                else:
                    slot = s_["free"].pop()
                    fr, st = frames_by_size[(s_["W"], s_["H"])]
                    k = s_["n"] % len(fr)
                    n_tag += 1
                    tag_slot[n_tag] = (s_, slot, s_["next"])
                    (srv.submit_rgb8 if s_.get("rgb8") else srv.submit)(s_["id"], fr[k], st[k], s_["outs"][slot],
                                                                       tag=n_tag)
                    s_["n"] += 1
                s_["next"] += g.exponential(1.0 / rate)
        for c in srv.poll(timeout_ms=1):
            s_, slot, t_sub = tag_slot.pop(c["tag"])
            s_["free"].append(slot)
            if c["status"] == 0 and t_sub >= warm:
                latencies.append(c["total_us"] / 1e3)
                batches.append(c["batch"])
                done_n += 1
    end = time.perf_counter() - t0
    while tag_slot:  # drain what is in flight before the next load
        for c in srv.poll(max_n=4096, timeout_ms=200):
            s_, slot, _ = tag_slot.pop(c["tag"])
            s_["free"].append(slot)
    lat = sorted(latencies)
    pct = lambda q: round(lat[min(len(lat) - 1, int(q * len(lat)))], 3) if lat else None
    return {"offered_frames_per_s": round(rate * len(streams), 1), "served_frames_per_s": round(done_n / (end - warm), 2),
            "p50_ms": pct(0.5), "p99_ms": pct(0.99), "mean_batch": round(float(np.mean(batches)), 2) if batches else None,
            "max_batch": int(max(batches)) if batches else None, "dropped_no_slot": int(dropped)}


def run_serve(args):
    """16 concurrent streams at mixed resolutions through tc_server_*: Poisson frame arrivals
    per stream, host buffers in and out, HBM-budget admission, streams of one size sharing a
    batch (their ready frames run as one step of shared launches, CUDA graphs per lane
    range).  The line reports the load of 30 frames/s per stream and a curve of higher loads
    up to saturation (served frames/s, p50/p99 submit-to-done latency, mean frames per step)."""
    import torch
    import paper_2301_00750_b300 as tc

    tmp = tempfile.mkdtemp(prefix="tcserve")
    path = os.path.join(tmp, "net.tcw")
    write_weights(path)
    srv = tc.Server(path, precision=args.precision, workers=args.workers, batch_lanes=args.batch_lanes,
                    hbm_budget_bytes=int(args.budget_gb * (1 << 30)) if args.budget_gb else 0)
    streams = []
    frames_by_size = {}
    q8 = lambda a: torch.from_numpy(np.ascontiguousarray(np.moveaxis(
        np.floor(np.clip(a, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8), 0, -1))).pin_memory()
    for W, H, count in SERVE_MIX:
        if (W, H) not in frames_by_size:
            fr, st = make_frames(seed=W, n=3, width=W, height=H)
            if args.rgb8:  # 8-bit interleaved RGB frames (the synthetic frames clipped and rounded)
                frames_by_size[(W, H)] = ([q8(f) for f in fr], [q8(p) for p in st])
            else:
                frames_by_size[(W, H)] = ([torch.from_numpy(f).pin_memory() for f in fr],
                                          [torch.from_numpy(p).pin_memory() for p in st])
        for _ in range(count):
            sid = srv.open(W, H)
            srv.set_consistency(sid, k1=0.5)
            if args.rgb8:
                outs = [torch.empty((H, W, 3), dtype=torch.uint8).pin_memory() for _ in range(args.ring)]
            else:
                outs = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(args.ring)]
            streams.append(dict(id=sid, W=W, H=H, outs=outs, n=0, rgb8=args.rgb8))
    base = serve_load(srv, streams, frames_by_size, 30.0, args.seconds, 7)
    curve = [base]
    if not args.skip_curve:
        for k, rate in enumerate((60.0, 120.0, 240.0, 1000.0)):
            curve.append(serve_load(srv, streams, frames_by_size, rate, max(3.0, args.seconds / 2), 8 + k))
    srv.destroy()
    px = sum(W * H * c for W, H, c in SERVE_MIX)
    cap = max(c["served_frames_per_s"] for c in curve)
    print(json.dumps({
        "metric": "serving: aggregate frames/s and p50/p99 frame latency, 16 mixed-resolution streams, Poisson 30 fps",
        "value": base["served_frames_per_s"], "unit": "frames/s", "higher_is_better": True,
        "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"], "mean_batch": base["mean_batch"],
        "offered_frames_per_s": base["offered_frames_per_s"], "dropped_no_slot": base["dropped_no_slot"],
        "capacity_frames_per_s": cap, "load_curve": curve,
        "dtype": {"fp16": "f16", "fp32": "f32"}.get(args.precision, args.precision), "data": "synthetic",
        "workers": args.workers, "batch_lanes": args.batch_lanes,
        "config": {"workload": "4x640x360, 4x1280x720, 6x1920x1080, 2x2560x1440; host buffers in/out per frame "
                               + ("(8-bit interleaved RGB, tc_server_submit_rgb8); " if args.rgb8 else
                                  "(float32 planar); ")
                               + f"{args.ring} output buffers per stream (a frame arriving with none free is skipped)",
                   "megapixels_per_round": round(px / 1e6, 2), "seconds": args.seconds},
    }), flush=True)


TRAIN_BATCH, TRAIN_SIZE, TRAIN_POOL = 32, 256, 4


def train_flops_per_step(spec, batch=TRAIN_BATCH, size=TRAIN_SIZE):
    """Algorithmic FLOPs of one training step's convolutions: the forward (pyramids of 2B
    images, the estimators a -> b for B pairs, heads included), the weight gradient of every
    conv and the data gradient of every conv but the first (same FLOPs as its forward), plus
    the correlation forward and backward (3 x its forward)."""
    L = spec.levels
    fwd = dgrad = corr = 0
    for name, cin, cout, stride, _ in spec.layer_table():
        l = int(name[3])
        if name.startswith("pyr"):
            f = 2 * (2 * batch) * (size >> l) ** 2 * cout * cin * 9
        else:
            f = 2 * batch * (size >> l) ** 2 * cout * cin * 9
        fwd += f
        if name != "pyr1a":
            dgrad += f
    d = (2 * spec.radius + 1) ** 2
    for l in range(2, L + 1):
        corr += 2 * batch * (size >> l) ** 2 * d * spec.chans[l - 1]
    return dict(forward=fwd, wgrad=fwd, dgrad=dgrad, correlation=3 * corr, total=2 * fwd + dgrad + 3 * corr)


def run_train(args):
    """Training throughput (SYS-4): the 5-level net on 256x256 synthetic pairs (|F| <= 16 px,
    0-3 occluding rectangles), batch 32, one AdamW step per batch through tc_trainer_run."""
    import torch
    import paper_2301_00750_b300 as tc  # noqa: F401
    import paper_2301_00750_b300.train as tr

    tmp = tempfile.mkdtemp(prefix="tctrain")
    path = os.path.join(tmp, "net.tcw")
    write_weights(path)
    host = [synth.training_batch(20000 + 1000 * k, TRAIN_BATCH, TRAIN_SIZE, 16.0) for k in range(TRAIN_POOL)]
    dev = [tuple(torch.from_numpy(x).cuda() for x in bt) for bt in host]
    t = tr.Trainer(TRAIN_BATCH, TRAIN_SIZE, TRAIN_SIZE, args.precision if args.precision != "fp8" else "bf16",
                   weights_path=path)
    stream = torch.cuda.current_stream()
    first = t.run(*dev[0], mode="forward", wait=True)
    for k in range(args.warmup):
        t.run(*dev[k % TRAIN_POOL], mode="step")
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        t.run(*dev[k % TRAIN_POOL], mode="step")
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = ev[0].elapsed_time(ev[args.steps])
    per = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps))
    last = t.loss()
    # end to end: pinned host batches copied in and the loss read back every step
    pinned = [tuple(torch.from_numpy(x).pin_memory() for x in bt) for bt in host]
    bufs = tuple(torch.empty_like(x) for x in dev[0])
    n_e2e = max(3, min(args.steps, 30))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        for dst, src in zip(bufs, pinned[k % TRAIN_POOL]):
            dst.copy_(src, non_blocking=True)
        t.run(*bufs, mode="step", wait=True)
    e2e_s = time.perf_counter() - t0
    steps_done = t.steps
    t.destroy()
    flops = train_flops_per_step(net_spec())
    achieved = flops["total"] * args.steps / (total_ms / 1e3) / 1e12
    h2d = sum(x.numel() * 4 for x in dev[0])
    line = {
        "metric": "training throughput, lite flow net 5 levels, 256x256 pairs, batch 32 (pairs/s)",
        "value": round(args.steps * TRAIN_BATCH / (total_ms / 1e3), 2), "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32"}.get(args.precision, "bf16") + " activations, f32 gradients and master weights",
        "data": "synthetic (seeded 256x256 pairs: blurred noise, smooth flow |F| <= 16 px, 0-3 rectangles)",
        "config": {"workload": "train 5-level net 16/32/64/96/128, radius 4, decoder 128/96/64/32/2; multi-scale "
                               "EPE (levels 5..2, equal weights); AdamW lr 1e-4", "batch": TRAIN_BATCH,
                   "size": TRAIN_SIZE, "batches_resident": TRAIN_POOL,
                   "l2": "per-step working set (activations ~4 GB) > 126 MB L2 (no flush needed)"},
        "latency_ms": {"p50": round(per[len(per) // 2], 3), "p99": round(per[min(len(per) - 1, int(0.99 * len(per)))], 3)},
        "loss": {"before": round(first, 4), "after_steps": round(last, 4), "steps": steps_done},
        "roofline": ({"kernel": "whole training step: all convs (forward, data and weight gradients) + correlation",
                      "bound": "tensor", "achieved": round(achieved, 2),
                      "peak": measured_peaks().get("bf16_tflops_sustained"), "unit": "TFLOP/s",
                      "frac": round(achieved / measured_peaks().get("bf16_tflops_sustained"), 4), "traffic": None,
                      "peak_source": "of measured bf16 sustained (MEASURED_PEAKS.json); convs, data and weight "
                                     "gradients run on tcgen05, the rest of the step on the CUDA cores",
                      "gflop_per_step": round(flops["total"] / 1e9, 1)}
                     if args.precision != "fp32" else
                     {"kernel": "whole training step", "bound": "alu", "achieved": round(achieved, 2),
                      "peak": round(FP32_SIMT_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
                      "frac": round(achieved / FP32_SIMT_PEAK_TFLOPS, 4), "traffic": None,
                      "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2032 MHz (FP32 trainer on the CUDA cores)",
                      "gflop_per_step": round(flops["total"] / 1e9, 1)}),
        "clocks": clk,
        "e2e": {"value": round(n_e2e * TRAIN_BATCH / e2e_s, 2), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8},
    }
    print(json.dumps(line), flush=True)


def _kernel_short(name):
    n = name.replace("void ", "").replace("tc::(anonymous namespace)::", "").replace("tc::", "")
    i = n.find(">(")
    return n[: i + 1] if i >= 0 else n.split("(")[0]


def run_timeline(args):
    """Kernel timeline of the 1080p stream (CUPTI through torch.profiler): K frames after the
    warm-up in pipelined and in sequential mode.  Reports per mode the time span per frame,
    the time the GPU had at least one kernel running, the sum of kernel durations (above the
    span when kernels of different frames overlap), each kernel's launches and time per frame,
    and the kernels of one sequential frame in order with their start offsets."""
    import torch
    from torch.profiler import profile, ProfilerActivity
    import paper_2301_00750_b300 as tc

    torch.cuda.set_device(0)
    tmp = tempfile.mkdtemp(prefix="tctl")
    path = os.path.join(tmp, "net.tcw")
    write_weights(path)
    frames, styl = make_frames(seed=0)
    dev_f = [torch.from_numpy(f).cuda() for f in frames]
    dev_s = [torch.from_numpy(p).cuda() for p in styl]
    scales = fp8_scales(tc, path, dev_f, dev_s) if args.precision == "fp8" else None
    H, W = dev_f[0].shape[1:]
    k = max(4, min(args.steps, 24))
    report = {}
    for mode in ("pipelined", "sequential"):
        s = open_stream(tc, path, W, H, args.precision, scales)
        if mode == "pipelined":
            s.set_pipelined(True)
        O = torch.empty((3, H, W), device="cuda")
        wc = torch.empty((H, W), device="cuda")
        m = torch.empty((H, W), device="cuda", dtype=torch.uint8)
        step = 0
        for _ in range(max(args.warmup, 8)):
            s.set_consistency(**consistency_controls(step, 0, 0))
            i = frame_order(step)
            s.process_frame(dev_f[i], dev_s[i], O, wc, m)
            step += 1
        s.synchronize()
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            for _ in range(k):
                s.set_consistency(**consistency_controls(step, 0, 0))
                i = frame_order(step)
                s.process_frame(dev_f[i], dev_s[i], O, wc, m)
                step += 1
            s.synchronize()
            torch.cuda.synchronize()
        s.destroy()
        ev = sorted([(e.time_range.start, e.time_range.end - e.time_range.start, _kernel_short(e.name))
                     for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA
                     and not e.name.startswith("Memcpy") and not e.name.startswith("Memset")])
        t0, t1 = ev[0][0], max(a + d for a, d, _ in ev)
        busy, cs, ce = 0.0, None, None
        for a, d, _ in ev:
            if ce is None or a > ce:
                if ce is not None:
                    busy += ce - cs
                cs, ce = a, a + d
            else:
                ce = max(ce, a + d)
        busy += ce - cs
        agg = {}
        for a, d, n in ev:
            c, t = agg.get(n, (0, 0.0))
            agg[n] = (c + 1, t + d)
        report[mode] = dict(
            us_per_frame=round((t1 - t0) / k, 1), busy_us_per_frame=round(busy / k, 1),
            kernel_us_per_frame=round(sum(d for _, d, _ in ev) / k, 1), launches_per_frame=round(len(ev) / k, 2),
            kernels={n: [round(c / k, 2), round(t / k, 1)] for n, (c, t) in sorted(agg.items(), key=lambda x: -x[1][1])})
        if mode == "sequential":
            per = len(ev) // k
            fr = ev[per * (k // 2): per * (k // 2 + 1)]
            report[mode]["one_frame"] = [[round(a - fr[0][0], 1), round(d, 1), n] for a, d, n in fr]
    for mode, r in report.items():
        print(f"== {mode}: {r['us_per_frame']} us per frame, GPU busy {r['busy_us_per_frame']} us, "
              f"kernel time {r['kernel_us_per_frame']} us, {r['launches_per_frame']} launches per frame")
        for n, (c, t) in r["kernels"].items():
            print(f"   {t:8.1f} us/frame  {c:5.2f}/frame  {n}")
        for a, d, n in r.get("one_frame", []):
            print(f"   one frame: start {a:8.1f}  {d:7.1f} us  {n}")
    print(json.dumps({"timeline": report, "precision": args.precision, "frames": k,
                      "config": workload_config(args)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp8", "fp32"])
    ap.add_argument("--skip-variants", action="store_true",
                    help="skip timing the other 16/8-bit variants and their EPE against FP32")
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-fp8", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-peaks", action="store_true", help="skip measuring the e4m3 and fp32 GEMM peaks")
    ap.add_argument("--skip-solver", action="store_true")
    ap.add_argument("--skip-latency", action="store_true")
    ap.add_argument("--sequential", action="store_true",
                    help="time the headline in the default mode (frames ordered on the caller's stream)")
    ap.add_argument("--skip-fast", action="store_true")
    ap.add_argument("--skip-refine", action="store_true")
    ap.add_argument("--flow-downscale", type=int, default=1, choices=[1, 2],
                    help="time the stream with the flow network on half-size frames (the fast preset's flow)")
    ap.add_argument("--latency", type=int, default=0, choices=[0, 1],
                    help="time the stream with one frame of latency (the next frame in the blend)")
    ap.add_argument("--solver-iters", type=int, default=0,
                    help="run the timed stream with the Eq. 1 / Eq. 8 solver (default: causal O_t = A_t)")
    ap.add_argument("--serve", action="store_true", help="run the multi-stream serving benchmark instead")
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--ring", type=int, default=4, help="output buffers per stream (frames in flight)")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--batch-lanes", type=int, default=4, help="serving: streams of one size per shared batch")
    ap.add_argument("--skip-curve", action="store_true", help="serving: only the 30 frames/s per stream load")
    ap.add_argument("--rgb8", action="store_true", help="serving: submit 8-bit interleaved RGB frames")
    ap.add_argument("--train", action="store_true", help="run the training-throughput benchmark instead")
    ap.add_argument("--timeline", action="store_true",
                    help="record the kernel timeline (CUPTI) of the 1080p stream in pipelined and sequential mode")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve:
        run_serve(args)
    elif args.train:
        run_train(args)
    elif args.timeline:
        run_timeline(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
