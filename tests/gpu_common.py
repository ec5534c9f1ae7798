"""Helpers shared by the GPU test files (inputs come from synth, expectations from oracle)."""
import os
import tempfile

import numpy as np

import oracle
import synth

_CACHE = {}


def weights_file(chans=(16, 32, 48), radius=3, seed=0, head_gain=1.0, refine=False):
    """Writes (once per process) the seeded He-init weight file; returns (path, oracle net).
    refine: add the depthwise-separable refinement network (TCW2 file)."""
    key = (tuple(chans), radius, seed, head_gain, refine)
    if key not in _CACHE:
        spec = synth.NetSpec(chans=tuple(chans), radius=radius)
        if refine:
            spec.refine, spec.refine_dil = synth.REFINE_CHANS, synth.REFINE_DIL
        layers = synth.he_weights(spec, seed=seed, head_gain=head_gain)
        d = tempfile.mkdtemp(prefix="tcw")
        path = os.path.join(d, "net.tcw")
        synth.write_weights(path, spec, layers)
        _CACHE[key] = (path, oracle.net_from_layers(spec.levels, spec.radius, spec.chans, spec.decoder, layers))
    return _CACHE[key]


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()


def planar_to_hw2(flow):
    """(2, h, w) -> (h, w, 2) float32."""
    return np.ascontiguousarray(np.moveaxis(np.asarray(flow, np.float32), 0, -1))


def nchw_to_nhwc(a):
    return np.ascontiguousarray(np.moveaxis(np.asarray(a), 1, -1), np.float32)


def nhwc_to_nchw(a):
    return np.ascontiguousarray(np.moveaxis(np.asarray(a), -1, 1))


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def f16_round(a):
    """Round float32 values to the nearest IEEE half (ties to even, subnormals kept), as
    float32."""
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float32)


def round16(prec, a):
    """The operand values of a 16-bit precision ("bf16" or "fp16"); float32 unchanged."""
    return bf16_round(a) if prec == "bf16" else f16_round(a) if prec == "fp16" else np.asarray(a, np.float32)


# Relative step of a 16-bit precision's stored values (8 significant bits for bfloat16,
# 11 for half): outputs rounded to it differ from float32 by at most half of it.
REL16 = {"bf16": 2.0 ** -8, "fp16": 2.0 ** -10}


def weight_scales_e4m3(w):
    """Per-output-channel E4M3 weight scales amax / 448 computed in float32, as a layer's
    planning does (w: (cout, cin, 3, 3) float32)."""
    a = np.abs(np.asarray(w, np.float32)).reshape(w.shape[0], -1).max(1)
    return np.where(a > 0, a / np.float32(448), np.float32(1)).astype(np.float32)


# Canary padding (the stand-in for a memory checker): an output buffer with guard elements
# on both sides, all set to a marker no kernel writes (a NaN with payload 0xDEAD for float32,
# 0xA5 for bytes).  After a call the guards must be intact (no out-of-bounds write) and the
# output region free of markers (every element written).
CANARY = 4096
_MARK = {"float32": 0x7FC0DEAD, "uint8": 0xA5}


def guarded(shape, dtype="float32"):
    """(buffer, view): a CUDA buffer of CANARY + prod(shape) + CANARY elements, all set to the
    marker, and the contiguous view of the middle (16 KiB-aligned for float32)."""
    import torch
    n = int(np.prod(shape))
    tdt = {"float32": torch.float32, "uint8": torch.uint8}[dtype]
    buf = torch.empty(2 * CANARY + n, dtype=tdt, device="cuda")
    if dtype == "float32":
        buf.view(torch.int32).fill_(_MARK[dtype])
    else:
        buf.fill_(_MARK[dtype])
    return buf, buf[CANARY:CANARY + n].view(*shape)


def check_guarded(buf, shape, dtype="float32", written=True):
    """Asserts the guards are intact and, with written, that no marker is left inside."""
    import torch
    n = int(np.prod(shape))
    raw = buf.view(torch.int32) if dtype == "float32" else buf
    m = _MARK[dtype]
    a = raw.cpu().numpy()
    if dtype == "float32":
        a = a.view(np.uint32)
        m = np.uint32(m)
    assert (a[:CANARY] == m).all(), "write before the output buffer"
    assert (a[CANARY + n:] == m).all(), "write past the output buffer"
    if written:
        assert not (a[CANARY:CANARY + n] == m).any(), "output elements left unwritten"
