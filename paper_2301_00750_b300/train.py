"""Python binding of the training ABI (include/tc_train.h): the native trainer, the stage
backward passes as ``torch.autograd.Function``s, and the brute-force flow.

Argument marshalling only; every forward, backward and update step runs in the library's
CUDA kernels.  Tensors are CUDA float32 and contiguous.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import PRECISION, TcError, _check, _lib, _ptr, _stream_handle, op_conv3x3, op_correlation, \
    op_upsample_flow, op_warp_features

_vp, _i, _f, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t


class TcTrainerDesc(ctypes.Structure):
    _fields_ = [("batch", _i), ("height", _i), ("width", _i), ("precision", _i), ("weights_path", ctypes.c_char_p),
                ("weights_blob", _vp), ("weights_bytes", _sz), ("lr", _f), ("beta1", _f), ("beta2", _f),
                ("eps", _f), ("weight_decay", _f)]


TRAIN_MODES = {"forward": 0, "backward": 1, "step": 2}

_lib.tc_trainer_default_desc.argtypes = [ctypes.POINTER(TcTrainerDesc)]
_lib.tc_trainer_default_desc.restype = None
_lib.tc_trainer_create.argtypes = [ctypes.POINTER(TcTrainerDesc), _vp, ctypes.POINTER(_vp)]
_lib.tc_trainer_run.argtypes = [_vp, _vp, _vp, _vp, _i, ctypes.POINTER(ctypes.c_double)]
_lib.tc_trainer_loss.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
_lib.tc_trainer_num_params.argtypes = [_vp]
_lib.tc_trainer_num_params.restype = _sz
for _n in ("tc_trainer_get_params", "tc_trainer_get_grads", "tc_trainer_set_params"):
    getattr(_lib, _n).argtypes = [_vp, ctypes.POINTER(_f), _sz]
_lib.tc_trainer_level_flow.argtypes = [_vp, _i, _vp]
_lib.tc_trainer_steps.argtypes = [_vp]
_lib.tc_trainer_steps.restype = ctypes.c_longlong
for _n in ("tc_trainer_save", "tc_trainer_load", "tc_trainer_export_weights"):
    getattr(_lib, _n).argtypes = [_vp, ctypes.c_char_p]
_lib.tc_trainer_last_error.argtypes = [_vp]
_lib.tc_trainer_last_error.restype = ctypes.c_char_p
_lib.tc_trainer_destroy.argtypes = [_vp]
_lib.tc_op_conv3x3_backward.argtypes = [_vp, _i, _i, _i, _i, _vp, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.tc_op_correlation_backward.argtypes = [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp]
_lib.tc_op_warp_features_backward.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp]
_lib.tc_op_upsample_flow_backward.argtypes = [_vp, _i, _i, _i, _i, _vp, _vp]
_lib.tc_op_bruteforce_flow.argtypes = [_vp, _vp, _i, _i, _i, _i, _vp, _vp]
for _n in ("tc_trainer_create", "tc_trainer_run", "tc_trainer_loss", "tc_trainer_get_params", "tc_trainer_get_grads",
           "tc_trainer_set_params", "tc_trainer_level_flow", "tc_trainer_save", "tc_trainer_load",
           "tc_trainer_export_weights", "tc_trainer_destroy", "tc_op_conv3x3_backward", "tc_op_correlation_backward",
           "tc_op_warp_features_backward", "tc_op_upsample_flow_backward", "tc_op_bruteforce_flow"):
    getattr(_lib, _n).restype = ctypes.c_int


def _tcheck(status, h):
    if status != 0:
        raise TcError(status, (_lib.tc_trainer_last_error(h) or b"").decode())


def default_hparams() -> dict:
    d = TcTrainerDesc()
    _lib.tc_trainer_default_desc(ctypes.byref(d))
    return dict(lr=d.lr, beta1=d.beta1, beta2=d.beta2, eps=d.eps, weight_decay=d.weight_decay)


class Trainer:
    """tc_trainer_*: multi-scale EPE training of the lite flow network on pairs (a, b) with
    ground-truth flow F_{a->b}."""

    def __init__(self, batch, height, width, precision="bf16", weights_path=None, weights_blob=None,
                 cuda_stream=None, **hparams):
        d = TcTrainerDesc()
        _lib.tc_trainer_default_desc(ctypes.byref(d))
        d.batch, d.height, d.width = int(batch), int(height), int(width)
        d.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self._blob = None
        if weights_path is not None:
            d.weights_path = os.fsencode(weights_path)
        elif weights_blob is not None:
            self._blob = ctypes.create_string_buffer(bytes(weights_blob), len(weights_blob))
            d.weights_blob = ctypes.cast(self._blob, ctypes.c_void_p)
            d.weights_bytes = len(weights_blob)
        for k, v in hparams.items():
            setattr(d, k, float(v))
        h = _vp()
        self.cuda_stream = _stream_handle(cuda_stream)
        _check(_lib.tc_trainer_create(ctypes.byref(d), self.cuda_stream, ctypes.byref(h)))
        self._h = h
        self.batch, self.height, self.width = d.batch, d.height, d.width

    def run(self, Ia, Ib, flow, mode="step", wait=False):
        """One forward(+backward(+AdamW)) over device (B,3,H,W), (B,3,H,W), (B,2,H,W) float32
        tensors.  Returns the loss if wait, else None (read it with .loss())."""
        out = ctypes.c_double()
        _tcheck(_lib.tc_trainer_run(self._h, _ptr(Ia, torch.float32, "I_a"), _ptr(Ib, torch.float32, "I_b"),
                                    _ptr(flow, torch.float32, "flow"), TRAIN_MODES[mode],
                                    ctypes.byref(out) if wait else None), self._h)
        return out.value if wait else None

    def loss(self) -> float:
        out = ctypes.c_double()
        _tcheck(_lib.tc_trainer_loss(self._h, ctypes.byref(out)), self._h)
        return out.value

    @property
    def num_params(self) -> int:
        return int(_lib.tc_trainer_num_params(self._h))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.num_params, np.float32)
        _tcheck(_lib.tc_trainer_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(_f)), a.size), self._h)
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(self.num_params, np.float32)
        _tcheck(_lib.tc_trainer_get_grads(self._h, a.ctypes.data_as(ctypes.POINTER(_f)), a.size), self._h)
        return a

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        _tcheck(_lib.tc_trainer_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(_f)), a.size), self._h)

    def level_flow(self, level):
        out = torch.empty((self.batch, self.height >> level, self.width >> level, 2), device="cuda")
        _tcheck(_lib.tc_trainer_level_flow(self._h, int(level), out.data_ptr()), self._h)
        return out

    @property
    def steps(self) -> int:
        return int(_lib.tc_trainer_steps(self._h))

    def save(self, path):
        _tcheck(_lib.tc_trainer_save(self._h, os.fsencode(path)), self._h)

    def load(self, path):
        _tcheck(_lib.tc_trainer_load(self._h, os.fsencode(path)), self._h)

    def export_weights(self, path):
        _tcheck(_lib.tc_trainer_export_weights(self._h, os.fsencode(path)), self._h)

    def destroy(self):
        if getattr(self, "_h", None):
            _lib.tc_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------ autograd functions

class Conv3x3(torch.autograd.Function):
    """3x3 conv (pad 1) + bias + optional LeakyReLU(0.1) on NHWC float32 CUDA tensors:
    forward tc_op_conv3x3, backward tc_op_conv3x3_backward."""

    @staticmethod
    def forward(ctx, x, w, b, stride=1, leaky=True):
        y = op_conv3x3(x.contiguous(), w.detach().cpu().numpy(), b.detach().cpu().numpy(), stride=stride,
                       leaky=leaky, precision="fp32")
        ctx.save_for_backward(x, w, y)
        ctx.stride, ctx.leaky = stride, leaky
        return y

    @staticmethod
    def backward(ctx, dy):
        x, w, y = ctx.saved_tensors
        n, h, wd, cin = x.shape
        cout = w.shape[0]
        dx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        dw = torch.empty_like(w, device=x.device)
        db = torch.empty((cout,), device=x.device)
        wdev = w.detach().to(x.device).contiguous()
        _check(_lib.tc_op_conv3x3_backward(x.data_ptr(), n, h, wd, cin, wdev.data_ptr(), cout, ctx.stride,
                                           int(ctx.leaky), y.data_ptr(), dy.contiguous().data_ptr(),
                                           dx.data_ptr() if dx is not None else None, dw.data_ptr(), db.data_ptr(),
                                           _stream_handle(None)))
        return dx, dw.to(w.device), db.to(w.device), None, None


class Correlation(torch.autograd.Function):
    """Cost volume (mean over channels, LeakyReLU) of NHWC float32 features."""

    @staticmethod
    def forward(ctx, f1, f2, r):
        cost = op_correlation(f1.contiguous(), f2.contiguous(), r, precision="fp32")
        ctx.save_for_backward(f1, f2, cost)
        ctx.r = r
        return cost

    @staticmethod
    def backward(ctx, dcost):
        f1, f2, cost = ctx.saved_tensors
        n, h, w, c = f1.shape
        df1, df2 = torch.empty_like(f1), torch.empty_like(f2)
        _check(_lib.tc_op_correlation_backward(f1.data_ptr(), f2.data_ptr(), n, h, w, c, ctx.r, cost.data_ptr(),
                                               dcost.contiguous().data_ptr(), df1.data_ptr(), df2.data_ptr(),
                                               _stream_handle(None)))
        return df1, df2, None


class WarpFeatures(torch.autograd.Function):
    """Bilinear backward warp of NHWC float32 features by a (n, h, w, 2) flow, zeros off the map."""

    @staticmethod
    def forward(ctx, f, flow):
        out = op_warp_features(f.contiguous(), flow.contiguous(), precision="fp32")
        ctx.save_for_backward(f, flow)
        return out

    @staticmethod
    def backward(ctx, dout):
        f, flow = ctx.saved_tensors
        n, h, w, c = f.shape
        df, dflow = torch.empty_like(f), torch.empty_like(flow)
        _check(_lib.tc_op_warp_features_backward(f.data_ptr(), flow.data_ptr(), n, h, w, c,
                                                 dout.contiguous().data_ptr(), df.data_ptr(), dflow.data_ptr(),
                                                 _stream_handle(None)))
        return df, dflow


class UpsampleFlow(torch.autograd.Function):
    """Bilinear flow upsampling by s (values times s) of a (n, h, w, 2) float32 flow."""

    @staticmethod
    def forward(ctx, flow, s):
        ctx.shape, ctx.s = flow.shape, s
        return op_upsample_flow(flow.contiguous(), s)

    @staticmethod
    def backward(ctx, dfine):
        n, h, w, _ = ctx.shape
        dc = torch.empty((n, h, w, 2), device=dfine.device)
        _check(_lib.tc_op_upsample_flow_backward(dfine.contiguous().data_ptr(), n, h, w, ctx.s, dc.data_ptr(),
                                                 _stream_handle(None)))
        return dc, None


def bruteforce_flow(a, b, r, cuda_stream=None):
    """Integer SSD-argmin displacement index per pixel of device planar (c, h, w) float32
    images a, b (tc_op_bruteforce_flow); returns (h, w) int32 on the device."""
    c, h, w = a.shape
    k = torch.empty((h, w), dtype=torch.int32, device=a.device)
    _check(_lib.tc_op_bruteforce_flow(_ptr(a, torch.float32, "a"), _ptr(b, torch.float32, "b"), c, h, w, int(r),
                                      k.data_ptr(), _stream_handle(cuda_stream)))
    return k


def index_to_flow(k, r):
    """(h, w) displacement indices -> (2, h, w) integer flow (u = dx, v = dy)."""
    n1 = 2 * r + 1
    return torch.stack([(k % n1) - r, (k // n1) - r]).to(torch.float32)
