"""Python binding of libtcstream (the C ABI in include/tc_stream.h).

Argument marshalling only: every stage of the hot path runs in the library's CUDA kernels.
PyTorch is used for device memory and streams; tensors are passed as raw pointers.  If
the compiled library is missing this module raises on import -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtcstream.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2301_00750_b300/build.py` "
                      "(or __graft_entry__.build()); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

TC_OK, TC_ERR_INVALID_ARG, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_BUSY, TC_ERR_TIMEOUT, TC_ERR_STATE, TC_ERR_IO, \
    TC_ERR_UNSUPPORTED = range(9)
_STATUS = ["TC_OK", "TC_ERR_INVALID_ARG", "TC_ERR_OOM", "TC_ERR_CUDA", "TC_ERR_BUSY", "TC_ERR_TIMEOUT",
           "TC_ERR_STATE", "TC_ERR_IO", "TC_ERR_UNSUPPORTED"]
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2, "fp16": 3}

EXPORTED = ["tc_default_consistency", "tc_create_stream", "tc_set_consistency", "tc_process_frame",
            "tc_process_frame_host", "tc_get_flows", "tc_destroy", "tc_last_error", "tc_last_launch_count",
            "tc_op_conv3x3", "tc_op_correlation", "tc_op_warp_features", "tc_op_upsample_flow",
            "tc_op_consistency", "tc_set_profiling", "tc_get_profile", "tc_synchronize", "tc_tensor_core_layers",
            "tc_op_last_used_tensor_cores", "tc_op_correlation_bf16_noalloc",
            "tc_tensor_core_correlation_levels", "tc_set_graphs", "tc_activation_segments",
            "tc_set_amax_recording", "tc_get_amax", "tc_set_fp8_scales", "tc_op_poisson_solve", "tc_set_latency",
            "tc_flush", "tc_last_output_frame", "tc_op_consistency_next", "tc_op_downscale2", "tc_op_sepconv",
            "tc_process_frame_host_async", "tc_set_pipelined", "tc_join", "tc_fp8_scales_from_amax",
            "tc_test_stall_next_convs", "tc_test_fail_device_allocation", "tc_create_batch", "tc_process_lanes",
            "tc_set_lane_consistency", "tc_reset_lane", "tc_get_lane_flows", "tc_set_frame_timing",
            "tc_get_frame_times", "tc_process_frame_host_rgb8_async"]
NOALLOC_SCRATCH_BYTES = 16 << 20
PROFILE_CATEGORIES = ["pyramid_conv", "estimator_conv", "head", "correlation", "warp", "upsample", "consistency",
                      "other", "solver", "refine"]


class TcConsistency(ctypes.Structure):
    _fields_ = [("k1", ctypes.c_float), ("k2", ctypes.c_float), ("alpha", ctypes.c_float),
                ("lambda_", ctypes.c_float), ("fb_check", ctypes.c_int), ("fb_c1", ctypes.c_float),
                ("fb_c2", ctypes.c_float), ("solver_iters", ctypes.c_int), ("eta", ctypes.c_float),
                ("kappa", ctypes.c_float)]


class TcStreamDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("precision", ctypes.c_int),
                ("weights_path", ctypes.c_char_p), ("weights_blob", ctypes.c_void_p),
                ("weights_bytes", ctypes.c_size_t), ("flow_downscale", ctypes.c_int)]


_vp, _i, _f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
_lib.tc_default_consistency.argtypes = [ctypes.POINTER(TcConsistency)]
_lib.tc_default_consistency.restype = None
_lib.tc_create_stream.argtypes = [ctypes.POINTER(TcStreamDesc), _vp, ctypes.POINTER(_vp)]
_lib.tc_set_consistency.argtypes = [_vp, ctypes.POINTER(TcConsistency)]
_lib.tc_process_frame.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.tc_process_frame_host.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.tc_process_frame_host_async.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.tc_process_frame_host_rgb8_async.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.tc_set_pipelined.argtypes = [_vp, _i]
_lib.tc_join.argtypes = [_vp]
_lib.tc_get_flows.argtypes = [_vp, _vp, _vp]
_lib.tc_destroy.argtypes = [_vp]
_lib.tc_last_error.argtypes = [_vp]
_lib.tc_last_error.restype = ctypes.c_char_p
_lib.tc_last_launch_count.argtypes = [_vp]
_lib.tc_op_conv3x3.argtypes = [_i, _vp, _i, _i, _i, _i, _vp, _vp, _i, _i, _i, _vp, _vp]
_lib.tc_op_correlation.argtypes = [_i, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp]
_lib.tc_op_warp_features.argtypes = [_i, _vp, _vp, _i, _i, _i, _i, _vp, _vp]
_lib.tc_op_upsample_flow.argtypes = [_vp, _i, _i, _i, _i, _vp, _vp]
_lib.tc_op_consistency.argtypes = [_vp] * 7 + [_i] * 5 + [ctypes.POINTER(TcConsistency), _vp, _vp, _vp, _vp]
_lib.tc_set_profiling.argtypes = [_vp, _i]
_lib.tc_set_graphs.argtypes = [_vp, _i]
_lib.tc_op_correlation_bf16_noalloc.argtypes = [_vp, _vp, _i, _i, _i, _i, _i, _vp, _vp]
_lib.tc_synchronize.argtypes = [_vp]
_lib.tc_op_poisson_solve.argtypes = [_vp, _vp, _vp, _i, _i, _i, _i, _f, _f, _vp, _vp]
_lib.tc_op_poisson_solve.restype = ctypes.c_int
_lib.tc_tensor_core_layers.argtypes = [_vp]
_lib.tc_tensor_core_correlation_levels.argtypes = [_vp]
_lib.tc_op_last_used_tensor_cores.argtypes = []
_lib.tc_activation_segments.argtypes = [_vp]
_lib.tc_set_amax_recording.argtypes = [_vp, _i]
_lib.tc_get_amax.argtypes = [_vp, ctypes.POINTER(_f), _i]
_lib.tc_set_fp8_scales.argtypes = [_vp, ctypes.POINTER(_f), _i]
_lib.tc_fp8_scales_from_amax.argtypes = [ctypes.POINTER(_f), _i, _f, ctypes.POINTER(_f)]
_lib.tc_set_frame_timing.argtypes = [_vp, _i]
_lib.tc_get_frame_times.argtypes = [_vp, ctypes.POINTER(_f), _i, ctypes.POINTER(_i)]
_lib.tc_set_frame_timing.restype = ctypes.c_int
_lib.tc_get_frame_times.restype = ctypes.c_int
_lib.tc_create_batch.argtypes = [ctypes.POINTER(TcStreamDesc), _i, _vp, ctypes.POINTER(_vp)]
_lib.tc_process_lanes.argtypes = [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                  ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]
_lib.tc_set_lane_consistency.argtypes = [_vp, _i, ctypes.POINTER(TcConsistency)]
_lib.tc_reset_lane.argtypes = [_vp, _i]
_lib.tc_get_lane_flows.argtypes = [_vp, _i, _vp, _vp]
for _n in ("tc_create_batch", "tc_process_lanes", "tc_set_lane_consistency", "tc_reset_lane", "tc_get_lane_flows"):
    getattr(_lib, _n).restype = ctypes.c_int
_lib.tc_test_stall_next_convs.argtypes = [_i]
_lib.tc_test_stall_next_convs.restype = None
_lib.tc_test_fail_device_allocation.argtypes = [ctypes.c_longlong]
_lib.tc_test_fail_device_allocation.restype = None
_lib.tc_get_profile.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), _i]
_lib.tc_set_latency.argtypes = [_vp, _i]
_lib.tc_op_downscale2.argtypes = [_vp, _i, _i, _i, _vp, _vp]
_lib.tc_op_sepconv.argtypes = [_i, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp]
_lib.tc_flush.argtypes = [_vp, _vp, _vp, _vp]
_lib.tc_last_output_frame.argtypes = [_vp]
_lib.tc_last_output_frame.restype = ctypes.c_longlong
_lib.tc_op_consistency_next.argtypes = [_vp] * 11 + [_i] * 5 + [ctypes.POINTER(TcConsistency), _vp, _vp, _vp, _vp]
for _n in ["tc_set_amax_recording", "tc_get_amax", "tc_set_fp8_scales", "tc_fp8_scales_from_amax", "tc_set_graphs", "tc_op_correlation_bf16_noalloc", "tc_synchronize", "tc_set_profiling", "tc_get_profile", "tc_create_stream", "tc_set_consistency", "tc_process_frame", "tc_process_frame_host", "tc_get_flows",
           "tc_process_frame_host_async", "tc_process_frame_host_rgb8_async", "tc_set_pipelined", "tc_join", "tc_destroy", "tc_op_conv3x3", "tc_op_correlation", "tc_op_warp_features", "tc_op_upsample_flow",
           "tc_op_consistency", "tc_set_latency", "tc_flush", "tc_op_consistency_next", "tc_op_downscale2",
           "tc_op_sepconv"]:
    getattr(_lib, _n).restype = ctypes.c_int


class TcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS[status] if 0 <= status < len(_STATUS) else status}: {msg}")
        self.status = status


def _check(status, handle=None):
    if status != TC_OK:
        raise TcError(status, (_lib.tc_last_error(handle) or b"").decode())


def _hbuf(a, dt):
    """Host address of a contiguous NumPy array or CPU torch tensor (or None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if a.dtype != dt or not a.flags.c_contiguous:
        raise TypeError("host buffers must be contiguous " + str(dt))
    return a.ctypes.data


def _ptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream_handle(cuda_stream):
    if cuda_stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        return torch.cuda.current_stream().cuda_stream
    return getattr(cuda_stream, "cuda_stream", cuda_stream)


def default_consistency() -> dict:
    c = TcConsistency()
    _lib.tc_default_consistency(ctypes.byref(c))
    return dict(k1=c.k1, k2=c.k2, alpha=c.alpha, lam=c.lambda_, fb_check=bool(c.fb_check), fb_c1=c.fb_c1,
                fb_c2=c.fb_c2)


def _consistency_struct(**kw) -> TcConsistency:
    c = TcConsistency()
    _lib.tc_default_consistency(ctypes.byref(c))
    for k, v in kw.items():
        if k == "lam":
            c.lambda_ = v
        elif k == "fb_check":
            c.fb_check = int(bool(v))
        else:
            setattr(c, k, v)
    return c


class Stream:
    """One video stream: tc_create_stream / tc_set_consistency / tc_process_frame / tc_destroy."""

    def __init__(self, width, height, precision="fp32", weights_path=None, weights_blob=None, cuda_stream=None,
                 flow_downscale=1):
        """flow_downscale = 2 runs the flow network on 2x2-mean half-size frames (with
        set_consistency(solver_iters=50): the paper's fast preset)."""
        desc = TcStreamDesc()
        desc.width, desc.height = int(width), int(height)
        desc.flow_downscale = int(flow_downscale)
        desc.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self._blob = None
        if weights_path is not None:
            desc.weights_path = os.fsencode(weights_path)
        elif weights_blob is not None:
            self._blob = ctypes.create_string_buffer(bytes(weights_blob), len(weights_blob))
            desc.weights_blob = ctypes.cast(self._blob, ctypes.c_void_p)
            desc.weights_bytes = len(weights_blob)
        h = _vp()
        self.cuda_stream = _stream_handle(cuda_stream)
        _check(_lib.tc_create_stream(ctypes.byref(desc), self.cuda_stream, ctypes.byref(h)))
        self._h = h
        self.width, self.height = int(width), int(height)

    def set_consistency(self, **kw):
        c = _consistency_struct(**kw)
        _check(_lib.tc_set_consistency(self._h, ctypes.byref(c)), self._h)

    def process_frame(self, I, P, O, wc=None, mask=None):
        import torch
        _check(_lib.tc_process_frame(self._h, _ptr(I, torch.float32, "I_t"), _ptr(P, torch.float32, "P_t"),
                                     _ptr(O, torch.float32, "O_t"), _ptr(wc, torch.float32, "wc"),
                                     _ptr(mask, torch.uint8, "mask")), self._h)

    def process_frame_host(self, I, P, O, wc=None, mask=None):
        """Host buffers (NumPy or CPU torch tensors, contiguous float32 / uint8)."""
        _check(_lib.tc_process_frame_host(self._h, _hbuf(I, np.float32), _hbuf(P, np.float32),
                                          _hbuf(O, np.float32), _hbuf(wc, np.float32), _hbuf(mask, np.uint8)),
               self._h)

    def process_frame_host_async(self, I, P, O, wc=None, mask=None):
        """Pipelined host-buffer call: enqueues the upload, the frame and the download and
        returns; the buffers (page-locked for the copies to overlap) must stay alive and
        untouched until synchronize()."""
        _check(_lib.tc_process_frame_host_async(self._h, _hbuf(I, np.float32), _hbuf(P, np.float32),
                                                _hbuf(O, np.float32), _hbuf(wc, np.float32),
                                                _hbuf(mask, np.uint8)), self._h)

    def process_frame_host_rgb8_async(self, I, P, O, wc=None, mask=None):
        """As process_frame_host_async for 8-bit frames: I, P, O host (H, W, 3) uint8
        interleaved RGB (code q = value q / 255; O quantised as floor(255 clamp(O, 0, 1) + 0.5)).
        The buffers (page-locked for the copies to overlap) must stay alive and untouched
        until synchronize()."""
        _check(_lib.tc_process_frame_host_rgb8_async(self._h, _hbuf(I, np.uint8), _hbuf(P, np.uint8),
                                                     _hbuf(O, np.uint8), _hbuf(wc, np.float32),
                                                     _hbuf(mask, np.uint8)), self._h)

    def set_pipelined(self, enable: bool):
        """Pipelined mode: frames are enqueued on the library's own streams with frame t + 1's
        pyramid overlapping the flow estimation of frames t and t - 1 (two estimator buffer
        sets); inputs must be valid at the call and
        stay unmodified, outputs are valid after join() or synchronize().  The asynchronous
        host-buffer calls work in this mode too.  Only before the first frame of a sequence."""
        _check(_lib.tc_set_pipelined(self._h, int(bool(enable))), self._h)

    def join(self):
        """Pipelined mode: the caller's CUDA stream waits for every frame given so far."""
        _check(_lib.tc_join(self._h), self._h)

    def set_latency(self, frames: int):
        """1: each process_frame with frame t+1 returns frame t blended with both neighbours
        (w_n, clamp k2); 0: the causal path.  Only before the first frame of a sequence."""
        _check(_lib.tc_set_latency(self._h, int(frames)), self._h)

    def flush(self, O, wc=None, mask=None):
        """One frame of latency: the last frame's outputs; ends the sequence."""
        import torch
        _check(_lib.tc_flush(self._h, _ptr(O, torch.float32, "O_t"), _ptr(wc, torch.float32, "wc"),
                             _ptr(mask, torch.uint8, "mask")), self._h)

    @property
    def last_output_frame(self) -> int:
        """Index in its sequence of the frame the last call wrote (-1: none)."""
        return int(_lib.tc_last_output_frame(self._h))

    def get_flows(self, Fb=None, Ff=None):
        import torch
        _check(_lib.tc_get_flows(self._h, _ptr(Fb, torch.float32, "Fb"), _ptr(Ff, torch.float32, "Ff")), self._h)

    def set_frame_timing(self, enable: bool):
        """Pipelined mode: record every frame's device latency (pyramid may start -> blend done)."""
        _check(_lib.tc_set_frame_timing(self._h, int(bool(enable))), self._h)

    def get_frame_times(self, n=100000) -> np.ndarray:
        """The recorded per-frame latencies in milliseconds (waits for the last frame)."""
        buf = (_f * n)()
        cnt = _i()
        _check(_lib.tc_get_frame_times(self._h, buf, n, ctypes.byref(cnt)), self._h)
        return np.array(buf[:min(n, cnt.value)], np.float32)

    def set_graphs(self, enable: bool):
        """Replay each frame as one CUDA graph launch (default) or launch kernel by kernel."""
        _check(_lib.tc_set_graphs(self._h, int(bool(enable))), self._h)

    def set_profiling(self, enable: bool):
        _check(_lib.tc_set_profiling(self._h, int(bool(enable))), self._h)

    def get_profile(self) -> dict:
        """{category: (milliseconds, launches)} since the last set_profiling."""
        n = len(PROFILE_CATEGORIES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _check(_lib.tc_get_profile(self._h, ms, cnt, n), self._h)
        return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_CATEGORIES)}

    def synchronize(self):
        """Waits for the stream; raises TcError(TC_ERR_TIMEOUT) if a device-side wait gave up."""
        _check(_lib.tc_synchronize(self._h), self._h)

    @property
    def activation_segments(self) -> int:
        return _lib.tc_activation_segments(self._h)

    def set_amax_recording(self, enable: bool):
        """FP32/BF16/FP16 streams: record the largest |activation| of every segment from now on."""
        _check(_lib.tc_set_amax_recording(self._h, int(bool(enable))), self._h)

    def get_amax(self) -> np.ndarray:
        n = self.activation_segments
        a = (_f * n)()
        _check(_lib.tc_get_amax(self._h, a, n), self._h)
        return np.array(a[:], np.float32)

    def set_fp8_scales(self, scales):
        """E4M3 streams: one scale per activation segment (x is stored as e4m3(x / scale))."""
        sc = np.ascontiguousarray(scales, np.float32)
        _check(_lib.tc_set_fp8_scales(self._h, sc.ctypes.data_as(ctypes.POINTER(_f)), int(sc.size)), self._h)

    @property
    def tensor_core_layers(self) -> int:
        return _lib.tc_tensor_core_layers(self._h)

    @property
    def tensor_core_correlation_levels(self) -> int:
        return _lib.tc_tensor_core_correlation_levels(self._h)

    @property
    def launch_count(self) -> int:
        return _lib.tc_last_launch_count(self._h)

    def destroy(self):
        if getattr(self, "_h", None):
            _check(_lib.tc_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def inject_stall_next_convs(count):
    """tc_test_stall_next_convs (failure injection for tests of the timeout path)."""
    _lib.tc_test_stall_next_convs(int(count))


def inject_device_allocation_failure(nth):
    """tc_test_fail_device_allocation (failure injection for tests of the OOM path)."""
    _lib.tc_test_fail_device_allocation(int(nth))


def fp8_scales_from_amax(amax, margin=1.0):
    """tc_fp8_scales_from_amax: the static E4M3 activation scales of a calibration record."""
    a = np.ascontiguousarray(amax, np.float32)
    out = np.empty_like(a)
    _check(_lib.tc_fp8_scales_from_amax(a.ctypes.data_as(ctypes.POINTER(_f)), int(a.size), float(margin),
                                        out.ctypes.data_as(ctypes.POINTER(_f))))
    return out


class Batch(Stream):
    """tc_create_batch: `lanes` independent causal streams of one size whose pyramids and
    flow estimations run in shared launches; process() takes one frame for each of several
    lanes.  The single-stream calls of Stream answer TC_ERR_STATE on a batch."""

    def __init__(self, width, height, lanes, precision="fp16", weights_path=None, weights_blob=None,
                 cuda_stream=None):
        desc = TcStreamDesc()
        desc.width, desc.height = int(width), int(height)
        desc.flow_downscale = 1
        desc.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self._blob = None
        if weights_path is not None:
            desc.weights_path = os.fsencode(weights_path)
        elif weights_blob is not None:
            self._blob = ctypes.create_string_buffer(bytes(weights_blob), len(weights_blob))
            desc.weights_blob = ctypes.cast(self._blob, ctypes.c_void_p)
            desc.weights_bytes = len(weights_blob)
        h = _vp()
        self.cuda_stream = _stream_handle(cuda_stream)
        _check(_lib.tc_create_batch(ctypes.byref(desc), int(lanes), self.cuda_stream, ctypes.byref(h)))
        self._h = h
        self.width, self.height, self.lanes = int(width), int(height), int(lanes)

    def process(self, lanes, I, P, O, wc=None, mask=None):
        """One frame for each lane in `lanes`: lists of CUDA (3, H, W) float32 tensors I, P, O
        (and optional (H, W) float32 wc, uint8 mask lists) in the order of `lanes`."""
        import torch
        n = len(lanes)
        ln = (_i * n)(*[int(x) for x in lanes])
        arr = lambda xs, dt, nm: (_vp * n)(*[_ptr(x, dt, nm) for x in xs]) if xs is not None else None
        _check(_lib.tc_process_lanes(self._h, n, ln, arr(I, torch.float32, "I_t"), arr(P, torch.float32, "P_t"),
                                     arr(O, torch.float32, "O_t"), arr(wc, torch.float32, "wc"),
                                     arr(mask, torch.uint8, "mask")), self._h)

    def set_lane_consistency(self, lane, **kw):
        c = _consistency_struct(**kw)
        _check(_lib.tc_set_lane_consistency(self._h, int(lane), ctypes.byref(c)), self._h)

    def reset_lane(self, lane):
        _check(_lib.tc_reset_lane(self._h, int(lane)), self._h)

    def get_lane_flows(self, lane, Fb=None, Ff=None):
        import torch
        _check(_lib.tc_get_lane_flows(self._h, int(lane), _ptr(Fb, torch.float32, "Fb"), _ptr(Ff, torch.float32, "Ff")),
               self._h)


def calibrate_fp8(width, height, frames, weights_path=None, weights_blob=None, margin=1.0, flow_downscale=1):
    """E4M3 scales from a BF16 pass: runs `frames` (a list of (I, P) CUDA (3, H, W) float32
    pairs) through a BF16 stream recording the amax of every activation segment, and returns
    the scales tc_fp8_scales_from_amax derives from that record (what tc_set_fp8_scales
    takes)."""
    import torch
    s = Stream(width, height, "bf16", weights_path=weights_path, weights_blob=weights_blob,
               flow_downscale=flow_downscale)
    try:
        s.set_amax_recording(True)
        out = torch.empty((3, height, width), device="cuda", dtype=torch.float32)
        for I, P in frames:
            s.process_frame(I, P, out)
        amax = s.get_amax()
    finally:
        s.destroy()
    return fp8_scales_from_amax(amax, margin)


# ----------------------------------------------------------------------------- stage ops

def _out(out, shape, like, dtype=None):
    """The caller's output buffer (checked: CUDA, contiguous, the op's shape and dtype), or a
    new one."""
    import torch
    dtype = dtype or torch.float32
    if out is None:
        return torch.empty(shape, device=like.device, dtype=dtype)
    if tuple(out.shape) != tuple(shape) or out.dtype != dtype or not out.is_cuda or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")
    return out


def op_conv3x3(x, w, b, stride=1, leaky=True, precision="fp32", cuda_stream=None, out=None):
    """x: CUDA (n, h, w, cin) float32; w: (cout, cin, 3, 3), b: (cout) on the host."""
    import torch
    n, h, wd, cin = x.shape
    w = np.ascontiguousarray(w, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    cout = w.shape[0]
    out = _out(out, (n, (h - 1) // stride + 1, (wd - 1) // stride + 1, cout), x)
    _check(_lib.tc_op_conv3x3(PRECISION[precision], _ptr(x, torch.float32), n, h, wd, cin, w.ctypes.data,
                              b.ctypes.data, cout, stride, int(leaky), out.data_ptr(), _stream_handle(cuda_stream)))
    return out


def op_last_used_tensor_cores() -> bool:
    return bool(_lib.tc_op_last_used_tensor_cores())


def op_correlation(f1, f2, r, precision="fp32", cuda_stream=None, out=None):
    import torch
    n, h, w, c = f1.shape
    out = _out(out, (n, h, w, (2 * r + 1) ** 2), f1)
    _check(_lib.tc_op_correlation(PRECISION[precision], _ptr(f1, torch.float32), _ptr(f2, torch.float32), n, h, w,
                                  c, r, out.data_ptr(), _stream_handle(cuda_stream)))
    return out


def op_correlation_bf16_noalloc(f1, f2, r, out=None, cuda_stream=None):
    """tc_op_correlation_bf16_noalloc: the BF16 cost volume without any device allocation
    inside the library (its staging lives in a fixed device array), for hosts that cannot
    allocate on the library's behalf.  Pass `out` pre-allocated ((n, h, w, (2r+1)^2) float32
    CUDA) to allocate nothing at all here either; returns without waiting."""
    import torch
    n, h, w, c = f1.shape
    if out is None:
        out = torch.empty((n, h, w, (2 * r + 1) ** 2), device=f1.device, dtype=torch.float32)
    _check(_lib.tc_op_correlation_bf16_noalloc(_ptr(f1, torch.float32), _ptr(f2, torch.float32), n, h, w, c, r,
                                               _ptr(out, torch.float32, "out"), _stream_handle(cuda_stream)))
    return out


def op_warp_features(f, flow, precision="fp32", cuda_stream=None, out=None):
    import torch
    n, h, w, c = f.shape
    out = _out(out, (n, h, w, c), f)
    _check(_lib.tc_op_warp_features(PRECISION[precision], _ptr(f, torch.float32), _ptr(flow, torch.float32), n, h,
                                    w, c, out.data_ptr(), _stream_handle(cuda_stream)))
    return out


def op_upsample_flow(flow, s, cuda_stream=None, out=None):
    import torch
    n, h, w, _ = flow.shape
    out = _out(out, (n, s * h, s * w, 2), flow)
    _check(_lib.tc_op_upsample_flow(_ptr(flow, torch.float32), n, h, w, s, out.data_ptr(),
                                    _stream_handle(cuda_stream)))
    return out


def op_poisson_solve(P, A, wc, iters=150, eta=0.15, kappa=0.2, cuda_stream=None, out=None):
    """Eq. 1 by Eq. 8 from O = A: P, A (c, h, w), wc (h, w) float32 CUDA tensors."""
    import torch
    c, h, w = P.shape
    O = _out(out, (c, h, w), P)
    _check(_lib.tc_op_poisson_solve(_ptr(P, torch.float32, "P"), _ptr(A, torch.float32, "A"),
                                    _ptr(wc, torch.float32, "wc"), c, h, w, int(iters), float(eta), float(kappa),
                                    O.data_ptr(), _stream_handle(cuda_stream)))
    return O


def op_sepconv(x, dw, db, pw, pb, dil=1, leaky=True, precision="fp32", cuda_stream=None, out=None):
    """One depthwise-separable refinement layer: x CUDA (n, h, w, cin) float32; dw (cin, 3, 3),
    db (cin), pw (cout, cin), pb (cout) on the host.  Returns (n, h, w, cout) float32."""
    import torch
    n, h, w, cin = x.shape
    cout = pw.shape[0]
    out = _out(out, (n, h, w, cout), x)
    arr = [np.ascontiguousarray(a, np.float32) for a in (dw, db, pw, pb)]
    _check(_lib.tc_op_sepconv(PRECISION[precision], _ptr(x, torch.float32, "x"), n, h, w, cin,
                              *[a.ctypes.data for a in arr], cout, int(dil), int(bool(leaky)), out.data_ptr(),
                              _stream_handle(cuda_stream)))
    return out


def op_downscale2(src, cuda_stream=None, out=None):
    """(c, h, w) float32 CUDA -> (c, ceil(h/2), ceil(w/2)): 2x2 block means, edges replicated."""
    import torch
    c, h, w = src.shape
    dst = _out(out, (c, (h + 1) // 2, (w + 1) // 2), src)
    _check(_lib.tc_op_downscale2(_ptr(src, torch.float32, "src"), c, h, w, dst.data_ptr(), _stream_handle(cuda_stream)))
    return dst


def op_consistency_next(It, Pt, Ip, Pp, Op, Fb, Ff, In, Pn, Fn, Fnb, scale=1, O=None, wc=None, mask=None,
                        cuda_stream=None, **params):
    """Images (3, h, w) float32 CUDA; flows (fh, fw, 2) float32 CUDA at 1/scale resolution:
    Fb = F_{t->t-1}, Ff = F_{t-1->t}, Fn = F_{t->t+1}, Fnb = F_{t+1->t}."""
    import torch
    _, h, w = It.shape
    fh, fw, _ = Fb.shape
    O = torch.empty_like(It) if O is None else O
    wc = torch.empty((h, w), device=It.device, dtype=torch.float32) if wc is None else wc
    mask = torch.empty((h, w), device=It.device, dtype=torch.uint8) if mask is None else mask
    c = _consistency_struct(**params)
    f32 = torch.float32
    _check(_lib.tc_op_consistency_next(*[_ptr(a, f32) for a in (It, Pt, Ip, Pp, Op, Fb, Ff, In, Pn, Fn, Fnb)],
                                       h, w, fh, fw, scale, ctypes.byref(c), O.data_ptr(), wc.data_ptr(),
                                       mask.data_ptr(), _stream_handle(cuda_stream)))
    return O, wc, mask


def op_consistency(It, Pt, Ip, Pp, Op, Fb, Ff, scale=1, O=None, wc=None, mask=None, cuda_stream=None, **params):
    """Images (3, h, w) float32 CUDA; flows (fh, fw, 2) float32 CUDA at 1/scale resolution."""
    import torch
    _, h, w = It.shape
    fh, fw, _ = Fb.shape
    O = torch.empty_like(It) if O is None else O
    wc = torch.empty((h, w), device=It.device, dtype=torch.float32) if wc is None else wc
    mask = torch.empty((h, w), device=It.device, dtype=torch.uint8) if mask is None else mask
    c = _consistency_struct(**params)
    f32 = torch.float32
    _check(_lib.tc_op_consistency(_ptr(It, f32), _ptr(Pt, f32), _ptr(Ip, f32), _ptr(Pp, f32), _ptr(Op, f32),
                                  _ptr(Fb, f32), _ptr(Ff, f32), h, w, fh, fw, scale, ctypes.byref(c), O.data_ptr(),
                                  wc.data_ptr(), mask.data_ptr(), _stream_handle(cuda_stream)))
    return O, wc, mask


# ----------------------------------------------------------------------------- server

class TcServerDesc(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weights_path", ctypes.c_char_p), ("weights_blob", ctypes.c_void_p),
                ("weights_bytes", ctypes.c_size_t), ("hbm_budget_bytes", ctypes.c_size_t), ("workers", ctypes.c_int),
                ("max_streams", ctypes.c_int), ("batch_lanes", ctypes.c_int)]


class TcCompletion(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int), ("frame", ctypes.c_longlong), ("tag", ctypes.c_ulonglong),
                ("status", ctypes.c_int), ("queued_us", ctypes.c_double), ("gpu_us", ctypes.c_double),
                ("total_us", ctypes.c_double), ("batch", ctypes.c_int)]


_lib.tc_server_create.argtypes = [ctypes.POINTER(TcServerDesc), ctypes.POINTER(_vp)]
_lib.tc_server_stream_bytes.argtypes = [_vp, _i, _i]
_lib.tc_server_stream_bytes.restype = ctypes.c_size_t
_lib.tc_server_bytes_in_use.argtypes = [_vp]
_lib.tc_server_bytes_in_use.restype = ctypes.c_size_t
_lib.tc_server_open.argtypes = [_vp, _i, _i, ctypes.POINTER(_i)]
_lib.tc_server_set_consistency.argtypes = [_vp, _i, ctypes.POINTER(TcConsistency)]
_lib.tc_server_submit.argtypes = [_vp, _i, _vp, _vp, _vp, ctypes.c_ulonglong]
_lib.tc_server_submit_rgb8.argtypes = [_vp, _i, _vp, _vp, _vp, ctypes.c_ulonglong]
_lib.tc_server_poll.argtypes = [_vp, ctypes.POINTER(TcCompletion), _i, _i]
_lib.tc_server_poll.restype = ctypes.c_int
_lib.tc_server_cancel.argtypes = [_vp, _i]
_lib.tc_server_close.argtypes = [_vp, _i]
_lib.tc_server_destroy.argtypes = [_vp]
_lib.tc_stream_device_bytes.argtypes = [_vp]
_lib.tc_stream_device_bytes.restype = ctypes.c_size_t
for _n in ["tc_server_create", "tc_server_open", "tc_server_set_consistency", "tc_server_submit",
           "tc_server_submit_rgb8", "tc_server_cancel",
           "tc_server_close", "tc_server_destroy"]:
    getattr(_lib, _n).restype = ctypes.c_int
EXPORTED += ["tc_server_create", "tc_server_stream_bytes", "tc_server_bytes_in_use", "tc_server_open",
             "tc_server_set_consistency", "tc_server_submit", "tc_server_submit_rgb8", "tc_server_poll",
             "tc_server_cancel",
             "tc_server_close", "tc_server_destroy", "tc_stream_device_bytes"]


def _host_ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise TypeError("host buffers must be contiguous float32")
    return a.ctypes.data


class Server:
    """tc_server_*: many streams of mixed resolutions on one GPU with HBM-budget admission
    and continuous batching.  Host buffers passed to submit() must stay alive until their
    completion is polled."""

    def __init__(self, weights_path, precision="bf16", hbm_budget_bytes=0, workers=4, max_streams=64, batch_lanes=1):
        """batch_lanes: streams of one resolution per shared batch (their frames run in
        shared launches when ready together); 1: a batch per stream."""
        d = TcServerDesc()
        d.precision = PRECISION[precision]
        d.weights_path = os.fsencode(weights_path)
        d.hbm_budget_bytes = int(hbm_budget_bytes)
        d.workers = int(workers)
        d.max_streams = int(max_streams)
        d.batch_lanes = int(batch_lanes)
        h = _vp()
        _check(_lib.tc_server_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def stream_bytes(self, width, height) -> int:
        return _lib.tc_server_stream_bytes(self._h, width, height)

    @property
    def bytes_in_use(self) -> int:
        return _lib.tc_server_bytes_in_use(self._h)

    def open(self, width, height) -> int:
        sid = _i()
        _check(_lib.tc_server_open(self._h, width, height, ctypes.byref(sid)))
        return sid.value

    def set_consistency(self, stream_id, **kw):
        c = _consistency_struct(**kw)
        _check(_lib.tc_server_set_consistency(self._h, stream_id, ctypes.byref(c)))

    def submit(self, stream_id, I, P, O, tag=0):
        self._keep[(stream_id, tag)] = (I, P, O)
        _check(_lib.tc_server_submit(self._h, stream_id, _host_ptr(I), _host_ptr(P), _host_ptr(O), tag))

    def submit_rgb8(self, stream_id, I, P, O, tag=0):
        """The next frame as 8-bit interleaved RGB: I, P, O host (H, W, 3) uint8 (as
        Stream.process_frame_host_rgb8_async)."""
        self._keep[(stream_id, tag)] = (I, P, O)
        _check(_lib.tc_server_submit_rgb8(self._h, stream_id, _hbuf(I, np.uint8), _hbuf(P, np.uint8),
                                          _hbuf(O, np.uint8), tag))

    def poll(self, max_n=256, timeout_ms=100):
        buf = (TcCompletion * max_n)()
        n = _lib.tc_server_poll(self._h, buf, max_n, timeout_ms)
        out = []
        for c in buf[:n]:
            self._keep.pop((c.stream_id, c.tag), None)
            out.append(dict(stream_id=c.stream_id, frame=c.frame, tag=c.tag, status=c.status, queued_us=c.queued_us,
                            gpu_us=c.gpu_us, total_us=c.total_us, batch=c.batch))
        return out

    def cancel(self, stream_id):
        _check(_lib.tc_server_cancel(self._h, stream_id))

    def close(self, stream_id):
        _check(_lib.tc_server_close(self._h, stream_id))

    def destroy(self):
        if getattr(self, "_h", None):
            _check(_lib.tc_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def stream_device_bytes(stream: "Stream") -> int:
    return _lib.tc_stream_device_bytes(stream._h)
