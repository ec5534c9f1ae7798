"""FP64 CPU oracle for the hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It wraps ``oracle.c`` (plain C, FP64, OpenMP) through ctypes and adds
the per-stream bookkeeping of Sec. 3.1 (first frame ``O_1 = P_1``; later frames need
``I_{t-1}, P_{t-1}, O_{t-1}``).  It shares no code with the CUDA library; the two read the
same weight *file*, each with its own parser.

Arrays are NumPy, planar (C, H, W).  Inputs are converted to float64.
"""
from __future__ import annotations

import ctypes
import os
import struct
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

# Defaults of the consistency step: k1 (Eq. 3 clamp), alpha (Eq. 3/7), lambda (Eq. 7) are the
# paper's final setting (Sec. 4.2); c1, c2 are the forward-backward test constants.
PAPER_FINAL = dict(k1=0.3, k2=0.5, alpha=6.5e3, lam=2.0)
PAPER_OBJECTIVE = dict(k1=0.3, k2=0.3, alpha=1.0e4, lam=0.7)
FB_C1, FB_C2 = 0.01, 0.5


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp, ip, u8p = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_uint8))
        c_int, c_double, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        _lib.orc_conv3x3.argtypes = [dp, c_int, c_int, c_int, dp, dp, c_int, c_int, c_int, dp]
        _lib.orc_warp.argtypes = [dp, c_int, c_int, c_int, dp, c_int, dp, u8p]
        _lib.orc_correlation.argtypes = [dp, dp, c_int, c_int, c_int, c_int, dp]
        _lib.orc_upsample_flow.argtypes = [dp, c_int, c_int, c_int, dp]
        _lib.orc_pad_replicate.argtypes = [dp, c_int, c_int, c_int, c_int, c_int, dp]
        _lib.orc_pyramid.argtypes = [dp, c_int, c_int, c_int, vp, vp]
        _lib.orc_poisson_grad.argtypes = [c_int, c_int, dp, dp, dp, dp, dp]
        _lib.orc_poisson_solve.argtypes = [c_int, c_int, c_int, dp, dp, dp, c_double, c_double, c_int, dp]
        _lib.orc_flow.argtypes = [vp, vp, ip, c_int, c_int, c_int, c_int, vp, dp, vp]
        _lib.orc_flow2.argtypes = [vp, vp, ip, c_int, c_int, c_int, c_int, vp, dp, vp, vp, c_int]
        _lib.orc_depthwise3x3.argtypes = [dp, c_int, c_int, c_int, dp, dp, c_int, dp]
        _lib.orc_pointwise.argtypes = [dp, c_int, c_int, c_int, dp, dp, c_int, c_int, dp]
        _lib.orc_refine.argtypes = [dp, dp, c_int, dp, c_int, c_int, c_int, vp, c_int, dp]
        _lib.orc_consistency.argtypes = [c_int, c_int, dp, dp, dp, dp, dp, dp, dp, c_double,
                                         c_double, c_double, c_int, c_double, c_double, dp, dp,
                                         u8p, u8p, dp]
        _lib.orc_consistency_next.argtypes = [c_int, c_int, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp,
                                              c_double, c_double, c_double, c_double, c_int, c_double,
                                              c_double, dp, dp, u8p, u8p, dp, dp]
        _lib.orc_bruteforce_flow.argtypes = [dp, dp, c_int, c_int, c_int, c_int, ip]
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


class _Layer(ctypes.Structure):
    _fields_ = [("cin", ctypes.c_int), ("cout", ctypes.c_int), ("stride", ctypes.c_int),
                ("leaky", ctypes.c_int), ("w", ctypes.POINTER(ctypes.c_double)),
                ("b", ctypes.POINTER(ctypes.c_double))]


class _SepLayer(ctypes.Structure):
    _fields_ = [("cin", ctypes.c_int), ("cout", ctypes.c_int), ("dil", ctypes.c_int), ("leaky", ctypes.c_int),
                ("dw", ctypes.POINTER(ctypes.c_double)), ("db", ctypes.POINTER(ctypes.c_double)),
                ("pw", ctypes.POINTER(ctypes.c_double)), ("pb", ctypes.POINTER(ctypes.c_double))]


# ----------------------------------------------------------------------------- primitives

def conv3x3(x, w, b=None, stride=1, leaky=True):
    """3x3 conv, zero pad 1 (Sec. 3.2).  x (cin,h,w), w (cout,cin,3,3) -> (cout,ho,wo)."""
    x, w = _d(x), _d(w)
    cin, h, wd = x.shape
    cout = w.shape[0]
    b = _d(b) if b is not None else None
    out = np.empty((cout, (h - 1) // stride + 1, (wd - 1) // stride + 1))
    lib().orc_conv3x3(_p(x), cin, h, wd, _p(w), _p(b), cout, stride, int(leaky), _p(out))
    return out


def warp(src, flow, zero_outside):
    """Backward bilinear warp (Sec. 3.1 Gamma).  Returns (warped, in_bounds)."""
    src, flow = _d(src), _d(flow)
    c, h, w = src.shape
    out = np.empty_like(src)
    inb = np.empty((h, w), np.uint8)
    lib().orc_warp(_p(src), c, h, w, _p(flow), int(zero_outside), _p(out), _p(inb, ctypes.c_uint8))
    return out, inb


def correlation(f1, f2, r):
    """Cost volume with LeakyReLU, ((2r+1)^2, h, w) (Sec. 3.2)."""
    f1, f2 = _d(f1), _d(f2)
    c, h, w = f1.shape
    out = np.empty(((2 * r + 1) ** 2, h, w))
    lib().orc_correlation(_p(f1), _p(f2), c, h, w, r, _p(out))
    return out


def upsample_flow(flow, s):
    """s-times bilinear flow upsampling with values times s."""
    flow = _d(flow)
    _, h, w = flow.shape
    out = np.empty((2, s * h, s * w))
    lib().orc_upsample_flow(_p(flow), h, w, s, _p(out))
    return out


def pad_replicate(img, hp, wp):
    img = _d(img)
    c, h, w = img.shape
    out = np.empty((c, hp, wp))
    lib().orc_pad_replicate(_p(img), c, h, w, hp, wp, _p(out))
    return out


def downscale2(img):
    """The half-size flow input of the fast preset (Table 3: flow on 2x downscaled frames):
    (c, h, w) -> (c, ceil(h/2), ceil(w/2)), each value the mean of a 2x2 block, the last row
    and column replicated when h or w is odd."""
    a = _d(img)
    c, h, w = a.shape
    hn, wn = (h + 1) // 2, (w + 1) // 2
    p = np.pad(a, ((0, 0), (0, 2 * hn - h), (0, 2 * wn - w)), mode="edge")
    return p.reshape(c, hn, 2, wn, 2).mean(axis=(2, 4))


def consistency(It, Pt, Ip, Pp, Op, Fb, Ff, k1=0.3, alpha=6.5e3, lam=2.0, fb_check=True,
                c1=FB_C1, c2=FB_C2):
    """Causal consistency step (Eqs. 2-7, w_n = 0).  Returns dict(O, wc, mask, band, wp)."""
    arrs = [_d(a) for a in (It, Pt, Ip, Pp, Op, Fb, Ff)]
    _, h, w = arrs[0].shape
    O = np.empty((3, h, w)); wc = np.empty((h, w)); wp = np.empty((h, w))
    mask = np.empty((h, w), np.uint8); band = np.empty((h, w), np.uint8)
    lib().orc_consistency(h, w, *[_p(a) for a in arrs], float(k1), float(alpha), float(lam),
                          int(fb_check), float(c1), float(c2), _p(O), _p(wc),
                          _p(mask, ctypes.c_uint8), _p(band, ctypes.c_uint8), _p(wp))
    return dict(O=O, wc=wc, mask=mask, band=band, wp=wp)


def consistency_next(It, Pt, Ip, Pp, Op, Fb, Ff, In, Pn, Fn, Fnb, k1=0.3, k2=0.5, alpha=6.5e3, lam=2.0,
                     fb_check=True, c1=FB_C1, c2=FB_C2):
    """Consistency step with both temporal neighbours (Eqs. 2-7): Fb = F_{t->t-1},
    Ff = F_{t-1->t}, Fn = F_{t->t+1}, Fnb = F_{t+1->t}, all (2, h, w).  Returns dict(O, wc,
    mask (bit 0: M_p, bit 1: M_n), band (same bits), wp, wn)."""
    arrs = [_d(a) for a in (It, Pt, Ip, Pp, Op, Fb, Ff, In, Pn, Fn, Fnb)]
    _, h, w = arrs[0].shape
    O = np.empty((3, h, w)); wc = np.empty((h, w)); wp = np.empty((h, w)); wn = np.empty((h, w))
    mask = np.empty((h, w), np.uint8); band = np.empty((h, w), np.uint8)
    lib().orc_consistency_next(h, w, *[_p(a) for a in arrs], float(k1), float(k2), float(alpha), float(lam),
                               int(fb_check), float(c1), float(c2), _p(O), _p(wc),
                               _p(mask, ctypes.c_uint8), _p(band, ctypes.c_uint8), _p(wp), _p(wn))
    return dict(O=O, wc=wc, mask=mask, band=band, wp=wp, wn=wn)


def poisson_grad(O, P, A, wc):
    """Gradient of the screened-Poisson energy (Eq. 1) for one (h, w) channel."""
    O, P, A, wc = _d(O), _d(P), _d(A), _d(wc)
    h, w = O.shape
    g = np.empty((h, w))
    lib().orc_poisson_grad(h, w, _p(O), _p(P), _p(A), _p(wc), _p(g))
    return g


def poisson_solve(P, A, wc, eta=0.15, kappa=0.2, iters=150):
    """Eq. 8 SGD-momentum iterations from O = A; P, A (c, h, w), wc (h, w)."""
    P, A, wc = _d(P), _d(A), _d(wc)
    c, h, w = P.shape
    O = np.empty((c, h, w))
    lib().orc_poisson_solve(c, h, w, _p(P), _p(A), _p(wc), float(eta), float(kappa), int(iters), _p(O))
    return O


def depthwise3x3(x, dw, db=None, dil=1):
    """Depthwise 3x3 conv with dilation (zero padding): x (c, h, w), dw (c, 3, 3), db (c)."""
    x, dw = _d(x), _d(dw)
    c, h, w = x.shape
    out = np.empty((c, h, w))
    lib().orc_depthwise3x3(_p(x), c, h, w, _p(dw), _p(_d(db)) if db is not None else None, int(dil), _p(out))
    return out


def pointwise(x, pw, pb=None, leaky=True):
    """1x1 conv: x (cin, h, w), pw (cout, cin), pb (cout); LeakyReLU 0.1 if leaky."""
    x, pw = _d(x), _d(pw)
    cin, h, w = x.shape
    cout = pw.shape[0]
    out = np.empty((cout, h, w))
    lib().orc_pointwise(_p(x), cin, h, w, _p(pw), _p(_d(pb)) if pb is not None else None, cout, int(leaky), _p(out))
    return out


def _sep_table(ref):
    arr = (_SepLayer * max(1, len(ref)))()
    for i, L in enumerate(ref):
        arr[i] = _SepLayer(L["cin"], L["cout"], L["dil"], L["leaky"], _p(L["dw"]), _p(L["db"]), _p(L["pw"]),
                           _p(L["pb"]))
    return arr


def refine(flow, x4, x3, ref):
    """Refinement of a flow (2, h, w) from the head input x4 (c4, h, w), x3 (c3, h, w) by
    the depthwise-separable layers `ref` (dicts cin, cout, dil, leaky, dw, db, pw, pb)."""
    flow, x4, x3 = _d(flow), _d(x4), _d(x3)
    _, h, w = flow.shape
    ref = [dict(L, dw=_d(L["dw"]), db=_d(L["db"]), pw=_d(L["pw"]), pb=_d(L["pb"])) for L in ref]
    tab = _sep_table(ref)
    out = np.empty((2, h, w))
    lib().orc_refine(_p(flow), _p(x4), x4.shape[0], _p(x3), x3.shape[0], h, w, ctypes.cast(tab, ctypes.c_void_p),
                     len(ref), _p(out))
    return out


def bruteforce_flow(a, b, r):
    """Integer SSD-argmin displacement index per pixel (3x3 patches, border clamp)."""
    a, b = _d(a), _d(b)
    c, h, w = a.shape
    k = np.empty((h, w), np.int32)
    lib().orc_bruteforce_flow(_p(a), _p(b), c, h, w, r, _p(k, ctypes.c_int))
    return k


def epe(f, g):
    """Average end-point error, Eq. 10: mean over pixels of ||f - g||_2."""
    f, g = _d(f), _d(g)
    return float(np.sqrt(((f - g) ** 2).sum(0)).mean())


# ----------------------------------------------------------------------------- network

@dataclass
class Net:
    levels: int
    radius: int
    chans: tuple
    decoder: tuple
    layers: list  # dicts with cin, cout, stride, leaky, w (float64), b (float64)
    ref: list = field(default_factory=list)  # refinement: dicts cin, cout, dil, leaky, dw, db, pw, pb

    def _table(self, lo, hi):
        arr = (_Layer * (hi - lo))()
        for i, L in enumerate(self.layers[lo:hi]):
            arr[i] = _Layer(L["cin"], L["cout"], L["stride"], L["leaky"], _p(L["w"]), _p(L["b"]))
        return arr


def load_weights(path) -> Net:
    """Parse the flat weight file (magic 'TCW1', or 'TCW2' with a refinement section after
    the conv layers; little-endian)."""
    with open(path, "rb") as f:
        data = f.read()
    if data[:4] not in (b"TCW1", b"TCW2"):
        raise ValueError("not a TCW1 / TCW2 weight file")
    off = 4
    levels, radius = struct.unpack_from("<ii", data, off); off += 8
    chans = struct.unpack_from(f"<{levels}i", data, off); off += 4 * levels
    decoder = struct.unpack_from("<4i", data, off); off += 16
    (n,) = struct.unpack_from("<i", data, off); off += 4
    layers = []
    for _ in range(n):
        cout, cin, stride, leaky = struct.unpack_from("<4i", data, off); off += 16
        w = np.frombuffer(data, "<f4", cout * cin * 9, off).reshape(cout, cin, 3, 3); off += 4 * w.size
        b = np.frombuffer(data, "<f4", cout, off); off += 4 * cout
        layers.append(dict(cin=cin, cout=cout, stride=stride, leaky=leaky,
                           w=w.astype(np.float64), b=b.astype(np.float64)))
    ref = []
    if data[:4] == b"TCW2":
        (nr,) = struct.unpack_from("<i", data, off); off += 4
        for _ in range(nr):
            cin, cout, dil, leaky = struct.unpack_from("<4i", data, off); off += 16
            arrs = []
            for shape in ((cin, 3, 3), (cin,), (cout, cin), (cout,)):
                a = np.frombuffer(data, "<f4", int(np.prod(shape)), off).reshape(shape); off += 4 * a.size
                arrs.append(a.astype(np.float64))
            ref.append(dict(cin=cin, cout=cout, dil=dil, leaky=leaky, dw=arrs[0], db=arrs[1], pw=arrs[2], pb=arrs[3]))
    return Net(levels, radius, tuple(chans), tuple(decoder), layers, ref)


def net_from_layers(spec_levels, radius, chans, decoder, layers) -> Net:
    conv = [L for L in layers if "dw" not in L]
    sep = [L for L in layers if "dw" in L]
    return Net(spec_levels, radius, tuple(chans), tuple(decoder),
               [dict(cin=L["cin"], cout=L["cout"], stride=L["stride"], leaky=L["leaky"],
                     w=_d(L["w"]), b=_d(L["b"])) for L in conv],
               [dict(cin=L["cin"], cout=L["cout"], dil=L["dil"], leaky=L["leaky"], dw=_d(L["dw"]), db=_d(L["db"]),
                     pw=_d(L["pw"]), pb=_d(L["pb"])) for L in sep])


def padded_size(h, w, levels):
    m = 1 << levels
    return -(-h // m) * m, -(-w // m) * m


def pyramid(net: Net, img_padded):
    """Feature pyramid of a padded (3, hp, wp) image: list of (chans[l], hp>>l, wp>>l)."""
    img = _d(img_padded)
    _, hp, wp = img.shape
    feats = [np.empty((c, hp >> l, wp >> l)) for l, c in enumerate(net.chans, start=1)]
    ptrs = (ctypes.c_void_p * net.levels)(*[f.ctypes.data for f in feats])
    tab = net._table(0, 3 * net.levels)
    lib().orc_pyramid(_p(img), hp, wp, net.levels, ctypes.cast(tab, ctypes.c_void_p),
                      ctypes.cast(ptrs, ctypes.c_void_p))
    return feats


def flow_from_pyramids(net: Net, feat_self, feat_other, hp, wp, level_flows=False):
    """Coarse-to-fine flow F_{self->other} at the padded resolution (2, hp, wp)."""
    out = np.empty((2, hp, wp))
    tab = net._table(3 * net.levels, len(net.layers))
    ps = (ctypes.c_void_p * net.levels)(*[f.ctypes.data for f in feat_self])
    po = (ctypes.c_void_p * net.levels)(*[f.ctypes.data for f in feat_other])
    chans = (ctypes.c_int * net.levels)(*net.chans)
    lf = None
    lfp = None
    if level_flows:
        lf = [np.empty((2, hp >> l, wp >> l)) for l in range(2, net.levels + 1)]
        lfp = ctypes.cast((ctypes.c_void_p * len(lf))(*[a.ctypes.data for a in lf]), ctypes.c_void_p)
    rt = _sep_table(net.ref)
    lib().orc_flow2(ctypes.cast(ps, ctypes.c_void_p), ctypes.cast(po, ctypes.c_void_p), chans,
                    hp, wp, net.levels, net.radius, ctypes.cast(tab, ctypes.c_void_p), _p(out), lfp,
                    ctypes.cast(rt, ctypes.c_void_p), len(net.ref))
    return (out, lf) if level_flows else out


def flow_pair(net: Net, I_a, I_b):
    """F_{a->b} and F_{b->a} for two (3, h, w) frames, cropped to (2, h, w)."""
    _, h, w = I_a.shape
    hp, wp = padded_size(h, w, net.levels)
    pa = pyramid(net, pad_replicate(I_a, hp, wp))
    pb = pyramid(net, pad_replicate(I_b, hp, wp))
    fab = flow_from_pyramids(net, pa, pb, hp, wp)[:, :h, :w]
    fba = flow_from_pyramids(net, pb, pa, hp, wp)[:, :h, :w]
    return np.ascontiguousarray(fab), np.ascontiguousarray(fba)


class Stream:
    """Oracle of one video stream (Sec. 3.1): O_1 = P_1; later frames blend along the flow.

    latency = 0: causal form, step(I_t, P_t) returns frame t (w_n = 0).
    latency = 1: step(I_{t+1}, P_{t+1}) returns frame t blended with both neighbours (w_n with
    the clamp k2), None for the first frame of a sequence; flush() returns the last frame
    (w_n = 0, no next frame) and starts a new sequence.
    flow_downscale = 2: the flow network runs on downscale2 of the frames (the fast preset
    of Table 3, with solver_iters = 50)."""

    def __init__(self, net: Net, k1=0.3, alpha=6.5e3, lam=2.0, fb_check=True, c1=FB_C1, c2=FB_C2,
                 solver_iters=0, eta=0.15, kappa=0.2, k2=0.5, latency=0, flow_downscale=1):
        self.net = net
        # flow_downscale = 2: the network sees downscale2(I) and its level-2 flow is upsampled
        # x8 to the frame (the fast preset); 1: the frame itself, x4
        self.fs = int(flow_downscale)
        self.params = dict(k1=k1, alpha=alpha, lam=lam, fb_check=fb_check, c1=c1, c2=c2)
        self.k2 = float(k2)
        self.latency = int(latency)
        self.solver = (int(solver_iters), float(eta), float(kappa))
        self.prev = None  # (I, P, O, pyramid)
        # latency 1: frames t-1 and t as (I, P, pyramid), O_{t-1}, flows of the pair (t, t-1)
        self.hist = []
        self.O_prev = None
        self.flows = None

    def _solve(self, r, P):
        iters, eta, kappa = self.solver
        if iters > 0:
            # Eq. 1 solved by Eq. 8 from A_t: the output and the next frame's O_{t-1}
            r["A"] = r["O"]
            r["O"] = poisson_solve(P, r["A"], r["wc"], eta=eta, kappa=kappa, iters=iters)
        return r

    def _pyramid(self, I):
        x = downscale2(I) if self.fs == 2 else I
        _, hn, wn = x.shape
        hp, wp = padded_size(hn, wn, self.net.levels)
        return pyramid(self.net, pad_replicate(x, hp, wp)), hp, wp

    def _flow(self, pyr_a, pyr_b, hp, wp, h, w):
        """F_{a->b} on the (h, w) frame."""
        if self.fs == 1:
            return np.ascontiguousarray(flow_from_pyramids(self.net, pyr_a, pyr_b, hp, wp)[:, :h, :w])
        _, lf = flow_from_pyramids(self.net, pyr_a, pyr_b, hp, wp, level_flows=True)
        return np.ascontiguousarray(upsample_flow(lf[0], 4 * self.fs)[:, :h, :w])

    def _first(self, P):
        _, h, w = P.shape
        return dict(O=P.copy(), wc=np.zeros((h, w)), mask=np.zeros((h, w), np.uint8),
                    band=np.zeros((h, w), np.uint8), Fb=None, Ff=None)

    def _step_latency(self, I, P):
        _, h, w = I.shape
        pyr, hp, wp = self._pyramid(I)
        if not self.hist:
            self.hist = [(I, P, pyr)]
            return None
        It, Pt, pyr_t = self.hist[-1]
        # the pair (t+1, t): F_{t+1->t} and F_{t->t+1}
        Fb1 = self._flow(pyr, pyr_t, hp, wp, h, w)
        Ff1 = self._flow(pyr_t, pyr, hp, wp, h, w)
        if len(self.hist) == 1:
            r = self._first(Pt)
        else:
            Ip, Pp, _ = self.hist[0]
            Fb, Ff = self.flows
            r = consistency_next(It, Pt, Ip, Pp, self.O_prev, Fb, Ff, I, P, Ff1, Fb1, k2=self.k2, **self.params)
            r = self._solve(r, Pt)
            r.update(Fb=Fb, Ff=Ff, Fn=Ff1, Fnb=Fb1)
        self.O_prev = r["O"]
        self.flows = (Fb1, Ff1)
        self.hist = [self.hist[-1], (I, P, pyr)]
        return r

    def flush(self):
        """latency 1: the last frame of the sequence (no next frame: w_n = 0)."""
        if self.latency != 1 or not self.hist:
            return None
        It, Pt, _ = self.hist[-1]
        if len(self.hist) == 1:
            r = self._first(Pt)
        else:
            Ip, Pp, _ = self.hist[0]
            Fb, Ff = self.flows
            r = self._solve(consistency(It, Pt, Ip, Pp, self.O_prev, Fb, Ff, **self.params), Pt)
            r.update(Fb=Fb, Ff=Ff)
        self.hist, self.O_prev, self.flows = [], None, None
        return r

    def step(self, I, P):
        I, P = _d(I), _d(P)
        if self.latency == 1:
            return self._step_latency(I, P)
        _, h, w = I.shape
        pyr, hp, wp = self._pyramid(I)
        if self.prev is None:
            self.prev = (I, P, P.copy(), pyr)
            return self._first(P)
        Ip, Pp, Op, pyr_p = self.prev
        Fb = self._flow(pyr, pyr_p, hp, wp, h, w)
        Ff = self._flow(pyr_p, pyr, hp, wp, h, w)
        r = self._solve(consistency(I, P, Ip, Pp, Op, Fb, Ff, **self.params), P)
        self.prev = (I, P, r["O"], pyr)
        r.update(Fb=Fb, Ff=Ff)
        return r
