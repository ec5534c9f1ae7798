"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module draws random numbers and renders test content only: it holds none of the
method's arithmetic (no bilinear warp, no correlation, no consistency weights).  Frames
that move along a known flow are rendered by sampling a texture with a cubic B-spline
(``scipy.ndimage.map_coordinates(order=3)``), which is a different interpolant from the
bilinear warping function of the method, so neither side of a parity test can borrow the
other's warp from here.

Workloads (all seeded with NumPy's PCG64):

* ``pair64``: the 64x64 one-step case.  frame0 is U[0,1] noise blurred with a Gaussian
  (sigma 2, reflect border) and stretched to [0,1]; frame1 is frame0 resampled at
  ``x + F(x)``, with F a sum of 4 random sinusoids per component scaled to max |F| = 4 px
  (so F is the ground-truth flow from frame1 back to frame0).
* ``Sequence``: the 1920x1080 sequence.  A blurred-noise canvas (2400x1600) seen through a
  camera under an accumulated random affine motion (rotation U(-1,1) deg and translation
  U(-8,8) px per frame) with 3 opaque textured squares (side U(64,200) px, velocity
  U(-12,12) px/frame) composited on top, which creates occlusions.  Ground-truth backward
  and forward flows are analytic.
* stylised frames ``P_t = M_t I_t + N(0, 0.02)`` with a per-frame colour matrix
  ``M_t = I + U(-0.1, 0.1)^{3x3}``.
* ``training_pair``: a 256x256 pair (a, b) with known flow F = F_{a->b}: b is blurred noise,
  a samples b at ``x + F(x)`` (F a smooth random field, max |F| <= 16 px), and 0-3 textured
  rectangles sit at q in a and at q + d in b (F = d on them), occluding the background.
* He-normal weights for the lite flow network, written to a flat weight file.
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

__all__ = [
    "rng", "blurred_noise", "smooth_flow", "resample", "stylize", "pair64", "Sequence",
    "NetSpec", "he_weights", "write_weights", "layer_names", "random_lowres_flow", "training_pair",
    "training_batch",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def blurred_noise(h: int, w: int, c: int, sigma: float, g: np.random.Generator) -> np.ndarray:
    """U[0,1] noise, Gaussian-blurred per channel (reflect border), stretched to [0,1]. (c,h,w) f32."""
    x = g.random((c, h, w))
    out = np.empty((c, h, w), np.float64)
    for k in range(c):
        b = ndimage.gaussian_filter(x[k], sigma, mode="reflect")
        lo, hi = b.min(), b.max()
        out[k] = (b - lo) / max(hi - lo, 1e-12)
    return out.astype(np.float32)


def smooth_flow(h: int, w: int, max_mag: float, g: np.random.Generator, waves: int = 4) -> np.ndarray:
    """Sum of `waves` random sinusoids per component (<= 2 cycles per image), max |F| = max_mag. (2,h,w) f32."""
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    comps = []
    for _ in range(2):
        f = np.zeros((h, w))
        for _ in range(waves):
            fx, fy = g.uniform(-2.0, 2.0, 2)
            amp = g.uniform(0.5, 1.0)
            ph = g.uniform(0.0, 2.0 * math.pi)
            f += amp * np.sin(2.0 * math.pi * (fx * xx / w + fy * yy / h) + ph)
        comps.append(f)
    flow = np.stack(comps)
    mag = np.sqrt((flow ** 2).sum(0)).max()
    flow *= max_mag / max(mag, 1e-12)
    return flow.astype(np.float32)


def resample(img: np.ndarray, ys: np.ndarray, xs: np.ndarray, prefiltered: bool = False) -> np.ndarray:
    """Cubic B-spline resampling of a (c,h,w) image at float coordinates (mirror border)."""
    out = np.empty((img.shape[0],) + ys.shape, np.float32)
    for k in range(img.shape[0]):
        out[k] = ndimage.map_coordinates(img[k], [ys, xs], order=3, mode="mirror",
                                         prefilter=not prefiltered, output=np.float32)
    return out


def stylize(img: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """P = M I + N(0, 0.02) with M = I + U(-0.1, 0.1)^{3x3}; a stand-in for a per-frame stylizer."""
    m = np.eye(3) + g.uniform(-0.1, 0.1, (3, 3))
    p = np.einsum("ij,jhw->ihw", m, img.astype(np.float64))
    p += g.normal(0.0, 0.02, img.shape)
    return p.astype(np.float32)


def pair64(seed: int = 0, size: int = 64, max_flow: float = 4.0):
    """The 64x64 one-step case. Returns dict(I0, I1, P0, P1, flow_gt) with flow_gt = F_{1->0}."""
    g0, g1, g2 = rng(seed), rng(seed + 1), rng(seed + 2)
    i0 = blurred_noise(size, size, 3, 2.0, g0)
    flow = smooth_flow(size, size, max_flow, g1)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    i1 = resample(i0, yy + flow[1], xx + flow[0])
    p0 = stylize(i0, g2)
    p1 = stylize(i1, g2)
    return dict(I0=i0, I1=i1, P0=p0, P1=p1, flow_gt=flow)


def training_pair(seed: int, size: int = 256, max_flow: float = 16.0, max_rects: int = 3):
    """(a, b, F) with a(x) = b(x + F(x)) on the background and on each rectangle: (3,s,s),
    (3,s,s), (2,s,s) float32, F in pixels (u, v).  Rectangles moving by d cover q + [0, side)
    in a and q + d + [0, side) in b; what they cover in b, and what they uncover, has no
    match (occlusion)."""
    g = rng(seed)
    b = blurred_noise(size, size, 3, 2.0, g)
    flow = smooth_flow(size, size, g.uniform(0.25, 1.0) * max_flow, g)
    yy, xx = np.mgrid[0:size, 0:size].astype(np.float64)
    a = resample(b, yy + flow[1], xx + flow[0])
    lim = max_flow / math.sqrt(2.0)
    for _ in range(int(g.integers(0, max_rects + 1))):
        sw, sh = (int(v) for v in g.integers(size // 8, size // 3 + 1, 2))
        qx, qy = int(g.integers(0, size - sw + 1)), int(g.integers(0, size - sh + 1))
        dx, dy = g.uniform(-lim, lim, 2)
        tex = blurred_noise(sh, sw, 3, 2.0, g)
        a[:, qy:qy + sh, qx:qx + sw] = tex
        flow[0, qy:qy + sh, qx:qx + sw] = dx
        flow[1, qy:qy + sh, qx:qx + sw] = dy
        ty, tx = yy - qy - dy, xx - qx - dx
        inside = (ty >= 0) & (ty <= sh - 1) & (tx >= 0) & (tx <= sw - 1)
        if inside.any():
            vals = resample(tex, ty[inside], tx[inside])
            b[:, inside] = vals
    return a.astype(np.float32), b.astype(np.float32), flow.astype(np.float32)


def training_batch(seed: int, n: int, size: int = 256, max_flow: float = 16.0):
    """n pairs of ``training_pair`` with seeds seed, seed + 1, ...: (n,3,s,s) x 2, (n,2,s,s)."""
    ps = [training_pair(seed + i, size, max_flow) for i in range(n)]
    return (np.stack([p[0] for p in ps]), np.stack([p[1] for p in ps]), np.stack([p[2] for p in ps]))


def random_lowres_flow(h: int, w: int, max_mag: float, seed: int) -> np.ndarray:
    """A smooth random flow field (2,h,w) used as a stand-in network output."""
    return smooth_flow(h, w, max_mag, rng(seed))


@dataclass
class _Square:
    side: int
    pos: np.ndarray          # top-left (x, y) at frame 0
    vel: np.ndarray          # (vx, vy) px/frame
    tex: np.ndarray          # (3, side, side), spline-prefiltered


class Sequence:
    """The 1080p sequence: textured canvas under accumulated affine camera motion + 3 squares.

    Frame t samples canvas point ``A_t(x) = R(theta_t) (x - c_f) + c_c + T_t``; square k covers
    ``p_k + t v_k + [0, side)^2`` and is drawn over the background (later squares on top).
    """

    def __init__(self, width: int = 1920, height: int = 1080, seed: int = 0, n_squares: int = 3,
                 max_rot_deg: float = 1.0, max_trans: float = 8.0, max_vel: float = 12.0,
                 side_range=(64, 200), canvas=(1600, 2400)):
        self.W, self.H = width, height
        g = rng(seed)
        ch, cw = canvas
        self.canvas = np.stack([ndimage.spline_filter(c, order=3, mode="mirror")
                                for c in blurred_noise(ch, cw, 3, 2.0, g)]).astype(np.float32)
        self.cf = np.array([(width - 1) / 2.0, (height - 1) / 2.0])
        self.cc = np.array([(cw - 1) / 2.0, (ch - 1) / 2.0])
        self._g = g
        self.max_rot, self.max_trans = max_rot_deg, max_trans
        self.theta = [0.0]
        self.trans = [np.zeros(2)]
        self.squares = []
        hi = min(side_range[1], min(width, height) - 1)
        lo = min(side_range[0], hi)
        for _ in range(n_squares):
            side = int(g.integers(lo, hi + 1))
            tex = blurred_noise(side, side, 3, 2.0, g)
            tex = np.stack([ndimage.spline_filter(c, order=3, mode="mirror") for c in tex])
            pos = np.array([g.uniform(0, width - side), g.uniform(0, height - side)])
            vel = g.uniform(-max_vel, max_vel, 2)
            self.squares.append(_Square(side, pos, vel, tex.astype(np.float32)))
        self._style_seed = seed + 1000
        yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
        self._xx, self._yy = xx, yy

    def _motion(self, t: int):
        while len(self.theta) <= t:
            self.theta.append(self.theta[-1] + math.radians(self._g.uniform(-self.max_rot, self.max_rot)))
            self.trans.append(self.trans[-1] + self._g.uniform(-self.max_trans, self.max_trans, 2))
        return self.theta[t], self.trans[t]

    def _cam(self, t: int, x: np.ndarray, y: np.ndarray):
        th, tr = self._motion(t)
        c, s = math.cos(th), math.sin(th)
        dx, dy = x - self.cf[0], y - self.cf[1]
        return c * dx - s * dy + self.cc[0] + tr[0], s * dx + c * dy + self.cc[1] + tr[1]

    def _cam_inv(self, t: int, cx: np.ndarray, cy: np.ndarray):
        th, tr = self._motion(t)
        c, s = math.cos(th), math.sin(th)
        dx, dy = cx - self.cc[0] - tr[0], cy - self.cc[1] - tr[1]
        return c * dx + s * dy + self.cf[0], -s * dx + c * dy + self.cf[1]

    def _square_ids(self, t: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        ids = np.full(x.shape, -1, np.int32)
        for k, sq in enumerate(self.squares):
            p = sq.pos + t * sq.vel
            inside = (x >= p[0]) & (x < p[0] + sq.side) & (y >= p[1]) & (y < p[1] + sq.side)
            ids[inside] = k
        return ids

    def frame(self, t: int) -> np.ndarray:
        """I_t as (3, H, W) float32."""
        cx, cy = self._cam(t, self._xx, self._yy)
        img = resample(self.canvas, cy, cx, prefiltered=True)
        ids = self._square_ids(t, self._xx, self._yy)
        for k, sq in enumerate(self.squares):
            sel = ids == k
            if not sel.any():
                continue
            p = sq.pos + t * sq.vel
            vals = resample(sq.tex, self._yy[sel] - p[1], self._xx[sel] - p[0], prefiltered=True)
            img[:, sel] = vals
        return img

    def stylized(self, t: int, img: np.ndarray) -> np.ndarray:
        return stylize(img, rng(self._style_seed + t))

    def flow_backward(self, t: int) -> np.ndarray:
        """Ground-truth F_{t->t-1} as (2, H, W) float32 (t >= 1)."""
        x, y = self._xx, self._yy
        px, py = self._cam_inv(t - 1, *self._cam(t, x, y))
        f = np.stack([px - x, py - y])
        ids = self._square_ids(t, x, y)
        for k, sq in enumerate(self.squares):
            sel = ids == k
            f[0][sel] = -sq.vel[0]
            f[1][sel] = -sq.vel[1]
        return f.astype(np.float32)

    def flow_forward(self, t: int) -> np.ndarray:
        """Ground-truth F_{t-1->t} on the pixels of frame t-1, (2, H, W) float32 (t >= 1)."""
        x, y = self._xx, self._yy
        px, py = self._cam_inv(t, *self._cam(t - 1, x, y))
        f = np.stack([px - x, py - y])
        ids = self._square_ids(t - 1, x, y)
        for k, sq in enumerate(self.squares):
            sel = ids == k
            f[0][sel] = sq.vel[0]
            f[1][sel] = sq.vel[1]
        return f.astype(np.float32)


# ---------------------------------------------------------------------------------------
# Network weights: He-normal initialisation of the lite flow network, written to a file.
# ---------------------------------------------------------------------------------------

@dataclass
class NetSpec:
    """Shape of the lite flow network: pyramid channels per level and correlation radius."""
    chans: tuple = (16, 32, 64, 96, 128)
    radius: int = 4
    decoder: tuple = (128, 96, 64, 32)
    layers: list = field(default_factory=list)
    # refinement network (depthwise-separable layers after the finest estimator): output
    # channels and dilations per layer, empty for none
    refine: tuple = ()
    refine_dil: tuple = ()

    @property
    def levels(self) -> int:
        return len(self.chans)

    def layer_table(self):
        """(name, cin, cout, stride, leaky) in file order: pyramid levels 1..L, then
        estimators at levels L..2 (conv1..conv5)."""
        t = []
        prev = 3
        for l, c in enumerate(self.chans, start=1):
            t.append((f"pyr{l}a", prev, c, 2, 1))
            t.append((f"pyr{l}b", c, c, 1, 1))
            t.append((f"pyr{l}c", c, c, 1, 1))
            prev = c
        d = (2 * self.radius + 1) ** 2
        c1, c2, c3, c4 = self.decoder
        for l in range(self.levels, 1, -1):
            cin0 = d + self.chans[l - 1] + 2
            t.append((f"est{l}c1", cin0, c1, 1, 1))
            t.append((f"est{l}c2", c1, c2, 1, 1))
            t.append((f"est{l}c3", c2, c3, 1, 1))
            t.append((f"est{l}c4", c3 + c2, c4, 1, 1))
            t.append((f"est{l}c5", c4 + c3, 2, 1, 0))
        return t


REFINE_CHANS = (128, 128, 128, 96, 64, 32, 2)
REFINE_DIL = (1, 2, 4, 8, 16, 1, 1)


def refine_table(spec: NetSpec):
    """(name, cin, cout, dil, leaky) of the refinement layers; the first reads cat(flow, x4,
    x3) of the level-2 estimator, the last (2 outputs) has no activation."""
    t = []
    cin = 2 + spec.decoder[3] + spec.decoder[2]
    for k, (cout, dil) in enumerate(zip(spec.refine, spec.refine_dil)):
        t.append((f"ref{k + 1}", cin, cout, dil, 0 if k == len(spec.refine) - 1 else 1))
        cin = cout
    return t


def layer_names(spec: NetSpec):
    return [n for n, *_ in spec.layer_table()]


def he_weights(spec: NetSpec, seed: int = 0, head_gain: float = 1.0):
    """He-normal weights, std = sqrt(2 / ((1 + 0.1^2) fan_in)), zero biases, PCG64(seed),
    drawn in file order.  `head_gain` scales the flow-head weights."""
    g = rng(seed)
    out = []
    for name, cin, cout, stride, leaky in spec.layer_table():
        std = math.sqrt(2.0 / ((1.0 + 0.01) * cin * 9))
        w = g.normal(0.0, std, (cout, cin, 3, 3))
        if name.endswith("c5"):
            w *= head_gain
        out.append(dict(name=name, cin=cin, cout=cout, stride=stride, leaky=leaky,
                        w=w.astype(np.float32), b=np.zeros(cout, np.float32)))
    # refinement layers after the conv layers: depthwise fan-in 9, pointwise fan-in cin
    for name, cin, cout, dil, leaky in refine_table(spec):
        dw = g.normal(0.0, math.sqrt(2.0 / ((1.0 + 0.01) * 9)), (cin, 3, 3))
        pw = g.normal(0.0, math.sqrt(2.0 / ((1.0 + 0.01) * cin)), (cout, cin))
        if not leaky:
            pw *= head_gain
        out.append(dict(name=name, cin=cin, cout=cout, dil=dil, leaky=leaky, dw=dw.astype(np.float32),
                        db=np.zeros(cin, np.float32), pw=pw.astype(np.float32), pb=np.zeros(cout, np.float32)))
    return out


WEIGHT_MAGIC = b"TCW1"


def write_weights(path: str, spec: NetSpec, layers) -> None:
    """Flat little-endian file: magic 'TCW1'; int32 levels, radius, chans[levels],
    decoder[4], n_layers; per layer int32 cout, cin, stride, leaky, float32 w (OIHW), b.
    With refinement layers (dicts holding 'dw') the magic is 'TCW2' and the conv layers are
    followed by int32 n_ref and per layer int32 cin, cout, dil, leaky, float32 dw[cin][3][3],
    db[cin], pw[cout][cin], pb[cout]."""
    conv = [L for L in layers if "dw" not in L]
    sep = [L for L in layers if "dw" in L]
    with open(path, "wb") as f:
        f.write(b"TCW2" if sep else WEIGHT_MAGIC)
        f.write(struct.pack("<ii", spec.levels, spec.radius))
        f.write(struct.pack(f"<{spec.levels}i", *spec.chans))
        f.write(struct.pack("<4i", *spec.decoder))
        f.write(struct.pack("<i", len(conv)))
        for L in conv:
            f.write(struct.pack("<4i", L["cout"], L["cin"], L["stride"], L["leaky"]))
            f.write(np.ascontiguousarray(L["w"], "<f4").tobytes())
            f.write(np.ascontiguousarray(L["b"], "<f4").tobytes())
        if sep:
            f.write(struct.pack("<i", len(sep)))
            for L in sep:
                f.write(struct.pack("<4i", L["cin"], L["cout"], L["dil"], L["leaky"]))
                for k in ("dw", "db", "pw", "pb"):
                    f.write(np.ascontiguousarray(L[k], "<f4").tobytes())
