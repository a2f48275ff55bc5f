"""Seeded synthetic inputs for the box-tracking hot path.

This module holds no step of the tracking method.  It renders analytic
textures at chosen coordinates, quantises them to uint8 frames, and draws
boxes, motions and resolutions from seeded generators.  Both the CUDA path's
tests and the oracle's tests take their inputs from here, so nothing in it
may depend on either of them.

Texture recipe (one texture T):
  * a base of 128;
  * 64 Gaussian blobs A*exp(-r^2 / (2 s^2)), centre uniform over the texture's
    domain, s ~ U[3, 20] px, |A| ~ U[40, 200] with a random sign, each blob
    truncated to r <= 6 s (its value there is below 4e-6 of its amplitude);
  * 3 sinusoidal gratings A*sin(2 pi (x cos th + y sin th) / P + phi) with
    P ~ U[8, 40] px, th ~ U[0, pi), A ~ U[10, 40], phi ~ U[0, 2 pi);
  * the sum clipped to [0, 255].
Frames are T evaluated at pixel centres (integer coordinates) through an
inverse map, then quantised as u8 = clamp(floor(v + 0.5), 0, 255).  Motion is
rendered by evaluating T at inverse-mapped coordinates, never by resampling a
raster.  Seeds: workload k uses 20191006 + k, stream s adds 1000 * s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20191006

SD = (720, 576)
HD720 = (1280, 720)
FHD = (1920, 1080)
UHD = (3840, 2160)


def seed_for(workload: int, stream: int = 0) -> int:
    return BASE_SEED + workload + 1000 * stream


def quantise(v: np.ndarray) -> np.ndarray:
    return np.clip(np.floor(v + 0.5), 0, 255).astype(np.uint8)


@dataclass
class Texture:
    """Analytic texture over a rectangular domain [ox, ox+w) x [oy, oy+h)."""
    bx: np.ndarray
    by: np.ndarray
    bs: np.ndarray
    ba: np.ndarray
    gp: np.ndarray
    gth: np.ndarray
    ga: np.ndarray
    gphi: np.ndarray
    base: float = 128.0

    @staticmethod
    def draw(rng: np.random.Generator, w: float, h: float, ox: float = 0.0,
             oy: float = 0.0, n_blobs: int = 64, n_gratings: int = 3,
             sigma=(3.0, 20.0), amp=(40.0, 200.0), period=(8.0, 40.0),
             gamp=(10.0, 40.0)) -> "Texture":
        bx = ox + rng.uniform(0.0, w, n_blobs)
        by = oy + rng.uniform(0.0, h, n_blobs)
        bs = rng.uniform(sigma[0], sigma[1], n_blobs)
        ba = rng.uniform(amp[0], amp[1], n_blobs) * rng.choice([-1.0, 1.0], n_blobs)
        gp = rng.uniform(period[0], period[1], n_gratings)
        gth = rng.uniform(0.0, math.pi, n_gratings)
        ga = rng.uniform(gamp[0], gamp[1], n_gratings)
        gphi = rng.uniform(0.0, 2.0 * math.pi, n_gratings)
        return Texture(bx, by, bs, ba, gp, gth, ga, gphi)

    @staticmethod
    def low_frequency(rng: np.random.Generator, w: float, h: float) -> "Texture":
        """Variant with blob sigma >= 6 px, grating periods >= 24 px and blob
        amplitudes in [20, 60], so that the sum stays inside [0, 255] (no
        clipped plateaus) and the blob density scales with the area."""
        nb = max(8, int(round(64 * w * h / (720.0 * 576.0))))
        return Texture.draw(rng, w, h, n_blobs=nb, sigma=(6.0, 20.0), amp=(20.0, 60.0),
                            period=(24.0, 64.0))

    def evaluate(self, X: np.ndarray, Y: np.ndarray, margin: float | None = None,
                 px0: int = 0, py0: int = 0) -> np.ndarray:
        """T at texture coordinates (X, Y), clipped to [0, 255], in float64.

        X, Y are 2-D grids for the pixel block whose top-left pixel is
        (px0, py0).  If ``margin`` bounds |X - x| and |Y - y| over the block
        (x, y the pixel coordinates), blobs are evaluated only on the pixel
        windows they can reach, which gives the same values faster.
        """
        v = np.full(X.shape, self.base, dtype=np.float64)
        H, W = X.shape
        for s, a, cx, cy in zip(self.bs, self.ba, self.bx, self.by):
            r = 6.0 * s
            if margin is None:
                ys, xs = slice(0, H), slice(0, W)
            else:
                x_lo = max(0, int(math.floor(cx - r - margin)) - px0)
                x_hi = min(W, int(math.ceil(cx + r + margin)) + 1 - px0)
                y_lo = max(0, int(math.floor(cy - r - margin)) - py0)
                y_hi = min(H, int(math.ceil(cy + r + margin)) + 1 - py0)
                if x_lo >= x_hi or y_lo >= y_hi:
                    continue
                ys, xs = slice(y_lo, y_hi), slice(x_lo, x_hi)
            dx = X[ys, xs] - cx
            dy = Y[ys, xs] - cy
            r2 = dx * dx + dy * dy
            contrib = a * np.exp(-r2 / (2.0 * s * s))
            contrib[r2 > r * r] = 0.0
            v[ys, xs] += contrib
        for p, th, a, phi in zip(self.gp, self.gth, self.ga, self.gphi):
            v += a * np.sin(2.0 * math.pi * (X * math.cos(th) + Y * math.sin(th)) / p + phi)
        return np.clip(v, 0.0, 255.0)


def render_bilinear(w: int, h: int, coef=(10.0, 0.3, 0.2, 0.02), dx: float = 0.0,
                    dy: float = 0.0) -> np.ndarray:
    """Unquantised frame of the bilinear surface c0 + c1 x + c2 y + c3 x y
    moved by (dx, dy).  Bilinear interpolation reproduces such a surface
    exactly, which makes it a test input with a known exact answer."""
    X, Y = pixel_grid(w, h)
    X, Y = X - dx, Y - dy
    return coef[0] + coef[1] * X + coef[2] * Y + coef[3] * X * Y


def pixel_grid(w: int, h: int, x0: int = 0, y0: int = 0):
    ys, xs = np.mgrid[y0:y0 + h, x0:x0 + w]
    return xs.astype(np.float64), ys.astype(np.float64)


def render_shift(tex: Texture, w: int, h: int, dx: float = 0.0, dy: float = 0.0,
                 quantised: bool = True) -> np.ndarray:
    """Frame whose content is T moved by (dx, dy): value(x, y) = T(x - dx, y - dy)."""
    X, Y = pixel_grid(w, h)
    v = tex.evaluate(X - dx, Y - dy, margin=abs(dx) + abs(dy) + 1.0)
    return quantise(v) if quantised else v


def uniform_boxes(rng: np.random.Generator, w: int, h: int, n: int,
                  side=(40.0, 150.0)) -> np.ndarray:
    """n boxes (x0, y0, x1, y1) with independent sides ~ U[side], placed to fit."""
    bw = rng.uniform(side[0], side[1], n)
    bh = rng.uniform(side[0], side[1], n)
    x0 = rng.uniform(0.0, w - bw)
    y0 = rng.uniform(0.0, h - bh)
    return np.stack([x0, y0, x0 + bw, y0 + bh], axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# Workload 1: SD pair with a global sub-pixel shift
# --------------------------------------------------------------------------

@dataclass
class SDPair:
    frame0: np.ndarray
    frame1: np.ndarray
    boxes: np.ndarray
    shift: tuple
    texture: Texture


def sd_pair(shift=(1.37, -0.62), size=SD, n_boxes: int = 10, seed: int | None = None,
            low_frequency: bool = False, quantised: bool = True) -> SDPair:
    """720x576 pair: frame 1 is frame 0's texture moved by ``shift``."""
    rng = np.random.default_rng(seed_for(1) if seed is None else seed)
    w, h = size
    tex = Texture.low_frequency(rng, w, h) if low_frequency else Texture.draw(rng, w, h)
    boxes = uniform_boxes(rng, w, h, n_boxes)
    f0 = render_shift(tex, w, h, 0.0, 0.0, quantised)
    f1 = render_shift(tex, w, h, shift[0], shift[1], quantised)
    return SDPair(f0, f1, boxes, tuple(shift), tex)


# --------------------------------------------------------------------------
# Rigid textured regions composited over a background (workloads 2 and 4)
# --------------------------------------------------------------------------

@dataclass
class Region:
    w: float
    h: float
    cx: float
    cy: float
    theta: float = 0.0
    scale: float = 1.0
    tex: Texture | None = None

    def corners(self):
        c, s = math.cos(self.theta), math.sin(self.theta)
        hw, hh = 0.5 * self.w * self.scale, 0.5 * self.h * self.scale
        pts = [(-hw, -hh), (hw, -hh), (hw, hh), (-hw, hh)]
        return [(self.cx + c * u - s * v, self.cy + s * u + c * v) for u, v in pts]

    def bounds(self, W: int, H: int) -> np.ndarray:
        cs = self.corners()
        xs = [p[0] for p in cs]
        ys = [p[1] for p in cs]
        return np.array([max(0.0, min(xs)), max(0.0, min(ys)),
                         min(float(W), max(xs)), min(float(H), max(ys))], dtype=np.float32)


def composite(bg: Texture, regions, W: int, H: int, bg_shift=(0.0, 0.0),
              quantised: bool = True) -> np.ndarray:
    """Background moved by bg_shift, then each region pasted in index order."""
    X, Y = pixel_grid(W, H)
    v = bg.evaluate(X - bg_shift[0], Y - bg_shift[1],
                    margin=abs(bg_shift[0]) + abs(bg_shift[1]) + 1.0)
    for r in regions:
        b = r.bounds(W, H)
        x0, y0 = int(math.floor(b[0])), int(math.floor(b[1]))
        x1, y1 = int(math.ceil(b[2])) + 1, int(math.ceil(b[3])) + 1
        x0, y0, x1, y1 = max(0, x0), max(0, y0), min(W, x1), min(H, y1)
        if x0 >= x1 or y0 >= y1:
            continue
        Xs, Ys = X[y0:y1, x0:x1], Y[y0:y1, x0:x1]
        c, s = math.cos(r.theta), math.sin(r.theta)
        u = (c * (Xs - r.cx) + s * (Ys - r.cy)) / r.scale
        q = (-s * (Xs - r.cx) + c * (Ys - r.cy)) / r.scale
        inside = (np.abs(u) <= 0.5 * r.w) & (np.abs(q) <= 0.5 * r.h)
        if not inside.any():
            continue
        tv = r.tex.evaluate(u, q)
        blk = v[y0:y1, x0:x1]
        blk[inside] = tv[inside]
    return quantise(v) if quantised else v


@dataclass
class Clip:
    frames: list
    gt_boxes: list
    size: tuple


def affine_clip(n_frames: int = 64, size=FHD, n_rects: int = 16, seed: int | None = None,
                side=(60.0, 400.0)) -> Clip:
    """1080p clip: drifting background and 16 rectangles with seeded affine motion.

    Per frame the background moves by U[-2, 2]^2 px, and each rectangle takes a
    translation U[-8, 8]^2, a rotation U[-2, 2] deg and a scale factor
    U[0.98, 1.02]; cumulative scale stays in [0.7, 1.4] and centres reflect off
    the frame edges.  gt_boxes[t] are the rectangles' axis-aligned bounds.
    """
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    W, H = size
    bg = Texture.draw(rng, W + 200, H + 200, ox=-100, oy=-100)
    regs = []
    for _ in range(n_rects):
        w = rng.uniform(*side)
        h = rng.uniform(*side)
        cx = rng.uniform(0.5 * w, W - 0.5 * w) if W > w else 0.5 * W
        cy = rng.uniform(0.5 * h, H - 0.5 * h) if H > h else 0.5 * H
        tex = Texture.draw(rng, w, h, ox=-0.5 * w, oy=-0.5 * h)
        regs.append(Region(w, h, cx, cy, 0.0, 1.0, tex))
    bg_t = np.zeros(2)
    frames, gts = [], []
    for t in range(n_frames):
        if t > 0:
            bg_t = bg_t + rng.uniform(-2.0, 2.0, 2)
            for r in regs:
                d = rng.uniform(-8.0, 8.0, 2)
                r.theta += math.radians(rng.uniform(-2.0, 2.0))
                r.scale = float(np.clip(r.scale * rng.uniform(0.98, 1.02), 0.7, 1.4))
                nx, ny = r.cx + d[0], r.cy + d[1]
                if nx < 0.0 or nx > W:
                    nx = r.cx - d[0]
                if ny < 0.0 or ny > H:
                    ny = r.cy - d[1]
                r.cx, r.cy = nx, ny
        frames.append(composite(bg, regs, W, H, (bg_t[0], bg_t[1])))
        gts.append(np.stack([r.bounds(W, H) for r in regs]))
    return Clip(frames, gts, size)


@dataclass
class RigidPair:
    frame0: np.ndarray
    frame1: np.ndarray
    boxes: np.ndarray
    motions: np.ndarray  # per region (tx, ty, theta)


def rigid_pair(size=UHD, n_regions: int = 200, seed: int | None = None,
               side=(60.0, 300.0), max_t: float = 40.0, max_deg: float = 3.0) -> RigidPair:
    """4K pair: rigid regions over a static background, each moved by a
    translation U[-max_t, max_t]^2 and a rotation U[-max_deg, max_deg] about
    its centre.  Boxes are the regions' frame-0 bounds."""
    rng = np.random.default_rng(seed_for(4) if seed is None else seed)
    W, H = size
    bg = Texture.draw(rng, W, H)
    regs0, regs1, mot = [], [], []
    for _ in range(n_regions):
        w = rng.uniform(*side)
        h = rng.uniform(*side)
        cx = rng.uniform(0.5 * w, W - 0.5 * w)
        cy = rng.uniform(0.5 * h, H - 0.5 * h)
        tex = Texture.draw(rng, w, h, ox=-0.5 * w, oy=-0.5 * h)
        t = rng.uniform(-max_t, max_t, 2)
        th = math.radians(rng.uniform(-max_deg, max_deg))
        regs0.append(Region(w, h, cx, cy, 0.0, 1.0, tex))
        regs1.append(Region(w, h, cx + t[0], cy + t[1], th, 1.0, tex))
        mot.append((t[0], t[1], th))
    f0 = composite(bg, regs0, W, H)
    f1 = composite(bg, regs1, W, H)
    boxes = np.stack([r.bounds(W, H) for r in regs0])
    return RigidPair(f0, f1, boxes, np.array(mot))


# --------------------------------------------------------------------------
# Workload 3: many independent streams with a smooth warp
# --------------------------------------------------------------------------

@dataclass
class StreamPair:
    frame0: np.ndarray
    frame1: np.ndarray
    boxes: np.ndarray
    n_target: int
    size: tuple


def warp_field(rng: np.random.Generator, W: int, H: int):
    """Smooth displacement d(x, y) with |d| <= 12 px: a global translation
    U[-6, 6]^2 plus a low-frequency sinusoidal field of amplitude <= 6 px
    (3 / sqrt(2) per axis keeps the vector length bounded)."""
    t = rng.uniform(-6.0, 6.0, 2)
    amp = rng.uniform(0.0, 6.0 / math.sqrt(2.0), 2)
    lx = rng.uniform(0.5, 1.5, 2) * W
    ly = rng.uniform(0.5, 1.5, 2) * H
    ph = rng.uniform(0.0, 2.0 * math.pi, 2)

    def d(X, Y):
        dx = t[0] + amp[0] * np.sin(2 * math.pi * (X / lx[0] + Y / ly[0]) + ph[0])
        dy = t[1] + amp[1] * np.sin(2 * math.pi * (X / lx[1] - Y / ly[1]) + ph[1])
        return dx, dy
    return d


def stream_pair(stream: int, workload: int = 3, grid=(8, 8),
                sizes=(SD, HD720, FHD), n_range=(2000, 20000)) -> StreamPair:
    """One stream of the batched workload: frame 1 = T(x - d(x)) for a smooth
    field d, a grid of boxes tiling frame 0, and a target point count
    n = round(exp(U[ln 2000, ln 20000]))."""
    rng = np.random.default_rng(seed_for(workload, stream))
    W, H = sizes[int(rng.integers(0, len(sizes)))]
    n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
    tex = Texture.draw(rng, W + 40, H + 40, ox=-20, oy=-20, n_blobs=max(64, W * H // 6000))
    d = warp_field(rng, W, H)
    X, Y = pixel_grid(W, H)
    f0 = quantise(tex.evaluate(X, Y, margin=1.0))
    dx, dy = d(X, Y)
    f1 = quantise(tex.evaluate(X - dx, Y - dy, margin=13.0))
    gx, gy = grid
    xs = np.linspace(0.0, W, gx + 1)
    ys = np.linspace(0.0, H, gy + 1)
    boxes = np.array([[xs[i], ys[j], xs[i + 1], ys[j + 1]]
                      for j in range(gy) for i in range(gx)], dtype=np.float32)
    return StreamPair(f0, f1, boxes, n, (W, H))


def random_points(rng: np.random.Generator, n: int, W: int, H: int) -> np.ndarray:
    """n points uniform over [0, W-1] x [0, H-1] as float32 (x, y)."""
    return np.stack([rng.uniform(0.0, W - 1.0, n), rng.uniform(0.0, H - 1.0, n)],
                    axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# Workload 5: serving arrivals
# --------------------------------------------------------------------------

@dataclass
class ServeStream:
    stream: int
    size: tuple
    fps: float
    n_boxes: int
    refresh: int
    arrivals: np.ndarray = field(default_factory=lambda: np.zeros(0))


def serve_streams(n_streams: int = 64, duration_s: float = 60.0, workload: int = 5,
                  sizes=(SD, FHD, UHD), fps=(25.0, 60.0), boxes=(20, 300),
                  refresh=(5, 15)) -> list:
    """Per-stream resolution, rate, box count, detection refresh period and a
    Poisson arrival schedule (exponential inter-arrival times) over duration_s."""
    out = []
    for s in range(n_streams):
        rng = np.random.default_rng(seed_for(workload, s))
        size = sizes[int(rng.integers(0, len(sizes)))]
        rate = float(rng.uniform(*fps))
        nb = int(rng.integers(boxes[0], boxes[1] + 1))
        rf = int(rng.integers(refresh[0], refresh[1] + 1))
        n_exp = int(duration_s * rate * 1.5) + 16
        t = np.cumsum(rng.exponential(1.0 / rate, n_exp))
        out.append(ServeStream(s, size, rate, nb, rf, t[t < duration_s]))
    return out
