"""Seeded synthetic RGB-D workloads.

The paper's Kinect recordings are not public, so these generators stand in for
them with the shapes of the five workloads this library is measured on: a
64x64 single crop, one 640x480 frame with 4 faces, a 256-frame batch of 4096
faces, a 65536 x 16384 scoring problem and a 32-stream serving mix.

This module holds no arithmetic of the method (no resampling, masking, LBP,
histogramming, normalisation or scoring).  It only draws inputs, and it is the
one module that both the CUDA path and the CPU oracle's tests read.  All draws
come from ``numpy.random.Generator(PCG64(seed))``; the default seed of
workload i is 1504 + i.

Recipe (per face):
  grey  -- smooth radial gradient + 6 Gaussian blobs (sigma 3-8 px at 64 px,
           scaled with the face side) + N(0, 8) noise, clipped to 0..255.
  depth -- ellipsoid face surface: base distance U(1000, 1100) mm minus a relief
           of U(60, 100) mm, semi-axes U(0.42, 0.5) x side (so the face covers more
           than half of its rect); background drawn per pixel from U(2500, 4000)
           mm; 2 % of pixels are zero holes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

RECT_DTYPE = np.dtype([("frame", "<i4"), ("x", "<i4"), ("y", "<i4"), ("w", "<i4"), ("h", "<i4")])

FRAME_H, FRAME_W = 480, 640
CELL = 8
NBINS = 59


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------------------------
# Single crops (64x64 plain case)
# ---------------------------------------------------------------------------------------------

def _blobs(rng, img, x0, y0, side, count=6):
    """Add `count` Gaussian blobs inside the square [x0, x0+side) x [y0, y0+side)."""
    H, W = img.shape
    scale = side / 64.0
    for _ in range(count):
        cx = x0 + rng.uniform(0.1, 0.9) * side
        cy = y0 + rng.uniform(0.1, 0.9) * side
        sig = rng.uniform(3.0, 8.0) * scale
        amp = rng.uniform(-70.0, 70.0)
        r = int(np.ceil(3 * sig))
        xa, xb = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        ya, yb = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb]
        img[ya:yb, xa:xb] += amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))


def _radial(rng, H, W):
    cx = W / 2 + rng.uniform(-W / 8, W / 8)
    cy = H / 2 + rng.uniform(-H / 8, H / 8)
    base = rng.uniform(60.0, 160.0)
    amp = rng.uniform(30.0, 80.0)
    yy, xx = np.mgrid[0:H, 0:W]
    r = np.sqrt((xx - cx) ** 2 + (yy - cy) ** 2) / (0.5 * max(H, W))
    return base + amp * (1.0 - r)


def _face_depth(rng, depth, x0, y0, side):
    """Write an ellipsoid face under the square rect (keeps the nearer surface)."""
    H, W = depth.shape
    cx = x0 + side / 2 + rng.uniform(-0.03, 0.03) * side
    cy = y0 + side / 2 + rng.uniform(-0.03, 0.03) * side
    ax = rng.uniform(0.42, 0.5) * side
    ay = rng.uniform(0.42, 0.5) * side
    base = rng.uniform(1000.0, 1100.0)
    relief = rng.uniform(60.0, 100.0)
    xa, xb = max(0, int(np.floor(cx - ax))), min(W, int(np.ceil(cx + ax)) + 1)
    ya, yb = max(0, int(np.floor(cy - ay))), min(H, int(np.ceil(cy + ay)) + 1)
    if xa >= xb or ya >= yb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb]
    rho2 = ((xx + 0.5 - cx) / ax) ** 2 + ((yy + 0.5 - cy) / ay) ** 2
    inside = rho2 < 1.0
    surf = base - relief * np.sqrt(np.clip(1.0 - rho2, 0.0, 1.0))
    win = depth[ya:yb, xa:xb]
    win[inside] = np.minimum(win[inside], surf[inside])


def _holes(rng, depth, frac=0.02):
    m = rng.random(depth.shape) < frac
    depth[m] = 0


def grey_crop(rng, side=64):
    img = _radial(rng, side, side)
    _blobs(rng, img, 0, 0, side)
    img += rng.normal(0.0, 8.0, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def depth_crop(rng, side=64):
    d = rng.uniform(2500.0, 4000.0, (side, side))
    _face_depth(rng, d, 0, 0, side)
    d = np.rint(d)
    _holes(rng, d)
    return d.astype(np.uint16)


def crops(seed, n, side=64):
    """n aligned (grey uint8, depth uint16) crops of side x side: arrays [n][side][side]."""
    rng = rng_for(seed)
    g = np.stack([grey_crop(rng, side) for _ in range(n)])
    d = np.stack([depth_crop(rng, side) for _ in range(n)])
    return g, d


# ---------------------------------------------------------------------------------------------
# Frames with face rects
# ---------------------------------------------------------------------------------------------

def rects_for_frame(rng, n, frame, smin, smax, H=FRAME_H, W=FRAME_W):
    """n square rects, side ~ U{smin..smax}; centres inside the frame, so a rect may stick out."""
    r = np.zeros(n, RECT_DTYPE)
    for k in range(n):
        s = int(rng.integers(smin, smax + 1))
        cx = int(rng.integers(0, W))
        cy = int(rng.integers(0, H))
        r[k] = (frame, cx - s // 2, cy - s // 2, s, s)
    return r


def frame_pair(rng, rects, H=FRAME_H, W=FRAME_W):
    """One grey uint8 / depth uint16 frame with a face drawn under each rect."""
    g = _radial(rng, H, W)
    d = rng.uniform(2500.0, 4000.0, (H, W))
    for r in rects:
        _blobs(rng, g, int(r["x"]), int(r["y"]), int(r["w"]))
        _face_depth(rng, d, int(r["x"]), int(r["y"]), int(r["w"]))
    g += rng.normal(0.0, 8.0, g.shape)
    d = np.rint(d)
    _holes(rng, d)
    return np.clip(np.rint(g), 0, 255).astype(np.uint8), d.astype(np.uint16)


def frames_with_rects(seed, n_frames, per_frame, smin, smax, H=FRAME_H, W=FRAME_W):
    """Frames [F][H][W] (uint8, uint16) and rects [F*per_frame] (per_frame may be a list)."""
    rng = rng_for(seed)
    greys, depths, rects = [], [], []
    for f in range(n_frames):
        k = per_frame[f] if isinstance(per_frame, (list, tuple, np.ndarray)) else per_frame
        r = rects_for_frame(rng, int(k), f, smin, smax, H, W)
        g, d = frame_pair(rng, r, H, W)
        greys.append(g)
        depths.append(d)
        rects.append(r)
    return np.stack(greys), np.stack(depths), np.concatenate(rects)


# ---------------------------------------------------------------------------------------------
# Depth-to-colour calibration and colour-image face boxes (inputs of the region-of-interest step)
# ---------------------------------------------------------------------------------------------

CALIB_FIELDS = np.dtype([("a", np.int32, 6), ("parallax", np.int32), ("d_min", np.int32), ("d_max", np.int32),
                         ("colour_w", np.int32), ("colour_h", np.int32)])


def calibration(rng, colour_w=FRAME_W, colour_h=FRAME_H):
    """Parameters of a depth-to-colour pixel mapping standing in for an RGB-D camera's: scale
    1 +- 3 %, shear up to 1 %, offsets up to 8 px (all Q16.16), a stereo shift of 20-30 px at
    1 m (in 1/256 px x mm) and a valid range of 400-8000 mm."""
    c = np.zeros((), CALIB_FIELDS)
    c["a"] = [int(65536 * rng.uniform(0.97, 1.03)), int(65536 * rng.uniform(-0.01, 0.01)),
              int(65536 * rng.uniform(-8, 8)), int(65536 * rng.uniform(-0.01, 0.01)),
              int(65536 * rng.uniform(0.97, 1.03)), int(65536 * rng.uniform(-8, 8))]
    c["parallax"] = int(rng.uniform(20, 30) * 1000 * 256)
    c["d_min"], c["d_max"] = 400, 8000
    c["colour_w"], c["colour_h"] = colour_w, colour_h
    return c


def colour_boxes(rng, rects):
    """Detector boxes in the colour image for faces drawn under `rects` (depth pixels): shifted
    right by 15-35 px (the stereo offset at face distance) and by up to 5 px vertically, side
    within 5 %."""
    out = rects.copy()
    n = len(rects)
    out["x"] = rects["x"] + rng.integers(15, 36, n)
    out["y"] = rects["y"] + rng.integers(-5, 6, n)
    side = np.maximum(8, np.rint(rects["w"] * rng.uniform(0.95, 1.05, n))).astype(np.int32)
    out["w"] = side
    out["h"] = side
    return out


# ---------------------------------------------------------------------------------------------
# SVM models and histogram-like count rows
# ---------------------------------------------------------------------------------------------

def poisson_counts(rng, n, dim, lam=3.0):
    """Histogram-like uint16 count rows [n][dim] (Poisson(lam) per bin)."""
    return rng.poisson(lam, (n, dim)).astype(np.uint16)


def poisson_counts_device(seed, n, dim, device, lam=3.0, chunk=4096):
    """The same kind of rows drawn on the GPU with a seeded torch generator (for the
    65536-row scoring workload, too large to draw on the host quickly).  Returns int16
    storage of the uint16 counts, [n][dim]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((n, dim), dtype=torch.int16, device=device)
    rate = torch.full((min(chunk, n), dim), float(lam), device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        out[r0:r1] = torch.poisson(rate[: r1 - r0], generator=g).to(torch.int16)
    return out


def rbf_coefficients(rng, n_classes, n_sv):
    """a[c][i] = alpha_ci * y_ci ~ N(0,1), shifted so each class sums to 0 (the KKT
    equality sum_i alpha_i y_i = 0 of a trained SVM); biases are 0."""
    a = rng.normal(0.0, 1.0, (n_classes, n_sv))
    a -= a.mean(axis=1, keepdims=True)
    return a.astype(np.float32), np.zeros(n_classes, np.float32)


def linear_model(rng, n_classes, dim):
    w = rng.normal(0.0, 1.0, (n_classes, dim)).astype(np.float32)
    b = rng.normal(0.0, 1.0, n_classes).astype(np.float32)
    return w, b


# ---------------------------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    crop: int
    grey: np.ndarray = None          # [F][H][W] uint8 (frames or pre-cut crops)
    depth: np.ndarray = None         # [F][H][W] uint16
    rects: np.ndarray | None = None  # RECT_DTYPE [n] or None for pre-cut crops
    kernel: str = "rbf"              # "rbf" or "linear"
    sv_counts: np.ndarray | None = None  # uint16 [n_sv][dim]
    coef: np.ndarray | None = None   # rbf: a [C][n_sv]; linear: w [C][dim]
    bias: np.ndarray | None = None   # [C]
    gamma: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return (self.crop // CELL) ** 2 * NBINS

    @property
    def n_crops(self):
        return self.grey.shape[0] if self.rects is None else self.rects.shape[0]


def plain_crop(seed=1504):
    """64x64 crop, 8x8 cells (3776-dim), linear SVM with 5 classes."""
    g, d = crops(seed, 1, 64)
    rng = rng_for(seed + 10_000)
    dim = 8 * 8 * NBINS
    w, b = linear_model(rng, 5, dim)
    return Workload("plain-64x64-crop/linear-5", 64, g, d, None, "linear", None, w, b, 0.0)


def single_frame(seed=1505):
    """One 640x480 frame, 4 faces of 80-200 px -> 128x128 (15104-dim), RBF 512 SV x 10 classes."""
    g, d, r = frames_with_rects(seed, 1, 4, 80, 200)
    rng = rng_for(seed + 10_000)
    dim = 16 * 16 * NBINS
    sv = poisson_counts(rng, 512, dim)
    a, b = rbf_coefficients(rng, 10, 512)
    return Workload("frame-640x480-4faces/rbf-512sv-10c", 128, g, d, r, "rbf", sv, a, b, 1.0 / dim)


def batching(seed=1506, n_frames=256, per_frame=16, n_sv=4096, n_classes=64):
    """256 frames, 4096 faces of side U{48..256} -> 128x128, RBF 4096 SV x 64 classes."""
    g, d, r = frames_with_rects(seed, n_frames, per_frame, 48, 256)
    rng = rng_for(seed + 10_000)
    dim = 16 * 16 * NBINS
    sv = poisson_counts(rng, n_sv, dim)
    a, b = rbf_coefficients(rng, n_classes, n_sv)
    return Workload(f"batch-{n_frames}x640x480-{r.shape[0]}faces/rbf-{n_sv}sv-{n_classes}c", 128,
                    g, d, r, "rbf", sv, a, b, 1.0 / dim)


def serving_arrivals(seed=1508, n_streams=32, fps=30.0, seconds=10.0, fmin=1, fmax=12):
    """Poisson frame arrivals of n_streams cameras: list of (t_arrival_s, stream, n_faces)."""
    rng = rng_for(seed)
    events = []
    for s in range(n_streams):
        t = rng.exponential(1.0 / fps)
        while t < seconds:
            events.append((t, s, int(rng.integers(fmin, fmax + 1))))
            t += rng.exponential(1.0 / fps)
    events.sort()
    return events
