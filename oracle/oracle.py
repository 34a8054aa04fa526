"""ctypes front-end of the plain-C oracle (``rgbd_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Each wrapper names the
paper passage the C function follows; the C file holds the arithmetic.

Every function takes and returns numpy arrays.  The shared library is built
with gcc on first use (or by ``build()``), with IEEE arithmetic: no fast-math
and no floating-point contraction, so the fp32 quotient matches a correctly
rounded division on any host.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib", "rect_coord_q16", "crop", "median_nonzero", "valid_mask", "lbp_code",
    "lbp_codes", "uniform_table", "histograms", "features_batch", "normalize_f64",
    "normalize_f32", "sv_centre", "centre_rows", "f32_to_bf16", "f32_to_e4m3", "e4m3_to_f64", "svm_rbf", "svm_linear",
    "argmax", "track_nearest", "track_streams", "face_roi", "CALIB_DTYPE", "svm_train_rbf", "RECT_DTYPE", "LBP_GE", "LBP_NBR_IGNORE_MASK",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgbd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "librgbd_oracle.so")
_lock = threading.Lock()
_lib = None

LBP_GE = 1
LBP_NBR_IGNORE_MASK = 2

# {frame, x, y, w, h} as five int32, the same plain struct the C side reads.
RECT_DTYPE = np.dtype([("frame", "<i4"), ("x", "<i4"), ("y", "<i4"), ("w", "<i4"), ("h", "<i4")])


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/librgbd_oracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.orc_rect_coord_q16.restype = i64
            L.orc_rect_coord_q16.argtypes = [i32, i32, i32, i32]
            L.orc_crop.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P, P]
            L.orc_median_nonzero.restype = i32
            L.orc_median_nonzero.argtypes = [P, ctypes.c_int]
            L.orc_valid_mask.argtypes = [P, ctypes.c_int, i32, ctypes.c_int, P]
            L.orc_lbp_code.restype = ctypes.c_int
            L.orc_lbp_code.argtypes = [P, P] + [ctypes.c_int] * 5
            L.orc_uniform_table.argtypes = [P]
            L.orc_histograms.argtypes = [P, P] + [ctypes.c_int] * 5 + [P]
            L.orc_features_batch.argtypes = ([P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
                                             + [ctypes.c_int] * 7 + [P, P])
            L.orc_normalize_f64.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.orc_normalize_f32.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.orc_f32_to_bf16.restype = ctypes.c_uint16
            L.orc_f32_to_bf16.argtypes = [ctypes.c_float]
            L.orc_f32_to_e4m3.restype = ctypes.c_uint8
            L.orc_f32_to_e4m3.argtypes = [ctypes.c_float]
            L.orc_e4m3_to_f64.restype = dbl
            L.orc_e4m3_to_f64.argtypes = [ctypes.c_uint8]
            L.orc_svm_rbf.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, dbl, P]
            L.orc_svm_linear.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P]
            L.orc_argmax.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---- S1: affine resample (Section 2.1, Eq. 1) ---------------------------------------------

def rect_coord_q16(origin: int, length: int, out_len: int, i: int) -> int:
    """Q16.16 source coordinate of crop index i (pixel centre to pixel centre)."""
    return int(lib().orc_rect_coord_q16(origin, length, out_len, i))


def crop(grey, depth, rect, out_h, out_w, affine=None):
    """Bilinear grey / nearest depth crop of one rect {x, y, w, h} (frame ignored)."""
    grey = _c(grey, np.uint8)
    depth = _c(depth, np.uint16)
    H, W = grey.shape
    r = np.zeros(1, RECT_DTYPE)
    r["frame"], r["x"], r["y"], r["w"], r["h"] = 0, rect[0], rect[1], rect[2], rect[3]
    aff = None if affine is None else _c(affine, np.int32)
    og = np.zeros((out_h, out_w), np.uint8)
    od = np.zeros((out_h, out_w), np.uint16)
    lib().orc_crop(_p(grey), _p(depth), H, W, _p(r), _p(aff), out_h, out_w, _p(og), _p(od))
    return og, od


# ---- S2: depth mask ------------------------------------------------------------------------

def median_nonzero(d) -> int:
    """Lower median of the non-zero values (index floor((n-1)/2) of the sorted list), -1 if none."""
    d = _c(d, np.uint16).ravel()
    return int(lib().orc_median_nonzero(_p(d), d.size))


def valid_mask(d, median: int, mask_mm: int = 150):
    d = _c(d, np.uint16)
    out = np.zeros(d.shape, np.uint8)
    lib().orc_valid_mask(_p(d), d.size, median, mask_mm, _p(out))
    return out


# ---- S3: LBP codes (Eq. 2, Fig. 7) ----------------------------------------------------------

def lbp_code(g, valid, i, j, flags=0) -> int:
    g = _c(g, np.uint8)
    valid = _c(valid, np.uint8)
    h, w = g.shape
    return int(lib().orc_lbp_code(_p(g), _p(valid), h, w, i, j, flags))


def lbp_codes(g, valid, flags=0):
    """Code image (int32), -1 where the centre is not depth-valid."""
    g = _c(g, np.uint8)
    valid = _c(valid, np.uint8)
    h, w = g.shape
    out = np.full((h, w), -1, np.int32)
    L = lib()
    for i in range(h):
        for j in range(w):
            if valid[i, j]:
                out[i, j] = L.orc_lbp_code(_p(g), _p(valid), h, w, i, j, flags)
    return out


# ---- S4: histograms (Eq. 3) -----------------------------------------------------------------

def uniform_table():
    lut = np.zeros(256, np.int32)
    lib().orc_uniform_table(_p(lut))
    return lut


def histograms(g, valid, cell=8, nbins=59, flags=0):
    g = _c(g, np.uint8)
    valid = _c(valid, np.uint8)
    h, w = g.shape
    out = np.zeros((h // cell) * (w // cell) * nbins, np.uint16)
    lib().orc_histograms(_p(g), _p(valid), h, w, cell, nbins, flags, _p(out))
    return out


def features_batch(grey, depth, rects=None, out_h=128, out_w=None, cell=8, mask_mm=150,
                   nbins=59, flags=0, affine=None, return_medians=False):
    """Steps S1-S4 for a batch.

    grey: uint8 [F][H][W]; depth: uint16 [F][H][W]; rects: RECT_DTYPE [n] or None, in which
    case the frames are the crops themselves.  Returns uint16 [n][cells*nbins].
    """
    out_w = out_h if out_w is None else out_w
    grey = _c(grey, np.uint8)
    depth = _c(depth, np.uint16)
    F, H, W = grey.shape
    if rects is None:
        n = F
        assert (H, W) == (out_h, out_w)
        rp = None
    else:
        rects = np.ascontiguousarray(rects, RECT_DTYPE)
        n = rects.shape[0]
        rp = rects
    aff = None if affine is None else _c(affine, np.int32).reshape(n, 6)
    dim = (out_h // cell) * (out_w // cell) * nbins
    feats = np.zeros((n, dim), np.uint16)
    meds = np.zeros(n, np.int32)
    lib().orc_features_batch(_p(grey), _p(depth), F, H, W, _p(rp), _p(aff), n, out_h, out_w, cell,
                             mask_mm, nbins, flags, _p(feats), _p(meds))
    return (feats, meds) if return_medians else feats


# ---- S5: normalisation and SVM scores -------------------------------------------------------

def normalize_f64(feats, nbins=59):
    feats = _c(feats, np.uint16)
    n, dim = feats.shape
    out = np.zeros((n, dim), np.float64)
    lib().orc_normalize_f64(_p(feats), n, dim // nbins, nbins, _p(out))
    return out


def normalize_f32(feats, nbins=59):
    feats = _c(feats, np.uint16)
    n, dim = feats.shape
    out = np.zeros((n, dim), np.float32)
    lib().orc_normalize_f32(_p(feats), n, dim // nbins, nbins, _p(out))
    return out


def sv_centre(x32):
    """Column means of normalised fp32 rows (the centre of a model packed with centring): the
    fp64 sum of each column taken in row order, divided by the row count in fp64, rounded to
    fp32.  The RBF kernel of Section 2.5 depends only on differences of rows, so subtracting one
    vector from every row leaves it unchanged."""
    x = np.asarray(x32, np.float32).astype(np.float64)
    s = np.cumsum(x, axis=0)[-1]  # a running sum: strictly in row order
    return (s / np.float64(x.shape[0])).astype(np.float32)


def centre_rows(x32, mu):
    """x - mu per column in fp32 (one IEEE rounding)."""
    x = np.asarray(x32, np.float32)
    return (x - np.asarray(mu, np.float32)[: x.shape[1]]).astype(np.float32)


def f32_to_bf16(x):
    """Bit patterns (uint16) of round-to-nearest-even bfloat16."""
    x = _c(x, np.float32)
    L = lib()
    return np.array([L.orc_f32_to_bf16(float(v)) for v in x.ravel()], np.uint16).reshape(x.shape)


def f32_to_e4m3(x):
    """Bit patterns (uint8) of saturating round-to-nearest-even FP8 E4M3."""
    x = _c(x, np.float32)
    L = lib()
    return np.array([L.orc_f32_to_e4m3(float(v)) for v in x.ravel()], np.uint8).reshape(x.shape)


def e4m3_to_f64(b):
    b = _c(b, np.uint8)
    L = lib()
    return np.array([L.orc_e4m3_to_f64(int(v)) for v in b.ravel()], np.float64).reshape(b.shape)


def svm_rbf(x, sv, a, b, gamma):
    """S[k][c] = sum_i a[c][i] exp(-gamma |x_k - sv_i|^2) + b[c]  (fp64, direct distances)."""
    x = _c(x, np.float64)
    sv = _c(sv, np.float64)
    a = _c(a, np.float64)
    b = _c(b, np.float64)
    n, dim = x.shape
    n_sv = sv.shape[0]
    C = a.shape[0]
    assert sv.shape[1] == dim and a.shape[1] == n_sv and b.shape == (C,)
    out = np.zeros((n, C), np.float64)
    lib().orc_svm_rbf(_p(x), n, _p(sv), n_sv, dim, _p(a), _p(b), C, float(gamma), _p(out))
    return out


def svm_linear(x, w, b):
    x = _c(x, np.float64)
    w = _c(w, np.float64)
    b = _c(b, np.float64)
    n, dim = x.shape
    C = w.shape[0]
    out = np.zeros((n, C), np.float64)
    lib().orc_svm_linear(_p(x), n, dim, _p(w), _p(b), C, _p(out))
    return out


def argmax(scores):
    scores = _c(scores, np.float64)
    n, C = scores.shape
    out = np.zeros(n, np.int32)
    lib().orc_argmax(_p(scores), n, C, _p(out))
    return out


# ---- Section 2.3: nearest-centre tracking ---------------------------------------------------

def svm_train_rbf(x64, labels, n_classes, gamma, cost=1.0, eps=1e-3, max_iter=100000):
    """One-vs-rest RBF SVM by SMO (maximal violating pair) in fp64.  x64 float64 [n][dim] (the
    normalised rows).  Returns (a [C][n] = y * alpha, b [C], iterations [C])."""
    x64 = np.ascontiguousarray(x64, np.float64)
    n, dim = x64.shape
    lab = np.ascontiguousarray(labels, np.int32)
    a = np.zeros((n_classes, n), np.float64)
    b = np.zeros(n_classes, np.float64)
    it = np.zeros(n_classes, np.int32)
    L = lib()
    L.orc_svm_train_rbf.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_svm_train_rbf(_p(x64), n, dim, _p(lab), n_classes, gamma, cost, eps, max_iter, _p(a), _p(b), _p(it))
    return a, b, it


CALIB_DTYPE = np.dtype([("a", np.int32, 6), ("parallax", np.int32), ("d_min", np.int32), ("d_max", np.int32),
                        ("colour_w", np.int32), ("colour_h", np.int32)])


def face_roi(depth, calib, rects):
    """Depth-space bounding rects of colour-detected faces (Section 2.1).  depth uint16
    [F][H][W]; calib a CALIB_DTYPE record; rects RECT_DTYPE [n] in colour pixels."""
    depth = np.ascontiguousarray(depth, np.uint16)
    if depth.ndim == 2:
        depth = depth[None]
    F, H, W = depth.shape
    rects = np.ascontiguousarray(rects, RECT_DTYPE)
    cal = np.ascontiguousarray(np.asarray(calib, CALIB_DTYPE).reshape(1))
    out = np.zeros(len(rects), RECT_DTYPE)
    L = lib()
    L.orc_face_roi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.orc_face_roi(_p(depth), F, H, W, _p(cal), _p(rects), len(rects), _p(out))
    return out


def track_streams(state, frame_stream, frame_start, rects, labels):
    """Per-stream tracking over a batch (Section 2.3); `state` = dict(rects [S][M] RECT_DTYPE,
    ids int32 [S][M], count int32 [S]) is updated in place.  Returns int32 ids [n]."""
    rects = np.ascontiguousarray(rects, RECT_DTYPE)
    labels = np.ascontiguousarray(labels, np.int32)
    fs = np.ascontiguousarray(frame_stream, np.int32)
    st = np.ascontiguousarray(frame_start, np.int32)
    S, M = state["ids"].shape
    for k in ("rects", "ids", "count"):
        assert state[k].flags["C_CONTIGUOUS"]
    L = lib()
    L.orc_track_streams.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 5
    ids = np.zeros(len(rects), np.int32)
    L.orc_track_streams(_p(state["rects"]), _p(state["ids"]), _p(state["count"]), S, M, len(fs), _p(fs), _p(st),
                        _p(rects), _p(labels), _p(ids))
    return ids


def track_nearest(prev, cur):
    """For each previous rect, the index of the nearest current rect of the same stream, or -1."""
    prev = np.ascontiguousarray(prev, RECT_DTYPE)
    cur = np.ascontiguousarray(cur, RECT_DTYPE)
    L = lib()
    L.orc_track_nearest.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    out = np.zeros(len(prev), np.int32)
    L.orc_track_nearest(_p(prev), len(prev), _p(cur), len(cur), _p(out))
    return out
