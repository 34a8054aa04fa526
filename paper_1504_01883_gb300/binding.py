"""Thin Python binding of ``librgbdlbp.so`` (argument marshalling only).

Every function here has the name of a C entry point in ``include/rgbd_lbp.h``
and does nothing but check tensor shapes / dtypes, allocate outputs with torch
(device memory is torch's), and pass raw pointers plus torch's current CUDA
stream to the library.  All arithmetic of the method runs in the library's
kernels.  If the library has not been built, ``lib()`` raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librgbdlbp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rgbd_lbp.h")

RGBD_OK = 0
DT_F32, DT_BF16, DT_FP8, DT_TF32, DT_BF16X3 = 1, 2, 3, 4, 5
DT_CENTRED = 0x100  # svm_train_data_pack flag: SVs stored relative to their mean
KERNEL_LINEAR, KERNEL_RBF = 0, 1
LBP_GE, LBP_NBR_IGNORE_MASK, LBP_FACE_HIST256 = 1, 2, 4
TUNE_LBP_CTAS_PER_SM, TUNE_TC_SPLITS, TUNE_TC_PAIRING, TUNE_LBP_SHAPE, TUNE_TC_SPLITK = 1, 2, 3, 4, 5
STATUS_BAD_RECT, STATUS_WAIT_TIMEOUT = 1, 2
NBINS, CELL = 59, 8

_DT_NAMES = {"f32": DT_F32, "fp32": DT_F32, "bf16": DT_BF16, "fp8": DT_FP8, "e4m3": DT_FP8, "tf32": DT_TF32,
             "bf16x3": DT_BF16X3}
_lib = None


class RgbdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rgbd error {code}: {msg}")
        self.code = code


class SvmInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n_sv", ctypes.c_int32),
                ("n_sv_pad", ctypes.c_int32), ("dim", ctypes.c_int32), ("k_pad", ctypes.c_int32),
                ("n_classes", ctypes.c_int32), ("scorable", ctypes.c_int32), ("gamma", ctypes.c_float),
                ("sv_scale", ctypes.c_float), ("centred", ctypes.c_int32)]


def declared_functions(header: str = HEADER):
    """Names of the functions the C header declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+([a-z_0-9]+)\s*\(", text, flags=re.M)))


def lib():
    """The loaded library; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, F, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        sig = {
            "rgbd_version": [],
            "rgbd_last_error": [P, Z],
            "rgbd_ctx_create": [I, P],
            "rgbd_ctx_destroy": [P],
            "rgbd_ctx_reserve": [P, Z],
            "rgbd_ctx_status": [P, P, I],
            "rgbd_crop_affine": [P, P, P, I, I, I, P, P, I, I, I, P, P, P],
            "lbp_fused_features": [P, P, P, I, I, I, P, P, I, I, I, I, I, P, I, P, I, F, P, P, P],
            "lbp_normalize_features": [P, P, I, I, I, I, P, I, F, P, P, P],
            "svm_train_data_pack": [P, P, I, I, I, P, P, I, I, F, I, P, P],
            "rgbd_svm_free": [P],
            "rgbd_svm_get_info": [P, P],
            "rgbd_svm_packed_sv": [P, P, P],
            "rgbd_svm_centre": [P, P],
            "svm_score": [P, P, P, P, I, F, P, P, P],
            "rgbd_ctx_set_tuning": [P, I, I],
            "rgbd_track_nearest": [P, P, I, P, I, P, P],
            "rgbd_debug_expm1": [P, P, I, P],
            "rgbd_debug_wait_timeout": [P, ctypes.c_uint64, P, P],
            "rgbd_face_roi": [P, P, I, I, I, P, P, I, P, P],
            "svm_train_rbf": [P, P, P, I, I, P, I, F, F, F, I, P, P, P, P],
            "rgbd_track_streams": [P, P, P, P, I, I, I, P, P, P, I, P, P, P],
            "rgbd_server_create": [P, P, P],
            "rgbd_server_submit": [P, I, P, P, P, I, P, P, P, P],
            "rgbd_server_poll": [P, P, I, P, I],
            "rgbd_server_stats": [P, P, P, P, P],
            "rgbd_server_destroy": [P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().rgbd_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc):
    if rc != RGBD_OK:
        raise RgbdError(rc, last_error())


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _centre(c):
    """x_centre argument: None, a device float tensor, or a model packed with DT_CENTRED."""
    if c is None:
        return None
    if isinstance(c, SvmModel):
        ptr = c.centre_ptr()
        if ptr is None:
            raise ValueError("the model was packed without DT_CENTRED")
        return ctypes.c_void_p(ptr)
    if c.dtype != torch.float32:
        raise ValueError("x_centre must be float32")
    return _p(c)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dt(x):
    if x is None or x == 0:
        return 0
    if isinstance(x, str):
        return _DT_NAMES[x.lower()]
    return int(x)


def x_torch_dtype(dt):
    dt = _dt(dt)
    return {DT_F32: torch.float32, DT_TF32: torch.float32, DT_BF16: torch.bfloat16, DT_FP8: torch.uint8,
            DT_BF16X3: torch.bfloat16}[dt]


def x_shape(dt, n, k_pad):
    """Shape of a normalised-row buffer: split bf16 rows are two planes (hi, then lo)."""
    return (2, n, k_pad) if _dt(dt) == DT_BF16X3 else (n, k_pad)


def k_pad_for(dim: int) -> int:
    return (dim + 127) // 128 * 128


class Context:
    """rgbd_ctx: status word and workspace of one device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check(lib().rgbd_ctx_create(device, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().rgbd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nbytes: int):
        _check(lib().rgbd_ctx_reserve(self.handle, ctypes.c_size_t(nbytes)))

    def set_tuning(self, key: int, value: int):
        _check(lib().rgbd_ctx_set_tuning(self.handle, int(key), int(value)))

    def status(self, clear: bool = True) -> int:
        v = ctypes.c_uint32(0)
        _check(lib().rgbd_ctx_status(self.handle, ctypes.byref(v), 1 if clear else 0))
        return v.value


def rects_tensor(rects, device="cuda"):
    """rects: numpy structured array (frame, x, y, w, h) or an int array [n][5] -> int32 [n][5]."""
    import numpy as np
    if isinstance(rects, torch.Tensor):
        return rects.to(device=device, dtype=torch.int32).contiguous()
    a = np.asarray(rects)
    if a.dtype.names:
        a = np.stack([a[k] for k in ("frame", "x", "y", "w", "h")], axis=1)
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device=device)


def rgbd_crop_affine(ctx, grey, depth, rects, out_h, out_w, affine=None, out_grey=None, out_depth=None,
                     stream=None):
    F, H, W = grey.shape
    n = rects.shape[0]
    if out_grey is None:
        out_grey = torch.empty((n, out_h, out_w), dtype=torch.uint8, device=grey.device)
    if out_depth is None:
        out_depth = torch.empty((n, out_h, out_w), dtype=torch.int16, device=grey.device)
    _check(lib().rgbd_crop_affine(ctx.handle, _p(grey), _p(depth), F, H, W, _p(rects), _p(affine), n, out_h,
                                  out_w, _p(out_grey), _p(out_depth), _stream(stream)))
    return out_grey, out_depth


def lbp_fused_features(ctx, grey, depth, rects=None, crop=128, cell=CELL, mask_mm=150, flags=0, feats=True,
                       x_dtype=0, k_pad=None, x_scale=448.0, xsq=True, affine=None, out=None, x_centre=None,
                       stream=None):
    """Returns (feats uint16-as-int16 [n][dim] or None, x [n][k_pad] or None, xsq [n] or None)."""
    F, H, W = grey.shape
    n = F if rects is None else rects.shape[0]
    if flags & LBP_FACE_HIST256:
        cell = crop  # one histogram over the whole face
    dim = 256 if flags & LBP_FACE_HIST256 else (crop // cell) ** 2 * NBINS
    dt = _dt(x_dtype)
    k_pad = k_pad_for(dim) if k_pad is None else k_pad
    out = out or {}
    f = out.get("feats")
    if feats and f is None:
        f = torch.empty((n, dim), dtype=torch.int16, device=grey.device)
    x = out.get("x")
    if dt and x is None:
        x = torch.empty(x_shape(dt, n, k_pad), dtype=x_torch_dtype(dt), device=grey.device)
    q = out.get("xsq")
    if dt and xsq and q is None:
        q = torch.empty((n,), dtype=torch.float32, device=grey.device)
    _check(lib().lbp_fused_features(ctx.handle, _p(grey), _p(depth), F, H, W, _p(rects), _p(affine), n, crop, cell,
                                    mask_mm, flags, _p(f) if feats else None, dt, _p(x) if dt else None, k_pad,
                                    float(x_scale), _centre(x_centre), _p(q) if (dt and xsq) else None,
                                    _stream(stream)))
    return (f if feats else None), (x if dt else None), (q if (dt and xsq) else None)


def rgbd_track_nearest(ctx, prev, cur, match=None, stream=None):
    """prev, cur: int32 [n][5] rects (frame = stream id).  Returns int32 [n_prev] indices into cur."""
    n_prev, n_cur = prev.shape[0], cur.shape[0]
    if match is None:
        match = torch.empty((n_prev,), dtype=torch.int32, device=prev.device)
    _check(lib().rgbd_track_nearest(ctx.handle, _p(prev), n_prev, _p(cur) if n_cur else None, n_cur, _p(match),
                                    _stream(stream)))
    return match


def svm_train_rbf(ctx, x, xsq, labels, n_classes, gamma, cost=1.0, eps=1e-3, max_iter=200000, stream=None):
    """One-vs-rest RBF SVM training (SMO) on normalised fp32 rows x [n][k_pad] with norms xsq [n]
    and int32 labels [n] (all CUDA).  Returns (coef [C][n], bias [C], iters [C])."""
    n, k_pad = x.shape
    coef = torch.empty((n_classes, n), dtype=torch.float32, device=x.device)
    bias = torch.empty((n_classes,), dtype=torch.float32, device=x.device)
    iters = torch.empty((n_classes,), dtype=torch.int32, device=x.device)
    _check(lib().svm_train_rbf(ctx.handle, _p(x), _p(xsq), n, k_pad, _p(labels), n_classes, gamma, cost, eps,
                               max_iter, _p(coef), _p(bias), _p(iters), _stream(stream)))
    return coef, bias, iters


class Calib(ctypes.Structure):
    """rgbd_calib: depth-to-colour mapping (see rgbd_face_roi)."""
    _fields_ = [("a", ctypes.c_int32 * 6), ("parallax", ctypes.c_int32), ("d_min", ctypes.c_int32),
                ("d_max", ctypes.c_int32), ("colour_w", ctypes.c_int32), ("colour_h", ctypes.c_int32)]

    @classmethod
    def from_record(cls, rec):
        """From a record with fields a[6], parallax, d_min, d_max, colour_w, colour_h."""
        c = cls()
        for i in range(6):
            c.a[i] = int(rec["a"][i])
        for f in ("parallax", "d_min", "d_max", "colour_w", "colour_h"):
            setattr(c, f, int(rec[f]))
        return c


def rgbd_face_roi(ctx, depth, calib, colour_rects, out=None, stream=None):
    """Depth-space rects of colour-detected faces (Section 2.1).  depth int16/uint16 [F][H][W]
    (CUDA), calib a Calib, colour_rects int32 [n][5] (CUDA).  Returns int32 [n][5]."""
    F, H, W = depth.shape
    n = colour_rects.shape[0]
    if out is None:
        out = torch.empty((n, 5), dtype=torch.int32, device=depth.device)
    _check(lib().rgbd_face_roi(ctx.handle, _p(depth), F, H, W, ctypes.addressof(calib), _p(colour_rects) if n else None,
                               n, _p(out) if n else None, _stream(stream)))
    return out


class TrackState:
    """Device-resident per-stream tracking state: the rects of each stream's last served frame
    and the identities of those faces (see rgbd_track_streams)."""

    def __init__(self, n_streams, max_faces=64, device=None):
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.n_streams, self.max_faces = n_streams, max_faces
        self.rects = torch.zeros((n_streams, max_faces, 5), dtype=torch.int32, device=dev)
        self.ids = torch.full((n_streams, max_faces), -1, dtype=torch.int32, device=dev)
        self.count = torch.zeros((n_streams,), dtype=torch.int32, device=dev)


def rgbd_track_streams(ctx, state, frame_stream, frame_start, rects, labels, ids=None, stream=None):
    """Identities of a batch's faces from each stream's previous frame (Section 2.3); updates
    `state` (a TrackState).  frame_stream int32 [F], frame_start int32 [F + 1], rects int32 [n][5],
    labels int32 [n] (all CUDA).  Returns ids int32 [n]."""
    n = rects.shape[0]
    if ids is None:
        ids = torch.empty((n,), dtype=torch.int32, device=rects.device)
    _check(lib().rgbd_track_streams(ctx.handle, _p(state.rects), _p(state.ids), _p(state.count), state.n_streams,
                                    state.max_faces, frame_stream.shape[0], _p(frame_stream), _p(frame_start),
                                    _p(rects) if n else None, n, _p(labels) if n else None, _p(ids) if n else None,
                                    _stream(stream)))
    return ids


def rgbd_debug_wait_timeout(ctx, limit_ns, stream=None):
    """Runs the scoring kernel's bounded wait on a barrier nothing completes; returns the device
    result (1 = the wait gave up after limit_ns and flagged RGBD_STATUS_WAIT_TIMEOUT)."""
    res = torch.full((1,), -1, dtype=torch.int32, device=torch.device("cuda", ctx.device))
    _check(lib().rgbd_debug_wait_timeout(ctx.handle, int(limit_ns), _p(res), _stream(stream)))
    return res


def rgbd_debug_expm1(z, stream=None):
    """e^z - 1 as the tensor-core epilogue evaluates it (z: float32 CUDA tensor)."""
    z = z.contiguous()
    out = torch.empty_like(z)
    _check(lib().rgbd_debug_expm1(_p(z), _p(out), z.numel(), _stream(stream)))
    return out


def lbp_normalize_features(ctx, feats, x_dtype, k_pad=None, x_scale=448.0, nbins=NBINS, x_centre=None,
                           stream=None):
    n, dim = feats.shape
    dt = _dt(x_dtype)
    k_pad = k_pad_for(dim) if k_pad is None else k_pad
    x = torch.empty(x_shape(dt, n, k_pad), dtype=x_torch_dtype(dt), device=feats.device)
    q = torch.empty((n,), dtype=torch.float32, device=feats.device)
    _check(lib().lbp_normalize_features(ctx.handle, _p(feats), n, dim, nbins, dt, _p(x), k_pad, float(x_scale),
                                        _centre(x_centre), _p(q), _stream(stream)))
    return x, q


class SvmModel:
    """rgbd_svm: a packed, device-resident SVM."""

    def __init__(self, handle):
        self.handle = handle
        info = SvmInfo()
        _check(lib().rgbd_svm_get_info(handle, ctypes.byref(info)))
        self.info = info

    @property
    def k_pad(self):
        return self.info.k_pad

    @property
    def dtype(self):
        return self.info.dtype

    @property
    def centred(self):
        return bool(self.info.centred)

    def centre_ptr(self):
        """Device address of the model's centre (float [k_pad]), or None."""
        p = ctypes.c_void_p()
        _check(lib().rgbd_svm_centre(self.handle, ctypes.byref(p)))
        return p.value

    def centre(self):
        """A copy of the model's centre, float32 [k_pad] on its device (None if uncentred)."""
        ptr = self.centre_ptr()
        if ptr is None:
            return None
        return torch.as_tensor(_DeviceArray(ptr, self.info.k_pad), device=f"cuda:{torch.cuda.current_device()}").clone()

    def free(self):
        if self.handle:
            lib().rgbd_svm_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _DeviceArray:
    """A library-owned float32 device buffer [n], seen by torch through the CUDA array
    interface (torch.as_tensor makes a view of it without copying)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def svm_train_data_pack(ctx, sv_feats, coef, bias=None, kernel=KERNEL_RBF, gamma=None, dtype=DT_F32, dim=None,
                        nbins=NBINS, centred=False, stream=None):
    if kernel == KERNEL_RBF:
        n_sv, dim = sv_feats.shape
        gamma = 1.0 / dim if gamma is None else gamma
    else:
        n_sv = 0
        dim = coef.shape[1] if dim is None else dim
        gamma = 0.0 if gamma is None else gamma
    C = coef.shape[0] if coef is not None else 0
    h = ctypes.c_void_p()
    dt = _dt(dtype) | (DT_CENTRED if centred else 0)
    _check(lib().svm_train_data_pack(ctx.handle, _p(sv_feats) if sv_feats is not None else None, n_sv, dim, nbins,
                                     _p(coef), _p(bias), C, kernel, float(gamma), dt, ctypes.byref(h),
                                     _stream(stream)))
    return SvmModel(h)


def svm_score(ctx, model, x, xsq=None, x_scale=448.0, scores=None, labels=None, want_labels=True, stream=None):
    n = x.shape[-2]  # rows (a split bf16 buffer is [2][n][k_pad])
    C = model.info.n_classes
    if scores is None:
        scores = torch.empty((n, C), dtype=torch.float32, device=x.device)
    if want_labels and labels is None:
        labels = torch.empty((n,), dtype=torch.int32, device=x.device)
    _check(lib().svm_score(ctx.handle, model.handle, _p(x), _p(xsq), n, float(x_scale), _p(scores),
                           _p(labels) if want_labels else None, _stream(stream)))
    return scores, (labels if want_labels else None)


def svm_score_noalloc(ctx, model, x, xsq, x_scale=448.0, scores=None, labels=None, want_labels=True, stream=None):
    """svm_score without any device allocation inside the call (see include/rgbd_lbp.h).

    For callers that cannot let the library call cudaMalloc (real-time loops that must not
    meet its device-wide synchronisation, processes whose device memory another allocator
    owns): the partial sums live in the library's fixed 16 MiB per-GPU scratch array.  Output tensors
    are allocated here only when the caller does not pass them.  Calls that overlap on the GPU
    share that array and race; keep them on one stream.
    """
    fn = lib().svm_score_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_float, P, P, P]
    fn.restype = ctypes.c_int
    n = x.shape[-2]  # rows (a split bf16 buffer is [2][n][k_pad])
    C = model.info.n_classes
    if scores is None:
        scores = torch.empty((n, C), dtype=torch.float32, device=x.device)
    if want_labels and labels is None:
        labels = torch.empty((n,), dtype=torch.int32, device=x.device)
    _check(fn(ctx.handle, model.handle, _p(x), _p(xsq), n, float(x_scale), _p(scores),
              _p(labels) if want_labels else None, _stream(stream)))
    return scores, (labels if want_labels else None)


# ---------------------------------------------------------------------------------------------
# Native request loop (rgbd_server_*)
# ---------------------------------------------------------------------------------------------

class ServerConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("max_batch_faces", ctypes.c_int32), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("crop", ctypes.c_int32), ("mask_mm", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("max_faces", ctypes.c_int32),
                ("x_scale", ctypes.c_float), ("idle_spin_us", ctypes.c_int32)]


class Completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("n_faces", ctypes.c_int32), ("t_submit", ctypes.c_double), ("t_done", ctypes.c_double)]


class NativeServer:
    """rgbd_server: the library's own request loop (a worker thread inside the library).

    submit() takes host tensors (pinned for asynchronous uploads) and returns a request id at
    once; the results land in the host tensors given to submit().  poll() returns finished
    requests with their submission and completion times (CLOCK_MONOTONIC seconds, the clock of
    time.clock_gettime(time.CLOCK_MONOTONIC)).  Tensors passed to submit() are kept referenced
    until their request is polled."""

    def __init__(self, model, H, W, n_streams, n_slots=96, max_batch_faces=2048, crop=128, mask_mm=150, flags=0,
                 max_faces=16, x_scale=448.0, idle_spin_us=2000):
        cfg = ServerConfig(n_slots, max_batch_faces, H, W, crop, mask_mm, flags, n_streams, max_faces, x_scale,
                           idle_spin_us)
        h = ctypes.c_void_p()
        _check(lib().rgbd_server_create(model.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self.model = model  # must outlive the server
        self.n_classes = model.info.n_classes
        self._held = {}

    def submit(self, stream_id, grey, depth, rects, scores, labels, ids=None):
        for t in (grey, depth, rects, scores, labels) + ((ids,) if ids is not None else ()):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("submit takes contiguous host tensors")
        rid = ctypes.c_uint64()
        hp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        _check(lib().rgbd_server_submit(self.handle, int(stream_id), hp(grey), hp(depth), hp(rects), int(rects.shape[0]),
                                        hp(scores), hp(labels), hp(ids), ctypes.byref(rid)))
        self._held[rid.value] = (grey, depth, rects, scores, labels, ids)
        return rid.value

    def poll(self, max_n=256, wait_us=0):
        buf = (Completion * max_n)()
        n = ctypes.c_int32()
        _check(lib().rgbd_server_poll(self.handle, buf, max_n, ctypes.byref(n), int(wait_us)))
        out = []
        for i in range(n.value):
            c = buf[i]
            self._held.pop(c.request_id, None)
            out.append((c.request_id, c.status, c.n_faces, c.t_submit, c.t_done, c.flags))
        return out

    def stats(self):
        v = [ctypes.c_uint64() for _ in range(4)]
        _check(lib().rgbd_server_stats(self.handle, *[ctypes.byref(x) for x in v]))
        return {"frames": v[0].value, "faces": v[1].value, "batches": v[2].value, "admission_waits": v[3].value}

    def close(self):
        if self.handle:
            lib().rgbd_server_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
