"""Continuous-batching request loop over simulated RGB-D camera streams.

Frames from many cameras arrive at Poisson times.  The loop keeps the packed SVM model and a
pool of frame slots resident on the GPU and runs, on one compute stream, batches of all faces
of all frames that have been uploaded.  While a batch runs, frames that arrive meanwhile are
admitted (when a slot is free, the frame's bytes fit the server's device-memory budget and the
device has memory to spare) and uploaded on a separate
copy stream, so they form the next batch as soon as the GPU frees up: uploads overlap compute
and batches follow each other with no gap.  Every frame's latency is measured from its arrival
to the moment its scores and labels are on the host.

``PerCropServer`` is the plain path it is compared with: each face of each frame is featurised
and scored by its own launches, one at a time, as soon as the frame arrives.

Everything on the GPU goes through the library's C ABI (``binding``); torch only provides the
device buffers, pinned host buffers, streams and events.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B
from . import synth


@dataclass
class StreamFrames:
    """Pre-generated frames of one simulated camera (cycled through on each arrival)."""
    grey: np.ndarray      # [P][H][W] uint8
    depth: np.ndarray     # [P][H][W] uint16
    rects: list           # P arrays of RECT_DTYPE (frame field = 0)


def make_streams(seed=1508, n_streams=32, frames_per_stream=4, fmin=1, fmax=12, smin=48, smax=256,
                 H=synth.FRAME_H, W=synth.FRAME_W):
    rng = synth.rng_for(seed + 77)
    out = []
    for s in range(n_streams):
        counts = [int(rng.integers(fmin, fmax + 1)) for _ in range(frames_per_stream)]
        g, d, r = synth.frames_with_rects(seed * 1000 + s, frames_per_stream, counts, smin, smax, H, W)
        per = []
        for f in range(frames_per_stream):
            rr = r[r["frame"] == f].copy()
            rr["frame"] = 0
            per.append(rr)
        out.append(StreamFrames(g, d, per))
    return out


@dataclass
class FrameRequest:
    t_arrival: float      # seconds since the start of the run
    stream: int
    index: int            # arrival index within its stream (selects the pre-generated frame)
    n_faces: int = 0
    slot: int = -1
    t_done: float = 0.0
    scores: np.ndarray | None = None
    labels: np.ndarray | None = None
    ids: np.ndarray | None = None         # tracked identities (Section 2.3), batched path only


class MemoryAdmission:
    """Admits a frame when a frame slot is free, the frame's device bytes fit the server's
    device-memory budget, and the device keeps `reserve_bytes` free for everyone else.

    A frame charges its upload (the grey and depth planes) plus, per face, the device rows its
    faces occupy until the frame is done (normalised feature row, norm, scores, label, identity,
    rect).  The charge is returned when the frame's results are on the host.  The server's
    buffers are allocated up front, so `budget_bytes` is the size of the part of them that
    frames draw on; the slot count bounds the frames in flight, the budget bounds their bytes
    (frames with many faces take more of it), and the free-memory check reacts to other users of
    the device.  Without a budget only the slots and the reserve apply."""

    def __init__(self, n_slots, reserve_bytes=256 << 20, mem_get_info=None, budget_bytes=None):
        self.free_slots = collections.deque(range(n_slots))
        self.reserve = reserve_bytes
        self.mem_get_info = mem_get_info or torch.cuda.mem_get_info
        self.budget = budget_bytes
        self.used = 0
        self.charged = {}
        self.rejections = 0

    def try_admit(self, nbytes=0):
        if not self.free_slots:
            return -1
        if self.budget is not None and self.used + nbytes > self.budget:
            self.rejections += 1
            return -1
        free, _ = self.mem_get_info()
        if free < self.reserve:
            self.rejections += 1
            return -1
        slot = self.free_slots.popleft()
        self.used += nbytes
        self.charged[slot] = nbytes
        return slot

    def release(self, slot):
        self.used -= self.charged.pop(slot, 0)
        self.free_slots.append(slot)


@dataclass
class _Batch:
    frames: list
    done: torch.cuda.Event
    scores_h: torch.Tensor
    labels_h: torch.Tensor
    n: int
    buffer: int
    ids_h: torch.Tensor | None = None


@dataclass
class ServeReport:
    latencies_ms: list = field(default_factory=list)
    crops: int = 0
    frames: int = 0
    batches: int = 0
    wall_s: float = 0.0
    rejections: int = 0
    submit_s: float = 0.0  # when the caller had handed over the last frame (the library's loop)

    def summary(self):
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.array([np.nan])
        return {"frames": self.frames, "crops": self.crops, "batches": self.batches,
                "crops_per_s": self.crops / self.wall_s if self.wall_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(np.max(lat)), "wall_s": self.wall_s, "admission_waits": self.rejections}


class BatchServer:
    """Continuous batching of faces across streams (see the module docstring)."""

    def __init__(self, ctx, model, streams, n_slots=96, max_faces=2048, crop=128, x_dtype="bf16",
                 mask_mm=150, admission=None, device=None):
        self.ctx, self.model, self.streams = ctx, model, streams
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        H, W = streams[0].grey.shape[1:]
        self.H, self.W = H, W
        self.crop, self.mask_mm = crop, mask_mm
        self.x_dtype = B._dt(x_dtype)
        self.max_faces = max_faces
        self.n_slots = n_slots
        self.grey = torch.empty((n_slots, H, W), dtype=torch.uint8, device=self.dev)
        self.depth = torch.empty((n_slots, H, W), dtype=torch.int16, device=self.dev)
        # pinned copies of every pre-generated frame
        self.h_grey = [torch.from_numpy(s.grey).pin_memory() for s in streams]
        self.h_depth = [torch.from_numpy(s.depth.view(np.int16)).pin_memory() for s in streams]
        dim = (crop // 8) ** 2 * 59
        self.dim = dim
        k_pad = model.k_pad
        C = model.info.n_classes
        # two sets of batch buffers, so one batch can be prepared while the other runs
        self.bufs = []
        for _ in range(2):
            self.bufs.append({
                "rects_h": torch.empty((max_faces, 5), dtype=torch.int32).pin_memory(),
                "rects": torch.empty((max_faces, 5), dtype=torch.int32, device=self.dev),
                "x": torch.empty((max_faces, k_pad), dtype=B.x_torch_dtype(self.x_dtype), device=self.dev),
                "xsq": torch.empty((max_faces,), dtype=torch.float32, device=self.dev),
                "scores": torch.empty((max_faces, C), dtype=torch.float32, device=self.dev),
                "labels": torch.empty((max_faces,), dtype=torch.int32, device=self.dev),
                "scores_h": torch.empty((max_faces, C), dtype=torch.float32).pin_memory(),
                "labels_h": torch.empty((max_faces,), dtype=torch.int32).pin_memory(),
                # frame -> stream ids and face ranges of the batch, for the tracking step
                "meta_h": torch.empty((2 * n_slots + 1,), dtype=torch.int32).pin_memory(),
                "meta": torch.empty((2 * n_slots + 1,), dtype=torch.int32, device=self.dev),
                "ids": torch.empty((max_faces,), dtype=torch.int32, device=self.dev),
                "ids_h": torch.empty((max_faces,), dtype=torch.int32).pin_memory(),
            })
        self.compute = torch.cuda.Stream(device=self.dev)
        self.copy = torch.cuda.Stream(device=self.dev)
        # device bytes a frame holds while it is in flight: its planes, and per face the rows
        # of the batch buffers (normalised row, norm, scores, label, identity, rect)
        self.frame_bytes = H * W * 3
        self.face_bytes = (self.bufs[0]["x"][0].numel() * self.bufs[0]["x"].element_size() + 4 + 4 * C + 4 + 4
                           + 20)
        budget = n_slots * self.frame_bytes + 2 * max_faces * self.face_bytes
        self.admission = admission or MemoryAdmission(n_slots, budget_bytes=budget)
        self.slot_ready = {}   # slot -> event recorded after its upload
        # per-stream state kept on the device: the faces of each stream's last served frame and
        # their identities (Section 2.3 tracking), updated by every batch in arrival order
        self.track = B.TrackState(len(streams), max_faces=16, device=self.dev)

    def _frame(self, req):
        s = self.streams[req.stream]
        k = req.index % len(s.rects)
        return k, s.rects[k]

    def _bytes(self, req):
        """Device bytes the request holds until its results are on the host."""
        return self.frame_bytes + len(self._frame(req)[1]) * self.face_bytes

    def _upload(self, req):
        k, rects = self._frame(req)
        req.n_faces = len(rects)
        with torch.cuda.stream(self.copy):
            self.grey[req.slot].copy_(self.h_grey[req.stream][k], non_blocking=True)
            self.depth[req.slot].copy_(self.h_depth[req.stream][k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy)
        self.slot_ready[req.slot] = ev

    def _launch(self, frames, buf_id):
        buf = self.bufs[buf_id]
        rows = []
        for req in frames:
            _, rects = self._frame(req)
            for r in rects:
                rows.append((req.slot, int(r["x"]), int(r["y"]), int(r["w"]), int(r["h"])))
        n = len(rows)
        buf["rects_h"][:n] = torch.tensor(rows, dtype=torch.int32)
        nfr = len(frames)
        starts = np.cumsum([0] + [req.n_faces for req in frames])
        buf["meta_h"][:nfr] = torch.tensor([req.stream for req in frames], dtype=torch.int32)
        buf["meta_h"][nfr:2 * nfr + 1] = torch.from_numpy(starts.astype(np.int32))
        cs = self.compute
        for req in frames:
            cs.wait_event(self.slot_ready.pop(req.slot))
        with torch.cuda.stream(cs):
            buf["rects"][:n].copy_(buf["rects_h"][:n], non_blocking=True)
            rects = buf["rects"][:n]
            B.lbp_fused_features(self.ctx, self.grey, self.depth, rects, crop=self.crop, mask_mm=self.mask_mm,
                                 feats=False, x_dtype=self.x_dtype,
                                 out={"x": buf["x"][:n], "xsq": buf["xsq"][:n]}, stream=cs)
            B.svm_score(self.ctx, self.model, buf["x"][:n], buf["xsq"][:n], scores=buf["scores"][:n],
                        labels=buf["labels"][:n], stream=cs)
            buf["meta"][:2 * nfr + 1].copy_(buf["meta_h"][:2 * nfr + 1], non_blocking=True)
            B.rgbd_track_streams(self.ctx, self.track, buf["meta"][:nfr], buf["meta"][nfr:2 * nfr + 1], rects,
                                 buf["labels"][:n], ids=buf["ids"][:n], stream=cs)
            buf["scores_h"][:n].copy_(buf["scores"][:n], non_blocking=True)
            buf["labels_h"][:n].copy_(buf["labels"][:n], non_blocking=True)
            buf["ids_h"][:n].copy_(buf["ids"][:n], non_blocking=True)
            done = torch.cuda.Event()
            done.record(cs)
        return _Batch(frames, done, buf["scores_h"], buf["labels_h"], n, buf_id, buf["ids_h"])

    def _complete(self, batch, t0, report, keep_results):
        now = time.perf_counter() - t0
        off = 0
        for req in batch.frames:
            k = req.n_faces
            if keep_results:
                req.scores = batch.scores_h[off:off + k].numpy().copy()
                req.labels = batch.labels_h[off:off + k].numpy().copy()
                if batch.ids_h is not None:
                    req.ids = batch.ids_h[off:off + k].numpy().copy()
            off += k
            req.t_done = now
            report.latencies_ms.append(1000.0 * (now - req.t_arrival))
            report.frames += 1
            report.crops += k
            self.admission.release(req.slot)
        report.batches += 1

    def serve_one(self, stream, index):
        """Serves frame `index` of `stream` alone (a batch of one frame); returns the request."""
        req = FrameRequest(0.0, int(stream), int(index))
        req.slot = self.admission.try_admit(self._bytes(req))
        if req.slot < 0:
            raise RuntimeError("no free frame slot")
        self._upload(req)
        b = self._launch([req], 0)
        b.done.synchronize()
        self._complete(b, time.perf_counter(), ServeReport(), keep_results=True)
        return req

    def run(self, events, keep_results=False, realtime=True):
        """events: list of (t_arrival_s, stream, n_faces) sorted by time.  Returns (report, requests)."""
        counters = collections.Counter()
        reqs = []
        for t, s, _ in events:
            reqs.append(FrameRequest(float(t), int(s), counters[s]))
            counters[s] += 1
        pending = collections.deque(reqs)
        waiting = collections.deque()
        admitted = []
        inflight = collections.deque()
        report = ServeReport()
        free_bufs = [0, 1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if not realtime:  # every frame has arrived at t = 0 (offline throughput)
            for r in reqs:
                r.t_arrival = 0.0
        while pending or waiting or admitted or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                waiting.append(pending.popleft())
            while waiting:
                slot = self.admission.try_admit(self._bytes(waiting[0]))
                if slot < 0:
                    break
                req = waiting.popleft()
                req.slot = slot
                self._upload(req)
                admitted.append(req)
            while inflight and inflight[0].done.query():
                b = inflight.popleft()
                self._complete(b, t0, report, keep_results)
                free_bufs.append(b.buffer)
            if admitted and free_bufs and len(inflight) < 2:
                batch, faces = [], 0
                while admitted and faces + admitted[0].n_faces <= self.max_faces:
                    req = admitted.pop(0)
                    batch.append(req)
                    faces += req.n_faces
                inflight.append(self._launch(batch, free_bufs.pop(0)))
                continue
            if not (waiting or admitted) and inflight:
                # nothing to prepare: wait for the next completion or arrival
                nxt = pending[0].t_arrival if pending else None
                while not inflight[0].done.query():
                    if nxt is not None and time.perf_counter() - t0 >= nxt:
                        break
            elif not inflight and not waiting and not admitted and pending:
                dt = pending[0].t_arrival - (time.perf_counter() - t0)
                if dt > 0.0005:
                    time.sleep(dt - 0.0003)
        torch.cuda.synchronize()
        report.wall_s = time.perf_counter() - t0
        report.rejections = self.admission.rejections
        return report, reqs


class PerCropServer(BatchServer):
    """The plain per-crop GPU path: each face is featurised and scored by its own launches."""

    def run(self, events, keep_results=False, realtime=True):
        counters = collections.Counter()
        reqs = []
        for t, s, _ in events:
            reqs.append(FrameRequest(float(t), int(s), counters[s]))
            counters[s] += 1
        report = ServeReport()
        buf = self.bufs[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if not realtime:
            for r in reqs:
                r.t_arrival = 0.0
        cs = self.compute
        for req in reqs:
            dt = req.t_arrival - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            req.slot = 0
            self._upload(req)
            cs.wait_event(self.slot_ready.pop(0))
            _, rects = self._frame(req)
            k = len(rects)
            scores = np.zeros((k, self.model.info.n_classes), np.float32)
            labels = np.zeros(k, np.int32)
            with torch.cuda.stream(cs):
                for i, r in enumerate(rects):
                    buf["rects_h"][0] = torch.tensor([0, int(r["x"]), int(r["y"]), int(r["w"]), int(r["h"])],
                                                     dtype=torch.int32)
                    buf["rects"][:1].copy_(buf["rects_h"][:1], non_blocking=True)
                    B.lbp_fused_features(self.ctx, self.grey, self.depth, buf["rects"][:1], crop=self.crop,
                                         mask_mm=self.mask_mm, feats=False, x_dtype=self.x_dtype,
                                         out={"x": buf["x"][:1], "xsq": buf["xsq"][:1]}, stream=cs)
                    B.svm_score(self.ctx, self.model, buf["x"][:1], buf["xsq"][:1], scores=buf["scores"][:1],
                                labels=buf["labels"][:1], stream=cs)
                    buf["scores_h"][:1].copy_(buf["scores"][:1], non_blocking=True)
                    buf["labels_h"][:1].copy_(buf["labels"][:1], non_blocking=True)
                    cs.synchronize()
                    scores[i] = buf["scores_h"][0].numpy()
                    labels[i] = buf["labels_h"][0].item()
            req.n_faces = k
            req.t_done = time.perf_counter() - t0
            if keep_results:
                req.scores, req.labels = scores, labels
            report.latencies_ms.append(1000.0 * (req.t_done - req.t_arrival))
            report.frames += 1
            report.crops += k
            report.batches += k
        report.wall_s = time.perf_counter() - t0
        return report, reqs


class NativeBatchServer:
    """The same continuous batching, run by the library's own request loop (``rgbd_server``: a
    worker thread in C++ that admits frames into device slots, uploads them on a copy stream and
    launches batches while the caller only submits frames and collects results).  Python here
    only replays the arrivals and reads the completion times the library stamps."""

    def __init__(self, ctx, model, streams, n_slots=96, max_faces=2048, crop=128, x_dtype="bf16", mask_mm=150,
                 device=None):
        del ctx, x_dtype  # the server has a context of its own and scores in the model's type
        H, W = streams[0].grey.shape[1:]
        self.streams = streams
        self.model = model
        self.C = model.info.n_classes
        self.srv = B.NativeServer(model, H, W, n_streams=len(streams), n_slots=n_slots, max_batch_faces=max_faces,
                                  crop=crop, mask_mm=mask_mm, max_faces=16)
        self.h_grey = [torch.from_numpy(s.grey).pin_memory() for s in streams]
        self.h_depth = [torch.from_numpy(s.depth.view(np.int16)).pin_memory() for s in streams]
        self.h_rects = [[torch.from_numpy(np.ascontiguousarray(r).view(np.int32).reshape(-1, 5)) for r in s.rects]
                        for s in streams]

    def _submit(self, req):
        k = req.index % len(self.streams[req.stream].rects)
        rects = self.h_rects[req.stream][k]
        n = rects.shape[0]
        req.n_faces = n
        req.scores = torch.empty((n, self.C), dtype=torch.float32)
        req.labels = torch.empty((n,), dtype=torch.int32)
        req.ids = torch.empty((n,), dtype=torch.int32)
        return self.srv.submit(req.stream, self.h_grey[req.stream][k], self.h_depth[req.stream][k], rects, req.scores,
                               req.labels, req.ids)

    def serve_one(self, stream, index):
        req = FrameRequest(0.0, int(stream), int(index))
        rid = self._submit(req)
        deadline = time.monotonic() + 60.0
        while True:
            done = self.srv.poll(wait_us=100000)
            if any(d[0] == rid for d in done):
                break
            if time.monotonic() > deadline:
                raise RuntimeError(f"request {rid} did not complete within 60 s")
        req.scores, req.labels, req.ids = req.scores.numpy(), req.labels.numpy(), req.ids.numpy()
        return req

    def run(self, events, keep_results=False, realtime=True):
        counters = collections.Counter()
        reqs = []
        for t, s, _ in events:
            reqs.append(FrameRequest(float(t), int(s), counters[s]))
            counters[s] += 1
        if not realtime:
            for r in reqs:
                r.t_arrival = 0.0
        by_id = {}
        report = ServeReport()
        b0 = self.srv.stats()["batches"]
        clock = time.CLOCK_MONOTONIC
        t0 = time.clock_gettime(clock)

        def collect(wait_us=0):
            for rid, status, n, _t_sub, t_done, _flags in self.srv.poll(wait_us=wait_us):
                req = by_id.pop(rid)
                if status != 0:
                    raise RuntimeError(f"request {rid} failed with status {status}")
                req.t_done = t_done - t0
                report.latencies_ms.append(1000.0 * (req.t_done - req.t_arrival))
                report.frames += 1
                report.crops += n

        for req in reqs:
            while True:
                dt = req.t_arrival - (time.clock_gettime(clock) - t0)
                if dt <= 0:
                    break
                if dt > 0.0005:
                    time.sleep(dt - 0.0003)
            by_id[self._submit(req)] = req
            collect()
        report.submit_s = time.clock_gettime(clock) - t0
        deadline = time.monotonic() + 60.0
        while by_id:
            left = len(by_id)
            collect(wait_us=1000)
            if len(by_id) < left:
                deadline = time.monotonic() + 60.0
            elif time.monotonic() > deadline:
                raise RuntimeError(f"{len(by_id)} requests did not complete within 60 s")
        report.wall_s = max(r.t_done for r in reqs) if reqs else 0.0
        report.batches = self.srv.stats()["batches"] - b0
        if keep_results:
            for r in reqs:
                r.scores, r.labels, r.ids = r.scores.numpy(), r.labels.numpy(), r.ids.numpy()
        return report, reqs

    def close(self):
        self.srv.close()
