"""Measurements of the workloads other than the headline batch (run through ``bench.py --workload``).

crop       one 64x64 pre-cut crop, 8x8 cells (3776-dim), linear SVM with 5 classes: latency of
           lbp_fused_features + svm_score per crop, eager (C-ABI calls) and as a CUDA graph.
frame      one 640x480 frame with 4 faces -> 128x128 crops, RBF SVM 512 SVs x 10 classes in
           exact fp32: frame latency from pinned host frame to scores on the host.
precision  65536 x 16384 SVs x 15104 dims, 128 classes: BF16 / FP8 / TF32 scoring on the tensor
           cores against exact fp32 (labels, all rows) and the fp64 oracle (errors, a row sample).
serving    32 Poisson streams at 30 fps, 1-12 faces per frame, 8192 SVs (BF16) x 64 classes
           resident: continuous batching vs the plain per-crop path, p50 / p99 frame latency.
roi        Section 2.1's depth-space face regions for 4096 colour boxes over 256 frames.
train      Section 2.5's classifier trained on the GPU: 64 one-vs-rest RBF SVMs on 4096 rows.
small-batch  scoring latency of 1-128 rows against the serving model: split over K vs tile kernel.
Each prints one JSON line.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def _emit(d):
    print(json.dumps(d))
    return 0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------------------------
def run_crop(args):
    import torch
    import oracle as orc
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    wl = synth.plain_crop()
    ctx = B.Context(0)
    g = torch.from_numpy(wl.grey).cuda()
    d = torch.from_numpy(wl.depth.view(np.int16)).cuda()
    model = B.svm_train_data_pack(ctx, None, torch.from_numpy(wl.coef).cuda(), torch.from_numpy(wl.bias).cuda(),
                                  kernel=B.KERNEL_LINEAR, dim=wl.dim)
    out = {"feats": torch.empty((1, wl.dim), dtype=torch.int16, device="cuda"),
           "x": torch.empty((1, model.k_pad), dtype=torch.float32, device="cuda"),
           "xsq": torch.empty((1,), dtype=torch.float32, device="cuda")}
    scores = torch.empty((1, 5), dtype=torch.float32, device="cuda")
    labels = torch.empty((1,), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()

    def step():
        B.lbp_fused_features(ctx, g, d, None, crop=64, x_dtype="f32", out=out, stream=s)
        B.svm_score(ctx, model, out["x"], out["xsq"], scores=scores, labels=labels, stream=s)

    with torch.cuda.stream(s):
        step()
    torch.cuda.synchronize()
    want = orc.features_batch(wl.grey, wl.depth, None, 64)
    assert (out["feats"].cpu().numpy().view(np.uint16) == want).all()
    ref = orc.svm_linear(orc.normalize_f64(want), wl.coef, wl.bias)
    assert np.allclose(scores.cpu().numpy(), ref, rtol=0, atol=1e-4)
    n = 1000
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for _ in range(50):
        with torch.cuda.stream(s):
            step()
    torch.cuda.synchronize()
    host = []
    for i in range(n):
        t = time.perf_counter()
        with torch.cuda.stream(s):
            evs[i][0].record(s)
            step()
            evs[i][1].record(s)
        s.synchronize()
        host.append(1e6 * (time.perf_counter() - t))
    dev_us = [1000.0 * a.elapsed_time(b) for a, b in evs]
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=s):
        step()
    for _ in range(20):
        gr.replay()
    torch.cuda.synchronize()
    ghost = []
    for i in range(n):
        t = time.perf_counter()
        gr.replay()
        torch.cuda.current_stream().synchronize()
        ghost.append(1e6 * (time.perf_counter() - t))
    return _emit({"workload": "crop: 64x64 pre-cut uint8 grey + uint16 depth, 8x8 cells (3776-dim), linear SVM 5 "
                              "classes, fp32", "metric": "latency per crop (us)", "runs": n,
                  "device_us_p50": float(np.median(dev_us)), "device_us_p99": float(np.percentile(dev_us, 99)),
                  "host_us_p50": float(np.median(host)), "host_us_p99": float(np.percentile(host, 99)),
                  "graph_host_us_p50": float(np.median(ghost)), "graph_host_us_p99": float(np.percentile(ghost, 99)),
                  "parity": "features bit-exact, scores within 1e-4 of the fp64 oracle"})


# ---------------------------------------------------------------------------------------------
def run_frame(args):
    import torch
    import oracle as orc
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    wl = synth.single_frame()
    ctx = B.Context(0)
    dev = torch.device("cuda")
    h_g = torch.from_numpy(wl.grey).pin_memory()
    h_d = torch.from_numpy(wl.depth.view(np.int16)).pin_memory()
    h_r = B.rects_tensor(wl.rects, "cpu").pin_memory()
    g = torch.empty_like(h_g, device=dev)
    d = torch.empty_like(h_d, device=dev)
    r = torch.empty_like(h_r, device=dev)
    sv = torch.from_numpy(wl.sv_counts.view(np.int16)).to(dev)
    model = B.svm_train_data_pack(ctx, sv, torch.from_numpy(wl.coef).to(dev), torch.from_numpy(wl.bias).to(dev),
                                  gamma=wl.gamma, dtype="f32")
    n = wl.rects.shape[0]
    out = {"feats": torch.empty((n, wl.dim), dtype=torch.int16, device=dev),
           "x": torch.empty((n, model.k_pad), dtype=torch.float32, device=dev),
           "xsq": torch.empty((n,), dtype=torch.float32, device=dev)}
    scores = torch.empty((n, 10), dtype=torch.float32, device=dev)
    labels = torch.empty((n,), dtype=torch.int32, device=dev)
    h_s = torch.empty((n, 10), dtype=torch.float32).pin_memory()
    h_l = torch.empty((n,), dtype=torch.int32).pin_memory()
    s = torch.cuda.Stream()

    def frame():
        with torch.cuda.stream(s):
            g.copy_(h_g, non_blocking=True)
            d.copy_(h_d, non_blocking=True)
            r.copy_(h_r, non_blocking=True)
            B.lbp_fused_features(ctx, g, d, r, crop=128, x_dtype="f32", out=out, stream=s)
            B.svm_score(ctx, model, out["x"], out["xsq"], scores=scores, labels=labels, stream=s)
            h_s.copy_(scores, non_blocking=True)
            h_l.copy_(labels, non_blocking=True)
        s.synchronize()

    frame()
    want = orc.features_batch(wl.grey, wl.depth, wl.rects, 128)
    assert (out["feats"].cpu().numpy().view(np.uint16) == want).all()
    ref = orc.svm_rbf(orc.normalize_f64(want), orc.normalize_f64(wl.sv_counts), wl.coef, wl.bias, wl.gamma)
    assert (h_l.numpy() == orc.argmax(ref)).all()
    for _ in range(20):
        frame()
    lat = []
    for _ in range(300):
        t = time.perf_counter()
        frame()
        lat.append(1000.0 * (time.perf_counter() - t))
    # the same frame as one CUDA graph (uploads, both launches, read-backs): one launch call
    gr = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gr, stream=s):
        g.copy_(h_g, non_blocking=True)
        d.copy_(h_d, non_blocking=True)
        r.copy_(h_r, non_blocking=True)
        B.lbp_fused_features(ctx, g, d, r, crop=128, x_dtype="f32", out=out, stream=s)
        B.svm_score(ctx, model, out["x"], out["xsq"], scores=scores, labels=labels, stream=s)
        h_s.copy_(scores, non_blocking=True)
        h_l.copy_(labels, non_blocking=True)
    for _ in range(20):
        gr.replay()
    torch.cuda.synchronize()
    h_l.zero_()
    gr.replay()
    torch.cuda.synchronize()
    assert (h_l.numpy() == orc.argmax(ref)).all()
    glat = []
    for _ in range(300):
        t = time.perf_counter()
        gr.replay()
        torch.cuda.current_stream().synchronize()
        glat.append(1000.0 * (time.perf_counter() - t))
    return _emit({"workload": "frame: one 640x480 frame (uint8 grey + uint16 depth), 4 faces 80-200 px -> 128x128, "
                              "15104-dim, RBF SVM 512 SVs x 10 classes, exact fp32", "metric": "frame latency (ms)",
                  "runs": 300, "p50_ms": float(np.median(lat)), "p99_ms": float(np.percentile(lat, 99)),
                  "graph_p50_ms": float(np.median(glat)), "graph_p99_ms": float(np.percentile(glat, 99)),
                  "includes": "H2D of the frame pair + rects, fused features, scoring, D2H of scores and labels "
                              "(eager C-ABI calls, and the same sequence as one CUDA graph)",
                  "parity": "features bit-exact, labels equal to the fp64 oracle (eager and graph)"})


# ---------------------------------------------------------------------------------------------
def _oracle_rows(job):
    """Worker: fp64 oracle scores of a block of rows (runs in a spawned process)."""
    import oracle as orc
    x, sv, a, b, gamma = job
    return orc.svm_rbf(x, sv, a, b, gamma)


def run_precision(args):
    import bench
    n_rows, n_sv, C = 65536, 16384, 128
    oracle_rows = int(os.environ.get("PRECISION_ORACLE_ROWS", "64"))
    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4))  # before any GPU work
    import torch
    import oracle as orc
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    orc.build()
    dim = 16 * 16 * 59
    ctx = B.Context(0)
    dev = torch.device("cuda")
    X = synth.poisson_counts_device(1507, n_rows, dim, dev)
    SV = synth.poisson_counts_device(1507 + 1, n_sv, dim, dev)
    a, b = synth.rbf_coefficients(synth.rng_for(1507 + 2), C, n_sv)
    at, bt = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    gamma = 1.0 / dim
    pk, src = _peaks()
    res = {}
    labels = {}
    sub_scores = {}
    x_scale = 448.0
    modes = [("f32", False), ("bf16", False), ("fp8", False), ("tf32", False), ("bf16x3", False),
             ("bf16", True), ("fp8", True)]
    for dt_base, centred in modes:
        dt = dt_base + ("_centred" if centred else "")
        model = B.svm_train_data_pack(ctx, SV, at, bt, gamma=gamma, dtype=dt_base, centred=centred)
        x, q = B.lbp_normalize_features(ctx, X, dt_base, x_scale=x_scale, x_centre=model if centred else None)
        s_out, l_out = B.svm_score(ctx, model, x, q, x_scale=x_scale)
        torch.cuda.synchronize()
        t_first = time.perf_counter()
        B.svm_score(ctx, model, x, q, x_scale=x_scale, scores=s_out, labels=l_out)
        torch.cuda.synchronize()
        ms0 = (time.perf_counter() - t_first) * 1e3
        # >= ~1.5 s of back-to-back launches per tensor-core mode: the power cap settles and the
        # 100 ms clock and power samples see it
        reps = 1 if dt == "f32" else max(20, int(1500.0 / max(ms0, 1e-3)) + 1)
        ts = []
        clocks = bench.ClockSampler(0)
        clocks.start()
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.svm_score(ctx, model, x, q, x_scale=x_scale, scores=s_out, labels=l_out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        clk = clocks.stop()
        flops = 2.0 * n_rows * n_sv * dim + 2.0 * n_rows * n_sv * C
        ratio = {"bf16": 1.0, "fp8": 2.0, "tf32": 1.1 / 2.25, "bf16x3": 1.0 / 3.0}.get(dt_base)
        peak = pk["bf16_tflops"] * ratio if ratio else None
        peak_s = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * ratio if ratio else None
        # the modes run back to back for a second or more: the sustained (power-capped) peak is
        # the one that applies; the burst fraction is kept beside it
        res[dt] = {"ms": ms, "tflops": flops / ms / 1e9, "frac_of_peak": (flops / ms / 1e9) / peak if peak else None,
                   "peak_tflops": peak, "frac_of_sustained_peak": (flops / ms / 1e9) / peak_s if peak_s else None,
                   "sustained_peak_tflops": peak_s, "reps": reps, "clocks": clk}
        labels[dt] = l_out.cpu().numpy()
        sub_scores[dt] = s_out[:int(os.environ.get("PRECISION_FP64_ROWS", "4096"))].cpu().numpy()
        if dt == "f32":
            Xbig = X[:int(os.environ.get("PRECISION_FP64_ROWS", "4096"))].cpu().numpy().view(np.uint16)
            Xs = Xbig[:oracle_rows]
            SVh = SV.cpu().numpy().view(np.uint16)
        model.free()
        del x, q, s_out, l_out
        torch.cuda.empty_cache()
    # fp64 oracle on the row sample, in parallel blocks of rows
    x64 = orc.normalize_f64(Xs)
    sv64 = orc.normalize_f64(SVh)
    t0 = time.perf_counter()
    blocks = np.array_split(np.arange(oracle_rows), min(oracle_rows, 16))
    parts = pool.map(_oracle_rows, [(x64[bl], sv64, a, b, gamma) for bl in blocks])
    ref = np.concatenate(parts)
    t_oracle = time.perf_counter() - t0
    pool.close()
    ref_lab = orc.argmax(ref)
    srt = np.sort(ref, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    scale = np.abs(a).sum(1)[None, :] + np.abs(b)[None, :]
    # fp64 labels of a larger row block through the norm expansion and fp64 BLAS (the oracle's
    # direct sum is too slow for it); checked against the oracle on the rows both cover
    t1 = time.perf_counter()
    big = min(n_rows, int(os.environ.get("PRECISION_FP64_ROWS", "4096")))
    xb = orc.normalize_f64(Xbig)
    d2 = (xb * xb).sum(1)[:, None] + (sv64 * sv64).sum(1)[None, :] - 2.0 * (xb @ sv64.T)
    ref_big = np.exp(-gamma * np.maximum(d2, 0.0)) @ a.astype(np.float64).T + b.astype(np.float64)[None, :]
    del d2
    t_blas = time.perf_counter() - t1
    blas_vs_oracle = float(np.abs(ref_big[:oracle_rows] - ref).max())
    lab_big = orc.argmax(ref_big)
    sb = np.sort(ref_big, axis=1)
    margin_big = sb[:, -1] - sb[:, -2]
    # fp64 top-1 / top-2 margins in decades, and per mode the rows whose label differs from
    # exact fp32's in each decade: where the labels part is set by the margin, not by the mode
    edges = [0.0] + [10.0 ** k for k in range(-9, -2)] + [np.inf]
    names = ["<1e-9"] + [f"1e{k}..1e{k + 1}" for k in range(-9, -3)] + [">=1e-3"]
    hist = {nm: int(((margin_big >= lo) & (margin_big < hi)).sum()) for nm, lo, hi in zip(names, edges[:-1], edges[1:])}
    for dt in res:
        err = np.abs(sub_scores[dt][:oracle_rows].astype(np.float64) - ref)
        # the same error over every row of the fp64 BLAS reference (checked against the oracle
        # on the rows both cover)
        err_big = np.abs(sub_scores[dt][:big].astype(np.float64) - ref_big)
        differs = labels[dt][:big] != labels["f32"][:big]
        res[dt]["rows_differing_from_f32_by_fp64_margin"] = {
            nm: int((differs & (margin_big >= lo) & (margin_big < hi)).sum())
            for nm, lo, hi in zip(names, edges[:-1], edges[1:])}
        res[dt]["max_abs_err_vs_fp64"] = float(err.max())
        res[dt]["max_rel_err_vs_fp64"] = float((err / scale).max())
        res[dt][f"max_abs_err_vs_fp64_{big}_rows"] = float(err_big.max())
        res[dt]["label_agreement_vs_fp64_sample"] = float((labels[dt][:oracle_rows] == ref_lab).mean())
        res[dt]["label_agreement_vs_f32_all_rows"] = float((labels[dt] == labels["f32"]).mean())
        agree = labels[dt][:big] == lab_big
        decided = margin_big > 2.0 * max(err.max(), err_big.max())  # rows whose label that error bound cannot flip
        res[dt][f"label_agreement_vs_fp64_{big}_rows"] = float(agree.mean())
        res[dt]["rows_with_fp64_margin_above_2x_error"] = float(decided.mean())
        res[dt]["label_agreement_where_margin_above_2x_error"] = float(agree[decided].mean())
    return _emit({"workload": f"precision: {n_rows} x {n_sv} SVs x {dim} dims (Poisson(3) counts normalised per "
                              f"cell), {C} classes, gamma=1/dim", "metric": "scoring TFLOP/s, error and label agreement",
                  "results": res, "oracle_rows": oracle_rows, "oracle_s": t_oracle,
                  "fp64_blas_rows": big, "fp64_blas_s": t_blas, "fp64_blas_vs_oracle_max_abs": blas_vs_oracle,
                  "fp64_margin_below_1e-6_fraction": float((margin_big < 1e-6).mean()),
                  "fp64_margin_histogram_rows": hist,
                  "fp64_margin_top1_top2": {"min": float(margin.min()), "median": float(np.median(margin))},
                  "peak_source": src})


# ---------------------------------------------------------------------------------------------
def serving_leg(ctx, seconds, warm_frames=50):
    """Serving workload: 32 Poisson camera streams at 30 fps against a resident 8192-SV model,
    served by the continuous-batching loop and by the plain per-crop path.  Latency of a frame:
    from its arrival to its scores and labels in host memory (upload, features, scoring and
    read-back included).  Returns the summaries of both paths."""
    import torch
    from paper_1504_01883_gb300 import serve, synth
    from paper_1504_01883_gb300 import binding as B
    dev = torch.device("cuda")
    dim = 16 * 16 * 59
    rng = synth.rng_for(1508 + 5)
    sv = synth.poisson_counts(rng, 8192, dim)
    a, b = synth.rbf_coefficients(rng, 64, 8192)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).to(dev), torch.from_numpy(a).to(dev),
                                  torch.from_numpy(b).to(dev), gamma=1.0 / dim, dtype="bf16")
    streams = serve.make_streams()
    events = synth.serving_arrivals(seconds=seconds)
    out = {"workload": f"serving: 32 RGB-D streams x 30 fps (Poisson arrivals, {seconds:g} s), 640x480, "
                       "1-12 faces per frame, sides U{48..256} -> 128x128, RBF 8192 SVs (BF16) x 64 classes "
                       "resident",
           "latency": "arrival of the frame -> its scores and labels in host memory",
           "frames": len(events), "offered_crops_per_s": sum(k for _, _, k in events) / seconds}
    for name, cls in [("batched_native", serve.NativeBatchServer), ("batched", serve.BatchServer),
                      ("per_crop", serve.PerCropServer)]:
        srv = cls(ctx, model, streams)
        # warm-up: large batches (every frame at once), then a short real-time stretch (small
        # batches), so that no first use of a launch shape or a workspace growth lands in the run
        srv.run(events[:warm_frames], realtime=False)
        srv.run(events[:4 * warm_frames], realtime=True)
        rep, _ = srv.run(events, realtime=True)
        out[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in rep.summary().items()}
        if name != "per_crop":
            # capacity: every frame of the run queued at once (the per-crop path's real-time run
            # already falls behind, so its crops/s is its capacity)
            cap, _ = srv.run(events, realtime=False)
            out[name]["capacity_crops_per_s"] = round(cap.crops / cap.wall_s, 1)
            out[name]["capacity_batches"] = cap.batches
            if cap.submit_s:
                # the caller's submission of the queued frames: when it takes most of the wall
                # time, the capacity figure is the submitting thread's rate, not the GPU's
                out[name]["capacity_submit_s"] = round(cap.submit_s, 4)
                out[name]["capacity_wall_s"] = round(cap.wall_s, 4)
        if hasattr(srv, "close"):
            srv.close()
        del srv
        torch.cuda.empty_cache()
    out["batched_native"]["loop"] = "the library's C++ request loop (rgbd_server)"
    out["batched"]["loop"] = "Python loop over the C-ABI calls"
    model.free()
    return out


def run_serving(args):
    from paper_1504_01883_gb300 import _build
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    ctx = B.Context(0)
    out = serving_leg(ctx, args.seconds)
    out["metric"] = "p50/p99 frame latency (ms) and crops/s"
    return _emit(out)


def run_roi(args):
    """Section 2.1's region-of-interest step on the batch workload's frames: 4096 colour-image
    face boxes over 256 depth frames -> depth-space rects."""
    import torch
    import oracle as orc
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    wl = synth.batching()
    rng = synth.rng_for(1506 + 11)
    cal = synth.calibration(rng)
    boxes = synth.colour_boxes(rng, wl.rects)
    ctx = B.Context(0)
    d = torch.from_numpy(wl.depth.view(np.int16)).cuda()
    bx = B.rects_tensor(boxes)
    c = B.Calib.from_record(cal)
    out = B.rgbd_face_roi(ctx, d, c, bx)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    sample = np.arange(0, len(boxes), len(boxes) // 64)
    want = orc.face_roi(wl.depth, cal, boxes[sample])
    for i, f in enumerate(["frame", "x", "y", "w", "h"]):
        assert (got[sample, i] == want[f]).all(), f
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ts = []
    for it in range(13):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.rgbd_face_roi(ctx, d, c, bx, out=out)
        e1.record()
        torch.cuda.synchronize()
        if it >= 3:
            ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    found = float((got[:, 3] > 0).mean())
    area = float(np.mean(got[:, 3].astype(np.float64) * got[:, 4]))
    return _emit({"workload": "roi: 256 depth frames 640x480, 4096 colour face boxes (side 48-256), synthetic "
                              "depth-to-colour calibration (scale, shear, offset, 20-30 px stereo shift at 1 m)",
                  "metric": "face regions per second", "value": len(boxes) / (ms * 1e-3), "ms": ms,
                  "faces_with_region": found, "mean_region_area_px": area, "status": ctx.status(clear=True),
                  "parity": f"{len(sample)} sampled faces equal to the oracle's full-frame scan",
                  "l2": "flushed between timed launches"})


def run_train(args):
    """One-vs-rest RBF SVM training on the GPU: 4096 face feature rows (64 identities x 64 views,
    16x16 cells x 59 bins), 64 classes, SMO to a gap of 1e-3; then the model is packed and scored."""
    import torch
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    rng = synth.rng_for(1509)
    C, per, cells = 64, 64, 256
    dim = cells * 59
    protos = rng.uniform(0.5, 1.5, (C, dim))
    lab = np.repeat(np.arange(C, dtype=np.int32), per)
    counts = rng.poisson(3.0 * protos[lab]).astype(np.uint16)
    test_lab = rng.integers(0, C, 1024).astype(np.int32)
    test = rng.poisson(3.0 * protos[test_lab]).astype(np.uint16)
    gamma, cost, eps = 0.5, 1.0, 1e-3
    ctx = B.Context(0)
    dev = torch.device("cuda")
    cnt = torch.from_numpy(counts.view(np.int16)).to(dev)
    x, q = B.lbp_normalize_features(ctx, cnt, "f32")
    labels = torch.from_numpy(lab).to(dev)
    B.svm_train_rbf(ctx, x, q, labels, C, gamma, cost, eps)  # warm-up (workspace, module load)
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        coef, bias, iters = B.svm_train_rbf(ctx, x, q, labels, C, gamma, cost, eps)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    it = iters.cpu().numpy()
    # the trained model scored in every precision on the held-out rows: label agreement with
    # the exact fp32 path and with fp64 where the classes are structured (real margins), beside
    # the precision workload's i.i.d. rows
    import oracle as orc
    orc.build()
    tcnt = torch.from_numpy(test.view(np.int16)).to(dev)
    a64 = coef.double().cpu().numpy()
    b64 = bias.double().cpu().numpy()
    x64 = orc.normalize_f64(test)
    sv64 = orc.normalize_f64(counts)
    d2 = (x64 * x64).sum(1)[:, None] + (sv64 * sv64).sum(1)[None, :] - 2.0 * (x64 @ sv64.T)
    ref = np.exp(-gamma * np.maximum(d2, 0.0)) @ a64.T + b64[None, :]
    ref_oracle = orc.svm_rbf(x64[:8], sv64, a64, b64, gamma)  # the BLAS expansion checked on 8 rows
    ref_lab = orc.argmax(ref)
    srt = np.sort(ref, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    per_mode = {}
    lab_f32 = None
    for dt_base, centred in [("f32", False), ("bf16", False), ("bf16", True), ("fp8", False), ("fp8", True),
                             ("tf32", False), ("bf16x3", False)]:
        m = B.svm_train_data_pack(ctx, cnt, coef, bias, gamma=gamma, dtype=dt_base, centred=centred)
        xt, qt = B.lbp_normalize_features(ctx, tcnt, dt_base, x_centre=m if centred else None)
        s, pred = B.svm_score(ctx, m, xt, qt)
        s = s.double().cpu().numpy()
        pred = pred.cpu().numpy()
        lab_f32 = pred if dt_base == "f32" else lab_f32
        err = float(np.abs(s - ref).max())
        per_mode[dt_base + ("_centred" if centred else "")] = {
            "max_abs_err_vs_fp64": err, "label_agreement_vs_fp64": float((pred == ref_lab).mean()),
            "label_agreement_vs_f32": float((pred == lab_f32).mean()),
            "heldout_accuracy": float((pred == test_lab).mean()),
            "rows_with_fp64_margin_above_2x_error": float((margin > 2.0 * err).mean())}
        m.free()
    n_sv = int((coef.abs().amax(0) > 0).sum().item())
    return _emit({"workload": f"train: {C * per} rows ({C} classes x {per}), {dim}-dim per-cell normalised "
                              f"histograms, RBF gamma={gamma}, cost={cost}, SMO gap {eps}",
                  "metric": "training time (ms) for all one-vs-rest classifiers", "ms": float(np.median(ts)),
                  "smo_steps_per_class": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max())},
                  "support_vectors": n_sv, "heldout_rows": int(test.shape[0]),
                  "fp64_blas_vs_oracle_max_abs": float(np.abs(ref[:8] - ref_oracle).max()),
                  "fp64_margin_top1_top2": {"min": float(margin.min()), "median": float(np.median(margin))},
                  "scoring_precision": per_mode, "status": ctx.status(clear=True)})


# ---------------------------------------------------------------------------------------------
def run_small_batch(args):
    """Scoring latency of serving-sized batches (1-128 rows) against the serving model (8192
    SVs x 15104, BF16, 64 classes): the small-batch split over K against the tile kernel
    (RGBD_TUNE_TC_SPLITK = 1), CUDA events around each call, median of `--steps` calls after
    `--warmup`."""
    import torch
    from paper_1504_01883_gb300 import _build, synth
    from paper_1504_01883_gb300 import binding as B
    _build.build()
    dev = torch.device("cuda")
    ctx = B.Context(0)
    dim = 16 * 16 * 59
    rng = synth.rng_for(1508 + 5)
    sv = synth.poisson_counts(rng, 8192, dim)
    a, b = synth.rbf_coefficients(rng, 64, 8192)
    model = B.svm_train_data_pack(ctx, torch.from_numpy(sv.view(np.int16)).to(dev), torch.from_numpy(a).to(dev),
                                  torch.from_numpy(b).to(dev), gamma=1.0 / dim, dtype="bf16")
    s = torch.cuda.Stream()
    res = {}
    for n in (1, 6, 12, 24, 64, 128):
        X = torch.from_numpy(synth.poisson_counts(rng, n, dim).view(np.int16)).to(dev)
        x, q = B.lbp_normalize_features(ctx, X, "bf16")
        sc, lb = B.svm_score(ctx, model, x, q)
        row = {}
        for name, knob in (("split_k", 0), ("tile_kernel", 1)):
            ctx.set_tuning(B.TUNE_TC_SPLITK, knob)
            ts = []
            for i in range(args.warmup + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                B.svm_score(ctx, model, x, q, scores=sc, labels=lb, stream=s)
                e1.record(s)
                e1.synchronize()
                if i >= args.warmup:
                    ts.append(1000.0 * e0.elapsed_time(e1))
            row[name + "_us"] = round(float(np.median(ts)), 1)
        ctx.set_tuning(B.TUNE_TC_SPLITK, 0)
        res[str(n)] = row
    status = ctx.status(clear=True)
    model.free()
    return _emit({"workload": "small-batch scoring: 1-128 rows x 8192 SVs x 15104 (BF16), 64 classes",
                  "metric": "scoring latency (us, CUDA events, median)", "calls": args.steps, "rows": res,
                  "status": status})


def run(args):
    return {"crop": run_crop, "frame": run_frame, "precision": run_precision, "serving": run_serving,
            "roi": run_roi, "train": run_train, "small-batch": run_small_batch}[args.workload](args)
