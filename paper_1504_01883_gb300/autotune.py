"""Autotuner of the launch layout.

It times the two stages of a workload (the fused feature kernel and the scoring kernels) under
candidate settings of the context's tuning knobs and keeps the fastest:

  K1  the fused kernel's tile shape and resident CTAs per SM: one CTA per face works on a
      128 x 128 crop laid out as 16 x 16 cells of 8 x 8 pixels, with either one thread per
      4 x 8 half cell (512 threads, 64 registers), one thread per cell (256 threads, up to
      128 registers) or one per 4 x 4 quarter cell (1024 threads, one CTA per SM), and one or
      two such CTAs in flight per SM;
  K2  how many SV-tile ranges ("splits") each 128-row block of the tensor-core scoring
      kernel is cut into (the row x SV tiling across SMs), and whether CTA pairs run one
      256-row MMA (tcgen05 cta_group::2) or every CTA runs its own 128-row MMA.

Choices never change the integer features, only the order of the SV sum (scores move within
rounding).  Results are cached in a JSON file keyed by GPU name and workload shape.
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import asdict, dataclass

import torch

from . import binding as B

CACHE_VERSION = 4  # bumped whenever the set of knobs changes
CACHE_PATH = os.environ.get("RGBD_TUNE_CACHE",
                            os.path.join(os.path.expanduser("~"), ".cache", "rgbd_lbp_gb300", "tune.json"))


@dataclass
class Tuning:
    lbp_ctas_per_sm: int = 0
    tc_splits: int = 0
    tc_pairing: int = 0
    lbp_shape: int = 0   # fused-kernel threads per cell (2: half cells, 1: whole cells, 3: quarter cells; 0 = default)

    def apply(self, ctx):
        ctx.set_tuning(B.TUNE_LBP_CTAS_PER_SM, self.lbp_ctas_per_sm)
        ctx.set_tuning(B.TUNE_LBP_SHAPE, self.lbp_shape)
        ctx.set_tuning(B.TUNE_TC_SPLITS, self.tc_splits)
        ctx.set_tuning(B.TUNE_TC_PAIRING, self.tc_pairing)


PAIRING_NAMES = {2: "single", 3: "pair"}
SHAPE_NAMES = {1: "cell", 2: "halfcell", 3: "quartercell"}


def _time(fn, stream, reps=3):
    ts = []
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts[1:])


def split_candidates(n_rows, n_sv, sms=152):
    """Split counts worth timing: the cost model's neighbourhood of whole-wave layouts."""
    mt = (n_rows + 127) // 128
    nt = max(1, (n_sv + 255) // 256)
    out = []
    for sp in range(1, nt + 1):
        tps = (nt + sp - 1) // sp
        if (nt + tps - 1) // tps != sp:
            continue  # not an exact split count
        if mt * sp <= 4 * sms:
            out.append(sp)
    return out[-8:] if len(out) > 8 else out


def _load_cache():
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(cache):
    try:
        os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)
    except OSError:
        pass


def tune(ctx, key, stage1, stage2, n_rows, n_sv, stream, use_cache=True, tensor_core=True):
    """Pick the fastest Tuning for the workload `key` (stage1 / stage2 enqueue the two stages
    on `stream`).  Returns (tuning, report)."""
    dev = torch.cuda.get_device_name()
    full_key = f"{dev}|{CACHE_VERSION}|{key}"
    cache = _load_cache() if use_cache else {}
    if full_key in cache:
        try:
            t = Tuning(**cache[full_key]["tuning"])
        except TypeError:
            t = None  # an entry written by another version of the knobs
        if t is not None:
            t.apply(ctx)
            return t, dict(cache[full_key], cached=True)
    report = {"k1": {}, "k2": {}}
    best = Tuning()
    # K1: tile shape x CTAs per SM
    best_ms = None
    for shape in (2, 1, 3):
        for c in ((2, 1) if shape != 3 else (1,)):  # a 1024-thread CTA fills an SM's registers
            ctx.set_tuning(B.TUNE_LBP_SHAPE, shape)
            ctx.set_tuning(B.TUNE_LBP_CTAS_PER_SM, c)
            ms = _time(stage1, stream)
            report["k1"][f"{SHAPE_NAMES[shape]}/{c}"] = ms
            if best_ms is None or ms < best_ms:
                best_ms, best.lbp_shape, best.lbp_ctas_per_sm = ms, shape, c
    ctx.set_tuning(B.TUNE_LBP_SHAPE, best.lbp_shape)
    ctx.set_tuning(B.TUNE_LBP_CTAS_PER_SM, best.lbp_ctas_per_sm)
    # K2: splits x CTA pairing
    if tensor_core:
        best_ms = None
        for sp in split_candidates(n_rows, n_sv, torch.cuda.get_device_properties(0).multi_processor_count):
            for pairing in (3, 2):
                ctx.set_tuning(B.TUNE_TC_SPLITS, sp)
                ctx.set_tuning(B.TUNE_TC_PAIRING, pairing)
                ms = _time(stage2, stream)
                report["k2"][f"{sp}/{PAIRING_NAMES[pairing]}"] = ms
                if best_ms is None or ms < best_ms:
                    best_ms, best.tc_splits, best.tc_pairing = ms, sp, pairing
    best.apply(ctx)
    entry = {"tuning": asdict(best), "report": report}
    cache[full_key] = entry
    if use_cache:
        _store_cache(cache)
    return best, dict(entry, cached=False)
