"""Autotuner for the scan's launch parameters.

For one loaded machine it times a small grid of ``pfsm_params`` candidates
(start-prefix depth, tile length, threads per CTA, persistent CTAs per SM)
on a sample text of the machine's alphabet, with CUDA events around the
scan on one stream, and keeps the fastest. Results are cached in a JSON file
keyed by (kind, |Q|, |Sigma|, GPU name), so a machine of the same shape is
tuned once per GPU model. Every candidate computes the same match set; only
the speed differs.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, List, Optional

import numpy as np

from . import (pfsm_get_params, pfsm_scan, pfsm_scan_async, pfsm_scan_batch,
               pfsm_scan_batch_async, pfsm_set_batch_params, pfsm_set_params)

CACHE_PATH = os.environ.get(
    "PFSM_TUNE_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json"))
_lock = threading.Lock()


def _key(kind: str, Q: int, S: int, gpu: str) -> str:
    return "%s/Q%d/S%d/%s" % (kind, Q, S, gpu)


def _load_cache() -> Dict[str, dict]:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(key: str, params: dict, ms: float):
    with _lock:
        c = _load_cache()
        c[key] = {"params": params, "ms": ms}
        tmp = CACHE_PATH + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)


def candidates(kind: str, S: int, default_k: int) -> List[dict]:
    sbits = max(1, int(np.ceil(np.log2(max(2, S)))))
    kmax = min(8, 16 // sbits)
    ks = sorted({k for k in (default_k - 1, default_k, default_k + 1, kmax) if 1 <= k <= kmax})
    # NFA settling cap: 16 by default; 8 measured faster on a motif NFA once
    # its starts reach settling 5 symbols past the prefix table
    settles = (8, 16) if kind == "nfa" else (0,)
    out = []
    for k in ks:
        for threads in (256, 512):
            for tile in (8192, 16384, 32768):
                for cps in (0, 1):
                    for settle in settles:
                        p = {"prefix_k": k, "threads": threads, "tile": tile, "halo": 2048,
                             "ctas_per_sm": cps}
                        if settle:
                            p["settle"] = settle
                        out.append(p)
    return out


def time_params(ctx: int, aut: int, text, out, status, params: dict, reps: int = 3,
                stream=None) -> Optional[float]:
    """Median CUDA-event time (ms) of one scan with `params`, or None when
    the combination does not fit the device."""
    import torch
    try:
        pfsm_set_params(ctx, aut, params)
    except Exception:
        return None
    stream = stream or torch.cuda.current_stream()
    times = []
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            pfsm_scan_async(ctx, aut, text, None, out, status, stream=stream)
        except Exception:
            return None
        e1.record(stream)
        stream.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def tune(ctx: int, aut: int, machine, sample_text, gpu_name: str = "", force: bool = False,
         reps: int = 3, max_candidates: int = 0) -> dict:
    """Pick launch parameters for the loaded machine `aut` (host description
    `machine`, shaped like workloads.Dfa/Nfa) using `sample_text` (a CUDA
    uint8 tensor in the machine's alphabet). Returns the chosen params."""
    import torch
    kind = "dfa" if hasattr(machine, "delta") else "nfa"
    Q = int(machine.Q)
    S = int(machine.S)
    if not gpu_name:
        gpu_name = torch.cuda.get_device_name(sample_text.device)
    key = _key(kind, Q, S, gpu_name)
    cache = _load_cache()
    if key in cache and not force:
        pfsm_set_params(ctx, aut, cache[key]["params"])
        return cache[key]["params"]
    default = pfsm_get_params(ctx, aut)
    st, cnt = pfsm_scan(ctx, aut, sample_text, None, None, 0)
    out = torch.empty((int(cnt) + 1024, 3), dtype=torch.int32, device=sample_text.device)
    status = torch.zeros(2, dtype=torch.int64, device=sample_text.device)
    best, best_ms = None, float("inf")
    cands = candidates(kind, S, max(1, default["prefix_k"]))
    if max_candidates:
        cands = cands[:max_candidates]
    for p in cands:
        ms = time_params(ctx, aut, sample_text, out, status, p, reps)
        if ms is not None and ms < best_ms:
            best, best_ms = p, ms
    if best is None:
        best = {}
    pfsm_set_params(ctx, aut, best)
    chosen = pfsm_get_params(ctx, aut)
    _store(key, chosen, best_ms)
    return chosen


def tune_batch(ctx: int, jobs, reps: int = 2, stream=None) -> dict:
    """Pick the batch launch shape (threads and CTAs per SM, tile length) for a
    representative batch `jobs` ([(aut, text_tensor, n), ...]) by timing each
    candidate with CUDA events; sets and returns the fastest."""
    import torch
    stream = stream or torch.cuda.current_stream()
    st, counts, total = pfsm_scan_batch(ctx, jobs, None, 0)
    dev = jobs[0][1].device if jobs else torch.device("cuda")
    out = torch.empty((int(total) + 1024, 4), dtype=torch.int32, device=dev)
    status = torch.zeros(len(jobs) + 2, dtype=torch.int64, device=dev)
    best, best_ms = None, float("inf")
    for threads, ctas in ((0, 0), (256, 1), (256, 2), (512, 1), (128, 4)):
        for tile in (8192, 16384, 32768):
            p = {"threads": threads, "ctas_per_sm": ctas, "tile": tile}
            try:
                pfsm_set_batch_params(ctx, p)
            except Exception:
                continue
            times = []
            for r in range(reps + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pfsm_scan_batch_async(ctx, jobs, out, status, stream=stream)
                e1.record(stream)
                stream.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            if ms < best_ms:
                best, best_ms = p, ms
    pfsm_set_batch_params(ctx, best)
    return dict(best or {}, ms=best_ms)
