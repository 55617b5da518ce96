"""Autotuner for the scan's launch parameters.

Single text (``tune``): for one loaded machine, a coordinate descent over the
``pfsm_params`` axes (start-prefix depth, starts each thread filters per
round, filtering threads, tile length, persistent CTAs per SM, DFA table
placement, NFA settling cap). Starting from the library's defaults, each
axis in turn tries its values with the others fixed at the best found so
far, timed with CUDA events around the scan on one stream; two sweeps. The
result is cached in a JSON file keyed by (kind, |Q|, |Sigma|, GPU name), so a
machine of the same shape is tuned once per GPU model.

Batch (``tune_batch``): the launch shape of the batch class kernels (threads
and CTAs per SM, tile length), then per machine the DFA table placement
(shared-memory table arena or global memory) and the NFA settling cap, each
timed on a representative batch.

Every candidate computes the same match set; only the speed differs.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, List, Optional

import numpy as np

from . import (pfsm_get_params, pfsm_scan, pfsm_scan_async, pfsm_scan_batch,
               pfsm_scan_batch_async, pfsm_set_batch_params, pfsm_set_params)


def _default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "pfsm", "tune_cache.json")


CACHE_PATH = os.environ.get("PFSM_TUNE_CACHE") or _default_cache_path()
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
        d = os.path.dirname(CACHE_PATH)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = CACHE_PATH + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)


def axes(kind: str, S: int, default_k: int) -> Dict[str, list]:
    """The values tried on each axis, in the order the descent visits them."""
    sbits = max(1, int(np.ceil(np.log2(max(2, S)))))
    kmax = min(8, 16 // sbits)
    ks = sorted({k for k in (default_k - 1, default_k, kmax) if 1 <= k <= kmax})
    ax = {"prefix_k": ks, "spt": [32, 8], "threads": [512, 256],
          "tile": [0, 8192, 16384, 32768], "ctas_per_sm": [0, 1]}
    if kind == "dfa":
        ax["table_smem"] = [-1, 0, 1]
    else:
        # NFA settling cap: 16 by default; 8 measured faster on a motif NFA
        # once its starts reach settling 5 symbols past the prefix table
        ax["settle"] = [16, 8]
    return ax


def candidates(kind: str, S: int, default_k: int) -> List[dict]:
    """Every combination of the axes (an exhaustive search; ``tune`` walks
    the axes one at a time instead)."""
    out = [{}]
    for name, vals in axes(kind, S, default_k).items():
        out = [dict(p, **{name: v}) for p in out for v in vals]
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


def _descend(start: dict, ax: Dict[str, list], timer, sweeps: int = 2, gain: float = 0.99):
    """Coordinate descent: returns (best params, best ms, evaluations). A
    candidate replaces the best when it takes less than `gain` times its
    time."""
    best = dict(start)
    best_ms = timer(best)
    if best_ms is None:
        best_ms = float("inf")
    evals = 1
    seen = {json.dumps(best, sort_keys=True): best_ms}
    for _ in range(sweeps):
        moved = False
        for name, vals in ax.items():
            for v in vals:
                p = dict(best, **{name: v})
                key = json.dumps(p, sort_keys=True)
                if key in seen:
                    continue
                ms = timer(p)
                evals += 1
                seen[key] = ms if ms is not None else float("inf")
                if ms is not None and ms < best_ms * gain:
                    best, best_ms, moved = p, ms, True
        if not moved:
            break
    return best, best_ms, evals


def tune(ctx: int, aut: int, machine, sample_text, gpu_name: str = "", force: bool = False,
         reps: int = 3, sweeps: int = 2, use_cache: bool = True) -> dict:
    """Pick launch parameters for the loaded machine `aut` (host description
    `machine`, shaped like workloads.Dfa/Nfa) using `sample_text` (a CUDA
    uint8 tensor in the machine's alphabet). Sets and returns the chosen
    params (as pfsm_get_params reports them)."""
    import torch
    kind = "dfa" if hasattr(machine, "delta") else "nfa"
    Q = int(machine.Q)
    S = int(machine.S)
    if not gpu_name:
        gpu_name = torch.cuda.get_device_name(sample_text.device)
    key = _key(kind, Q, S, gpu_name)
    if use_cache and not force:
        cache = _load_cache()
        if key in cache:
            pfsm_set_params(ctx, aut, cache[key]["params"])
            return pfsm_get_params(ctx, aut)
    default = pfsm_get_params(ctx, aut)
    st, cnt = pfsm_scan(ctx, aut, sample_text, None, None, 0)
    out = torch.empty((int(cnt) + 1024, 3), dtype=torch.int32, device=sample_text.device)
    status = torch.zeros(2, dtype=torch.int64, device=sample_text.device)
    ax = axes(kind, S, max(1, default["prefix_k"]))
    start = dict(default)   # the fields not searched keep their values
    best, best_ms, _ = _descend(
        start, ax, lambda p: time_params(ctx, aut, sample_text, out, status, p, reps), sweeps)
    pfsm_set_params(ctx, aut, best)
    chosen = pfsm_get_params(ctx, aut)
    if use_cache:
        _store(key, chosen, best_ms)
    return chosen


def _time_batch(ctx, jobs, out, status, stream, reps) -> Optional[float]:
    import torch
    times = []
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            pfsm_scan_batch_async(ctx, jobs, out, status, stream=stream)
        except Exception:
            return None
        e1.record(stream)
        stream.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def tune_batch(ctx: int, jobs, reps: int = 3, stream=None, machines: Optional[dict] = None,
               sweeps: int = 1, warmup: int = 5, gain: float = 0.97) -> dict:
    """Pick the batch launch shape and per-machine placement for a
    representative batch `jobs` ([(aut, text_tensor, n), ...] or a job
    table) on the current CUDA device by timing
    each candidate with CUDA events (the median of `reps` runs after one
    untimed run; the batch runs `warmup` times first, so that the first
    candidate does not pay for the GPU's clocks ramping up). A candidate
    must beat the best so far by 1 - `gain` (3 %) to replace it. `machines`
    maps each automaton id of the batch to "dfa" or "nfa" (its per-machine
    axes are searched; omit it to tune the launch shape only). Sets the
    fastest and returns {"batch": shape, "machines": {aut: params}, "ms":
    time}."""
    import torch
    stream = stream or torch.cuda.current_stream()
    st, counts, total = pfsm_scan_batch(ctx, jobs, None, 0)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((int(total) + 1024, 4), dtype=torch.int32, device=dev)
    status = torch.zeros(len(jobs) + 2, dtype=torch.int64, device=dev)
    for _ in range(warmup):
        pfsm_scan_batch_async(ctx, jobs, out, status, stream=stream)
    stream.synchronize()

    # 1. launch shape: threads x CTAs per SM, then the tile
    def shape_timer(p):
        try:
            pfsm_set_batch_params(ctx, p)
        except Exception:
            return None
        return _time_batch(ctx, jobs, out, status, stream, reps)

    shape_axes = {"shape": [(0, 0), (256, 1), (256, 2), (512, 1), (128, 4)],
                  "tile": [16384, 8192, 32768]}

    def shape_params(p):
        threads, ctas = p["shape"]
        return {"threads": threads, "ctas_per_sm": ctas, "tile": p["tile"]}

    best, best_ms, _ = _descend({"shape": (0, 0), "tile": 16384}, shape_axes,
                                lambda p: shape_timer(shape_params(p)), sweeps, gain)
    shape = shape_params(best)
    pfsm_set_batch_params(ctx, shape)

    # 2. per machine: DFA table placement, NFA settling cap
    chosen = {}
    for aut, kind in (machines or {}).items():
        cur = pfsm_get_params(ctx, aut)
        ax = {"table_smem": [-1, 0]} if kind == "dfa" else {"settle": [16, 8]}
        name = next(iter(ax))
        best_v, best_v_ms = cur[name], best_ms
        for v in ax[name]:
            if v == cur[name]:
                continue
            try:
                pfsm_set_params(ctx, aut, dict(cur, **{name: v}))
            except Exception:
                continue
            ms = _time_batch(ctx, jobs, out, status, stream, reps)
            if ms is not None and ms < best_v_ms * gain:
                best_v, best_v_ms = v, ms
        pfsm_set_params(ctx, aut, dict(cur, **{name: best_v}))
        best_ms = min(best_ms, best_v_ms)
        chosen[aut] = {name: best_v}
    return {"batch": shape, "machines": chosen, "ms": best_ms}
