"""Python binding of libpfsm (the GB300 PFSM scan library).

Thin ctypes marshalling over the C ABI declared in ``include/pfsm.h``: the
functions below carry the same names and arguments, take torch CUDA tensors
for device buffers and streams, and do no computation of their own. Every
step of a scan runs in the library's CUDA kernels; there is no CPU fallback:
if ``libpfsm.so`` is missing or cannot be loaded, importing the binding's
functions raises.

``Pfsm`` is a small convenience wrapper (a context plus load/scan helpers
that size the output and retry on overflow).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PFSM_CHECKED=1 in the environment selects the build whose device code tests
# its data-dependent indices (libpfsm_checked.so; build.build(checked=True))
LIB_PATH = os.path.join(_HERE, "libpfsm_checked.so" if os.environ.get("PFSM_CHECKED") == "1"
                        else "libpfsm.so")

PFSM_OK = 0
PFSM_E_INVAL = 1
PFSM_E_NOMEM = 2
PFSM_E_OVERFLOW = 3
PFSM_E_NOENT = 4
PFSM_E_TIMEOUT = 5
PFSM_E_CUDA = 6
PFSM_E_CHECK = 7

EXPORTS = ("pfsm_ctx_create", "pfsm_ctx_destroy", "pfsm_load_dfa", "pfsm_load_nfa",
           "pfsm_evict", "pfsm_unload", "pfsm_set_params", "pfsm_get_params", "pfsm_scan",
           "pfsm_scan_async", "pfsm_scan_batch", "pfsm_scan_batch_async", "pfsm_set_batch_params", "pfsm_get_stats", "pfsm_set_timing",
           "pfsm_kernel_time", "pfsm_strerror", "pfsm_scan_dfa_noalloc", "pfsm_aut_bytes",
           "pfsm_scan_union", "pfsm_scan_union_async", "pfsm_load_nfa_eps",
           "pfsm_test_hold_tiles", "pfsm_test_carry_cap")


class pfsm_params(ctypes.Structure):
    _fields_ = [("prefix_k", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("halo", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("spt", ctypes.c_int32), ("table_smem", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("settle", ctypes.c_int32),
                ("partition", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pfsm_stats(ctypes.Structure):
    _fields_ = [("resident_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("loads", ctypes.c_uint64), ("evictions", ctypes.c_uint64),
                ("reloads", ctypes.c_uint64), ("resident", ctypes.c_int32),
                ("loaded", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pfsm_job(ctypes.Structure):
    _fields_ = [("aut", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("text", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class PfsmError(RuntimeError):
    def __init__(self, status: int, what: str, required: Optional[int] = None):
        self.status = status
        self.required = required
        super().__init__("%s: %s (status %d)" % (what, strerror(status), status))


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpfsm.so (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("%s is not built: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` (the checked "
                           "build: paper_1110_1716_gb300.build.build(checked=True))" % path)
    lib = ctypes.CDLL(path)
    P, I32, U32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "pfsm_ctx_create": [ctypes.c_int, U64, ctypes.POINTER(P)],
        "pfsm_ctx_destroy": [P],
        "pfsm_load_dfa": [P, P, I32, I32, I32, I32, P, ctypes.POINTER(I32)],
        "pfsm_load_nfa": [P, P, I32, I32, I32, P, ctypes.POINTER(I32)],
        "pfsm_load_nfa_eps": [P, P, P, I32, I32, I32, P, ctypes.POINTER(I32)],
        "pfsm_evict": [P, I32],
        "pfsm_unload": [P, I32],
        "pfsm_set_params": [P, I32, ctypes.POINTER(pfsm_params)],
        "pfsm_get_params": [P, I32, ctypes.POINTER(pfsm_params)],
        "pfsm_scan": [P, I32, P, U64, P, U64, ctypes.POINTER(U64), P],
        "pfsm_scan_async": [P, I32, P, U64, P, U64, P, P],
        "pfsm_scan_batch": [P, P, I32, P, U64, P, ctypes.POINTER(U64), P],
        "pfsm_scan_batch_async": [P, P, I32, P, U64, P, P],
        "pfsm_set_batch_params": [P, ctypes.POINTER(pfsm_params)],
        "pfsm_get_stats": [P, ctypes.POINTER(pfsm_stats)],
        "pfsm_set_timing": [P, ctypes.c_int],
        "pfsm_test_hold_tiles": [P, I32],
        "pfsm_test_carry_cap": [P, U32, U32],
        "pfsm_kernel_time": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(U64)],
        "pfsm_strerror": [ctypes.c_int],
        "pfsm_scan_dfa_noalloc": [P, I32, I32, I32, I32, P, P, U64, P, U64, P, P],
        "pfsm_aut_bytes": [P, I32, ctypes.POINTER(U64), ctypes.POINTER(I32)],
        "pfsm_scan_union": [P, P, I32, P, U64, P, U64, P, ctypes.POINTER(U64), P],
        "pfsm_scan_union_async": [P, P, I32, P, U64, P, U64, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "pfsm_strerror" else ctypes.c_int
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load_library().pfsm_strerror(status).decode()


def _check(status: int, what: str, required: Optional[int] = None):
    if status != PFSM_OK:
        raise PfsmError(status, what, required)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dev_ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


# ---------------------------------------------------------------- C ABI names
def pfsm_ctx_create(device: int = 0, budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(load_library().pfsm_ctx_create(device, budget_bytes, ctypes.byref(h)),
           "pfsm_ctx_create")
    return h.value


def pfsm_ctx_destroy(ctx: int) -> None:
    _check(load_library().pfsm_ctx_destroy(ctx), "pfsm_ctx_destroy")


def pfsm_load_dfa(ctx: int, delta: np.ndarray, q0: int, dead: int,
                  is_final: np.ndarray) -> int:
    delta = np.ascontiguousarray(delta, dtype=np.int16)
    fin = np.ascontiguousarray(is_final, dtype=np.uint8)
    Q, S = delta.shape
    if fin.shape != (Q,):
        raise ValueError("is_final must have Q entries")
    out = ctypes.c_int32()
    _check(load_library().pfsm_load_dfa(ctx, delta.ctypes.data, Q, S, q0, dead, fin.ctypes.data,
                                        ctypes.byref(out)), "pfsm_load_dfa")
    return out.value


def pfsm_load_nfa(ctx: int, delta_bits: np.ndarray, q0: int, is_final: np.ndarray) -> int:
    bits = np.ascontiguousarray(delta_bits, dtype=np.uint32)
    fin = np.ascontiguousarray(is_final, dtype=np.uint8)
    Q, S, W = bits.shape
    if W != (Q + 31) // 32 or fin.shape != (Q,):
        raise ValueError("delta_bits must be [Q][S][ceil(Q/32)] and is_final [Q]")
    out = ctypes.c_int32()
    _check(load_library().pfsm_load_nfa(ctx, bits.ctypes.data, Q, S, q0, fin.ctypes.data,
                                        ctypes.byref(out)), "pfsm_load_nfa")
    return out.value


def pfsm_load_nfa_eps(ctx: int, delta_bits: np.ndarray, eps_bits: np.ndarray, q0: int,
                      is_final: np.ndarray) -> int:
    """An NFA whose epsilon edges (eps_bits [Q][ceil(Q/32)]) are followed at
    scan time."""
    bits = np.ascontiguousarray(delta_bits, dtype=np.uint32)
    eps = np.ascontiguousarray(eps_bits, dtype=np.uint32)
    fin = np.ascontiguousarray(is_final, dtype=np.uint8)
    Q, S, W = bits.shape
    if W != (Q + 31) // 32 or fin.shape != (Q,) or eps.shape != (Q, W):
        raise ValueError("delta_bits [Q][S][W], eps_bits [Q][W] and is_final [Q] expected")
    out = ctypes.c_int32()
    _check(load_library().pfsm_load_nfa_eps(ctx, bits.ctypes.data, eps.ctypes.data, Q, S, q0,
                                            fin.ctypes.data, ctypes.byref(out)), "pfsm_load_nfa_eps")
    return out.value


def pfsm_evict(ctx: int, aut: int) -> None:
    _check(load_library().pfsm_evict(ctx, aut), "pfsm_evict")


def pfsm_unload(ctx: int, aut: int) -> None:
    _check(load_library().pfsm_unload(ctx, aut), "pfsm_unload")


def pfsm_set_params(ctx: int, aut: int, params: Optional[dict] = None) -> None:
    p = None
    if params is not None:
        p = pfsm_params(**{k: int(v) for k, v in params.items()})
    _check(load_library().pfsm_set_params(ctx, aut, ctypes.byref(p) if p is not None else None),
           "pfsm_set_params")


def pfsm_get_params(ctx: int, aut: int) -> dict:
    p = pfsm_params()
    _check(load_library().pfsm_get_params(ctx, aut, ctypes.byref(p)), "pfsm_get_params")
    return p.as_dict()


def pfsm_scan(ctx: int, aut: int, text, n: Optional[int], out, cap: Optional[int] = None,
              stream=None):
    """Scan `n` bytes of the CUDA uint8 tensor `text` into the CUDA int32
    tensor `out` (shape [cap, 3]). Returns (status, n_matches): the caller
    checks for PFSM_E_OVERFLOW; every other non-OK status raises."""
    n = text.numel() if n is None else n
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    cnt = ctypes.c_uint64()
    st = load_library().pfsm_scan(ctx, aut, _dev_ptr(text), n, _dev_ptr(out), cap,
                                  ctypes.byref(cnt), _stream_ptr(stream))
    if st not in (PFSM_OK, PFSM_E_OVERFLOW):
        _check(st, "pfsm_scan")
    return st, cnt.value


def pfsm_scan_async(ctx: int, aut: int, text, n: Optional[int], out, status,
                    cap: Optional[int] = None, stream=None) -> None:
    """Enqueue a scan; `status` is a CUDA int64 tensor of 2 entries that
    receives (match count, error bits) when the stream reaches it."""
    n = text.numel() if n is None else n
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    _check(load_library().pfsm_scan_async(ctx, aut, _dev_ptr(text), n, _dev_ptr(out), cap,
                                          _dev_ptr(status), _stream_ptr(stream)),
           "pfsm_scan_async")


# numpy layout of pfsm_job, for building large job tables without a Python loop
JOB_DTYPE = np.dtype([("aut", "<i4"), ("reserved", "<u4"), ("text", "<u8"), ("n", "<u8")])


def job_table(auts, text_ptrs, lengths) -> np.ndarray:
    """A pfsm_job table as a numpy structured array (JOB_DTYPE) from three
    equal-length sequences: automaton ids, device text addresses, lengths.
    The batch functions accept it in place of a list of tuples."""
    t = np.zeros(len(auts), dtype=JOB_DTYPE)
    t["aut"] = auts
    t["text"] = text_ptrs
    t["n"] = lengths
    return t


def _job_array(jobs):
    """(pointer, count, keep-alive) of a job table given as a JOB_DTYPE array
    or as a sequence of (aut, text, n) tuples."""
    if isinstance(jobs, np.ndarray):
        if jobs.dtype != JOB_DTYPE:
            raise TypeError("job table must have dtype JOB_DTYPE")
        jobs = np.ascontiguousarray(jobs)
        return jobs.ctypes.data, len(jobs), jobs
    k = len(jobs)
    arr = (pfsm_job * max(1, k))()
    for i, (aut, text, n) in enumerate(jobs):
        arr[i].aut = aut
        arr[i].reserved = 0
        arr[i].text = text if isinstance(text, int) else _dev_ptr(text)
        arr[i].n = text.numel() if n is None else n
    return ctypes.addressof(arr), k, arr


def pfsm_scan_batch(ctx: int, jobs: Sequence, out, cap: Optional[int] = None, stream=None):
    """`jobs` = [(aut, text, n), ...] with `text` a CUDA uint8 tensor (or a
    device address and n given), or a ``job_table``; `out` CUDA int32
    [cap, 4] of (text, start, end, state) rows. Returns (status, per-job
    counts as uint64, total)."""
    ptr, k, _keep = _job_array(jobs)
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    counts = np.zeros(max(1, k), dtype=np.uint64)
    total = ctypes.c_uint64()
    st = load_library().pfsm_scan_batch(ctx, ptr, k, _dev_ptr(out), cap, counts.ctypes.data,
                                        ctypes.byref(total), _stream_ptr(stream))
    if st not in (PFSM_OK, PFSM_E_OVERFLOW):
        _check(st, "pfsm_scan_batch")
    return st, counts[:k], total.value


def pfsm_scan_batch_async(ctx: int, jobs: Sequence, out, status, cap: Optional[int] = None,
                          stream=None) -> None:
    """Enqueue a batch; `status` is a CUDA int64 tensor of len(jobs) + 2
    entries: (total, error bits, count of job 0, ...)."""
    ptr, k, _keep = _job_array(jobs)
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    _check(load_library().pfsm_scan_batch_async(ctx, ptr, k, _dev_ptr(out), cap,
                                                _dev_ptr(status), _stream_ptr(stream)),
           "pfsm_scan_batch_async")


def pfsm_scan_union(ctx: int, auts: Sequence[int], text, n: Optional[int], out,
                    cap: Optional[int] = None, stream=None):
    """Union machine over one CUDA text: (status, per-component counts,
    total); `out` rows are (component index, start, end, state)."""
    k = len(auts)
    a = np.ascontiguousarray(auts, dtype=np.int32)
    n = text.numel() if n is None else n
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    counts = np.zeros(max(1, k), dtype=np.uint64)
    total = ctypes.c_uint64()
    st = load_library().pfsm_scan_union(ctx, a.ctypes.data, k, _dev_ptr(text), n, _dev_ptr(out), cap,
                                        counts.ctypes.data, ctypes.byref(total), _stream_ptr(stream))
    if st not in (PFSM_OK, PFSM_E_OVERFLOW):
        _check(st, "pfsm_scan_union")
    return st, counts[:k], total.value


def pfsm_scan_union_async(ctx: int, auts: Sequence[int], text, n: Optional[int], out, status,
                          cap: Optional[int] = None, stream=None) -> None:
    """Enqueue a union scan; `status` as for pfsm_scan_batch_async."""
    a = np.ascontiguousarray(auts, dtype=np.int32)
    n = text.numel() if n is None else n
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    _check(load_library().pfsm_scan_union_async(ctx, a.ctypes.data, len(a), _dev_ptr(text), n,
                                                _dev_ptr(out), cap, _dev_ptr(status),
                                                _stream_ptr(stream)), "pfsm_scan_union_async")


def pfsm_set_batch_params(ctx: int, params: Optional[dict] = None) -> None:
    """Batch launch shape: {"threads": 0|128|256|512, "ctas_per_sm": 0..4,
    "tile": 4096..32768}; 0 (or None for all) selects the per-class defaults."""
    p = None
    if params is not None:
        p = pfsm_params(**{k: int(v) for k, v in params.items()})
    _check(load_library().pfsm_set_batch_params(ctx, ctypes.byref(p) if p is not None else None),
           "pfsm_set_batch_params")


def pfsm_get_stats(ctx: int) -> dict:
    s = pfsm_stats()
    _check(load_library().pfsm_get_stats(ctx, ctypes.byref(s)), "pfsm_get_stats")
    return s.as_dict()


def pfsm_aut_bytes(ctx: int, aut: int):
    """(device bytes of `aut` while resident, resident now)."""
    b = ctypes.c_uint64()
    r = ctypes.c_int32()
    _check(load_library().pfsm_aut_bytes(ctx, aut, ctypes.byref(b), ctypes.byref(r)), "pfsm_aut_bytes")
    return b.value, bool(r.value)


def pfsm_test_hold_tiles(ctx: int, enable: bool) -> None:
    """Test hook for the timeout path (see include/pfsm.h)."""
    _check(load_library().pfsm_test_hold_tiles(ctx, 1 if enable else 0), "pfsm_test_hold_tiles")


def pfsm_test_carry_cap(ctx: int, entries: int = 0, pool_states: int = 0) -> None:
    """Test hook for a full carry queue (see include/pfsm.h)."""
    _check(load_library().pfsm_test_carry_cap(ctx, entries, pool_states), "pfsm_test_carry_cap")


def pfsm_set_timing(ctx: int, enable: bool) -> None:
    _check(load_library().pfsm_set_timing(ctx, 1 if enable else 0), "pfsm_set_timing")


def pfsm_kernel_time(ctx: int):
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(load_library().pfsm_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)),
           "pfsm_kernel_time")
    return ms.value, n.value


def pfsm_strerror(status: int) -> str:
    return strerror(status)


def pfsm_scan_dfa_noalloc(delta, q0: int, dead: int, is_final, text, n: Optional[int], out,
                          status, cap: Optional[int] = None, stream=None) -> None:
    """Allocation-free DFA scan on caller buffers: `delta` CUDA int16 [Q, S],
    `is_final` CUDA uint8 [Q], `text` CUDA uint8, `out` CUDA int32 [cap, 3],
    `status` CUDA int64 [2] receiving (match count, error bits)."""
    Q, S = delta.shape
    n = text.numel() if n is None else n
    cap = (out.shape[0] if out is not None else 0) if cap is None else cap
    _check(load_library().pfsm_scan_dfa_noalloc(_dev_ptr(delta), Q, S, q0, dead,
                                                _dev_ptr(is_final), _dev_ptr(text), n,
                                                _dev_ptr(out), cap, _dev_ptr(status),
                                                _stream_ptr(stream)),
           "pfsm_scan_dfa_noalloc")


# ---------------------------------------------------------------- convenience
class Pfsm:
    """A context on one CUDA device with load/scan helpers.

    ``load`` takes objects shaped like ``workloads.Dfa`` (delta, q0, dead,
    final) or ``workloads.Nfa`` (bits, q0, final); ``scan`` returns the
    matches as a CUDA int32 tensor of (start, end, state) rows (unordered).
    """

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = pfsm_ctx_create(device, budget_bytes)

    def close(self):
        if self.ctx:
            pfsm_ctx_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, aut) -> int:
        """Load a workloads.Dfa or Nfa; an Nfa with epsilon edges keeps them
        for the scan to follow (pfsm_load_nfa_eps)."""
        if hasattr(aut, "delta"):
            return pfsm_load_dfa(self.ctx, aut.delta, aut.q0, aut.dead, aut.final)
        if getattr(aut, "eps", None) is not None:
            return pfsm_load_nfa_eps(self.ctx, aut.bits, aut.eps, aut.q0, aut.final)
        return pfsm_load_nfa(self.ctx, aut.bits, aut.q0, aut.final)

    def to_device(self, text: np.ndarray):
        t = self.torch.from_numpy(np.ascontiguousarray(text, dtype=np.uint8))
        return t.to("cuda:%d" % self.device)

    def scan(self, aut: int, text, cap: Optional[int] = None, stream=None):
        torch = self.torch
        if isinstance(text, np.ndarray):
            text = self.to_device(text)
        n = text.numel()
        cap = max(1024, n // 2) if cap is None else cap
        while True:
            out = torch.empty((cap, 3), dtype=torch.int32, device=text.device)
            st, cnt = pfsm_scan(self.ctx, aut, text, n, out, cap, stream)
            if st == PFSM_OK:
                return out[:cnt]
            cap = int(cnt)

    def scan_batch(self, jobs, cap: Optional[int] = None, stream=None):
        """jobs = [(aut, text), ...] (numpy or CUDA texts). Returns
        (matches as an int32 CUDA tensor of (text, start, end, state) rows,
        per-job counts)."""
        torch = self.torch
        dj = []
        for aut, text in jobs:
            if isinstance(text, np.ndarray):
                text = self.to_device(text)
            dj.append((aut, text, text.numel()))
        total_n = sum(x[2] for x in dj)
        cap = max(1024, total_n // 2) if cap is None else cap
        while True:
            out = torch.empty((cap, 4), dtype=torch.int32, device="cuda:%d" % self.device)
            st, counts, total = pfsm_scan_batch(self.ctx, dj, out, cap, stream)
            if st == PFSM_OK:
                return out[:total], counts
            cap = int(total)

    def scan_numpy(self, aut: int, text, cap: Optional[int] = None) -> np.ndarray:
        """Matches as an (m, 3) uint32 numpy array (unordered)."""
        return self.scan(aut, text, cap).cpu().numpy().view(np.uint32)
