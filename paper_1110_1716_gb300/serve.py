"""Continuous-batching scan server on one GPU.

Requests (machine, text) arrive at any time. A scheduler thread admits them
into batch slots as device memory and slots free up: each slot owns a CUDA
stream, a device text arena, a device match buffer and pinned host mirrors.
Admitted requests are packed into the slot's arena, copied to the device and
scanned with one ``pfsm_scan_batch_async`` call (one persistent launch replayed
from a CUDA graph); while a slot's batch runs, newly arrived requests fill
the next free slot, so batches from several slots overlap on the device.

Machines stay resident on the device under the context's byte budget; the
library evicts the least recently used ones and reloads them when a batch
names them again (cold machines leave fast memory, Sec. I-II's insomnia).

Each request's result is its own match set, bit-identical to a scan of that
text alone; latency is measured from arrival to the moment its matches are
on the host.
"""
from __future__ import annotations

import collections
import gc
import threading
import time
from concurrent.futures import Future
from typing import Dict, List, Optional

import numpy as np

from . import (PFSM_E_NOMEM, PFSM_OK, Pfsm, PfsmError, pfsm_aut_bytes, pfsm_get_stats,
               pfsm_scan_batch, pfsm_scan_batch_async)


class Request:
    __slots__ = ("rid", "aut", "text", "arrival", "future", "t_done")

    def __init__(self, rid, aut, text, arrival):
        self.rid = rid
        self.aut = aut
        self.text = text
        self.arrival = arrival
        self.future = Future()
        self.t_done = None


def pack_batch(pending, max_jobs: int, text_bytes: int, aut_bytes, budget: int,
               one_machine: bool = False):
    """Take requests from the front of `pending` (a deque of objects with
    .aut and .text) for one batch, in arrival order: at most `max_jobs`, their
    texts (each padded to 16 bytes) within `text_bytes` (the first one that
    does not fit ends the batch), and only while the batch's distinct
    machines fit the residency `budget` together (`aut_bytes[aut]` device
    bytes each; a request whose machine would not fit is left at the front
    for the next batch; the first machine is always taken). With
    `one_machine`, only requests for the first pending request's machine are
    taken. At most 4 * max_jobs requests are examined. Returns (requests,
    arena bytes used)."""
    reqs, used, skipped = [], 0, []
    machines, mbytes = set(), 0
    first = pending[0].aut if pending else None
    scanned = 0
    while pending and len(reqs) < max_jobs and scanned < 4 * max_jobs:
        r = pending[0]
        if used + len(r.text) > text_bytes:
            break
        pending.popleft()
        scanned += 1
        new = r.aut not in machines
        if (one_machine and r.aut != first) or (
                new and machines and mbytes + aut_bytes[r.aut] > budget):
            skipped.append(r)
            continue
        if new:
            machines.add(r.aut)
            mbytes += aut_bytes[r.aut]
        reqs.append(r)
        used += (len(r.text) + 15) & ~15
    for r in reversed(skipped):
        pending.appendleft(r)
    return reqs, used


class _Slot:
    def __init__(self, torch, dev, text_bytes, out_rows, max_jobs):
        self.stream = torch.cuda.Stream(device=dev)
        self.text_dev = torch.empty(text_bytes, dtype=torch.uint8, device=dev)
        self.text_host = torch.empty(text_bytes, dtype=torch.uint8).pin_memory()
        self.out_dev = torch.empty((out_rows, 4), dtype=torch.int32, device=dev)
        self.out_host = torch.empty((out_rows, 4), dtype=torch.int32).pin_memory()
        self.status_dev = torch.zeros(max_jobs + 2, dtype=torch.int64, device=dev)
        self.status_host = torch.zeros(max_jobs + 2, dtype=torch.int64).pin_memory()
        self.done = torch.cuda.Event()
        self.reqs: List[Request] = []
        self.busy = False
        self.t_launch = 0.0
        self.text_bytes = text_bytes
        self.out_rows = out_rows
        self.max_jobs = max_jobs


class Server:
    """Scan server over a ``Pfsm`` context.

    automata     machines (``workloads.Dfa``/``Nfa``-shaped); request.aut
                 indexes this list
    slots        batch slots = CUDA streams with their own buffers
    slot_bytes   text arena per slot (the largest request must fit)
    out_rows     match capacity per slot (a batch that overflows is rerun
                 synchronously with the exact capacity)
    max_jobs     requests per batch
    """

    def __init__(self, pf: Pfsm, automata, slots: int = 3, slot_bytes: int = 64 << 20,
                 out_rows: int = 4 << 20, max_jobs: int = 1024):
        import torch
        if not 1 <= max_jobs <= 65535:   # batch job indices are grouped as 16-bit keys
            raise ValueError("max_jobs must be in [1, 65535]")
        self.torch = torch
        self.pf = pf
        self.ids = [pf.load(a) for a in automata]
        # device bytes of each machine and the context's budget: a batch
        # takes requests only while its distinct machines fit together
        self.aut_bytes = [pfsm_aut_bytes(pf.ctx, i)[0] for i in self.ids]
        self.budget = pfsm_get_stats(pf.ctx)["budget_bytes"]
        dev = torch.device("cuda", pf.device)
        self.slots = [_Slot(torch, dev, slot_bytes, out_rows, max_jobs) for _ in range(slots)]
        self.pending = collections.deque()
        self.lock = threading.Condition()
        self.running = False
        self.thread = None
        # latency (s) of every completed request; finished Request objects are
        # not kept, so the interpreter's cycle collector has less to scan
        self.latencies: List[float] = []
        self.max_loop_gap_s = 0.0
        self.max_loop_gap_at = 0.0
        self.max_loop_gap_parts = {}
        self.max_batch_s = 0.0
        self.max_admit_s = 0.0
        self.max_complete_s = 0.0
        self.batches = 0
        self.overflow_reruns = 0
        self.nomem_splits = 0
        self.bytes_scanned = 0
        self.next_rid = 0

    # -------------------------------------------------------------- client side
    def submit(self, aut: int, text: np.ndarray, arrival: Optional[float] = None) -> Future:
        text = np.ascontiguousarray(text, dtype=np.uint8)
        if len(text) > self.slots[0].text_bytes:
            raise ValueError("request larger than a slot's text arena")
        with self.lock:
            r = Request(self.next_rid, aut, text, time.perf_counter() if arrival is None else arrival)
            self.next_rid += 1
            self.pending.append(r)
            self.lock.notify()
        return r.future

    def start(self):
        self.running = True
        self.thread = threading.Thread(target=self._loop, name="pfsm-serve", daemon=True)
        self.thread.start()
        return self

    def stop(self):
        with self.lock:
            self.running = False
            self.lock.notify()
        if self.thread:
            self.thread.join()

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.stop()
        return False

    # -------------------------------------------------------------- scheduler
    def _admit(self, slot: _Slot, one_machine: bool = False) -> bool:
        """Pack pending requests into a free slot (``pack_batch``) and launch
        its batch."""
        with self.lock:
            reqs, used = pack_batch(self.pending, slot.max_jobs, slot.text_bytes, self.aut_bytes,
                                    self.budget, one_machine)
        if not reqs:
            return False
        torch = self.torch
        host = slot.text_host.numpy()
        jobs, off = [], 0
        base = slot.text_dev.data_ptr()
        for r in reqs:
            n = len(r.text)
            host[off:off + n] = r.text
            jobs.append((self.ids[r.aut], base + off, n))
            off += (n + 15) & ~15
        try:
            with torch.cuda.stream(slot.stream):
                slot.text_dev[:off].copy_(slot.text_host[:off], non_blocking=True)
                pfsm_scan_batch_async(self.pf.ctx, jobs, slot.out_dev,
                                      slot.status_dev[:len(jobs) + 2], stream=slot.stream)
                slot.status_host[:len(jobs) + 2].copy_(slot.status_dev[:len(jobs) + 2],
                                                       non_blocking=True)
                slot.done.record(slot.stream)
        except PfsmError as e:
            slot.stream.synchronize()
            if e.status == PFSM_E_NOMEM and not one_machine:
                # the batch's machines exceed the budget together: requeue
                # and retry with one machine per batch
                with self.lock:
                    for r in reversed(reqs):
                        self.pending.appendleft(r)
                self.nomem_splits += 1
                return self._admit(slot, one_machine=True)
            for r in reqs:
                r.future.set_exception(e)
            return True
        slot.reqs = reqs
        slot.jobs = jobs
        slot.busy = True
        slot.t_launch = time.perf_counter()
        self.batches += 1
        self.bytes_scanned += used
        return True

    def _complete(self, slot: _Slot):
        st = slot.status_host.numpy()
        k = len(slot.reqs)
        total, err = int(st[0]), int(st[1])
        counts = st[2:2 + k].astype(np.int64)
        if err:
            exc = RuntimeError("scan error bits %d" % err)
            for r in slot.reqs:
                r.future.set_exception(exc)
        else:
            torch = self.torch
            if total > slot.out_rows:
                # overflow: rerun this batch synchronously with room for all
                self.overflow_reruns += 1
                out = torch.empty((total, 4), dtype=torch.int32, device=slot.out_dev.device)
                s2, counts2, total2 = pfsm_scan_batch(self.pf.ctx, slot.jobs, out, total,
                                                      stream=slot.stream)
                m = out[:total2].cpu().numpy().view(np.uint32)
            else:
                with torch.cuda.stream(slot.stream):
                    slot.out_host[:total].copy_(slot.out_dev[:total], non_blocking=True)
                slot.stream.synchronize()
                m = slot.out_host[:total].numpy().view(np.uint32)
            # group the rows by request: job indices fit 16 bits (a batch holds
            # at most max_jobs <= 65535 requests), for which numpy's stable
            # sort is a radix sort, linear in the number of matches
            order = np.argsort(m[:, 0].astype(np.uint16), kind="stable")
            m = m[order]
            bounds = np.searchsorted(m[:, 0], np.arange(k + 1))
            now = time.perf_counter()
            self.max_batch_s = max(self.max_batch_s, now - slot.t_launch)
            for i, r in enumerate(slot.reqs):
                r.t_done = now
                r.future.set_result(m[bounds[i]:bounds[i + 1], 1:])
                self.latencies.append(now - r.arrival)
        slot.reqs = []
        slot.busy = False

    def _loop(self):
        try:
            self._run()
        except BaseException as e:   # never leave futures hanging
            with self.lock:
                pend = list(self.pending)
                self.pending.clear()
            for r in pend + [r for s in self.slots for r in s.reqs]:
                if not r.future.done():
                    r.future.set_exception(e)
            raise

    def _run(self):
        while True:
            progressed = False
            for slot in self.slots:
                if slot.busy and slot.done.query():
                    self._complete(slot)
                    progressed = True
            for slot in self.slots:
                if not slot.busy:
                    if self._admit(slot):
                        progressed = True
            with self.lock:
                if not self.running and not self.pending and not any(s.busy for s in self.slots):
                    return
                if not progressed and not any(s.busy for s in self.slots):
                    self.lock.wait(timeout=0.001)
            if not progressed:
                time.sleep(20e-6)

    def run_trace(self, arrivals: np.ndarray, auts: np.ndarray, texts,
                  t0: Optional[float] = None) -> List[Future]:
        """Serve a recorded request trace in real time on the calling thread:
        each pass of the loop moves every request whose arrival time has come
        into the pending queue, completes finished batches and launches new
        ones on free slots. Latency counts from the scheduled arrival."""
        if self.running:
            raise RuntimeError("run_trace needs the scheduler thread stopped")
        # the interpreter's cycle collector stops the whole loop for tens of
        # milliseconds once many objects are alive: pause it for the trace and
        # re-enable it afterwards (reference counting still frees everything
        # that is not in a cycle)
        gc_was_enabled = gc.isenabled()
        gc.disable()
        t0 = time.perf_counter() if t0 is None else t0
        due = t0 + np.asarray(arrivals, dtype=np.float64)
        futs: List[Future] = []
        i, k = 0, len(due)
        self.running = True
        prev = time.perf_counter()
        prev_cpu = time.thread_time()
        parts = [0.0, 0.0, 0.0, 0.0]   # the last pass: intake, completion, admission, sleep
        try:
            while True:
                now = time.perf_counter()
                cpu = time.thread_time()
                # the longest pass of the loop (a stall of the host thread, as
                # opposed to a batch that took long on the device), with where
                # its time went and how much of it this thread was on a CPU
                if now - prev > self.max_loop_gap_s:
                    self.max_loop_gap_s = now - prev
                    self.max_loop_gap_at = now - t0
                    self.max_loop_gap_parts = {
                        "intake_ms": parts[0] * 1e3, "complete_ms": parts[1] * 1e3,
                        "admit_ms": parts[2] * 1e3, "sleep_ms": parts[3] * 1e3,
                        "thread_cpu_ms": (cpu - prev_cpu) * 1e3}
                prev = now
                prev_cpu = cpu
                with self.lock:
                    while i < k and due[i] <= now:
                        r = Request(self.next_rid, int(auts[i]),
                                    np.ascontiguousarray(texts[i], dtype=np.uint8), float(due[i]))
                        self.next_rid += 1
                        self.pending.append(r)
                        futs.append(r.future)
                        i += 1
                t1 = time.perf_counter()
                progressed = False
                for slot in self.slots:
                    if slot.busy and slot.done.query():
                        tc = time.perf_counter()
                        self._complete(slot)
                        self.max_complete_s = max(self.max_complete_s, time.perf_counter() - tc)
                        progressed = True
                t2 = time.perf_counter()
                for slot in self.slots:
                    if not slot.busy:
                        ta = time.perf_counter()
                        if self._admit(slot):
                            progressed = True
                        self.max_admit_s = max(self.max_admit_s, time.perf_counter() - ta)
                t3 = time.perf_counter()
                if i >= k and not self.pending and not any(s.busy for s in self.slots):
                    break
                if not progressed:
                    nxt = due[i] if i < k else now + 20e-6
                    time.sleep(max(0.0, min(nxt - time.perf_counter(), 20e-6)))
                parts = [t1 - now, t2 - t1, t3 - t2, time.perf_counter() - t3]
        finally:
            self.running = False
            if gc_was_enabled:
                gc.enable()
        return futs

    # -------------------------------------------------------------- reporting
    def reset_stats(self):
        """Forget completed requests and counters (between measured runs)."""
        self.latencies = []
        self.max_loop_gap_s = 0.0   # longest pass of the trace loop
        self.max_loop_gap_at = 0.0  # its end, in seconds from the trace start
        self.max_loop_gap_parts = {}  # that pass: time per step and on-CPU time
        self.max_batch_s = 0.0      # longest batch, launch to completion seen
        self.max_admit_s = 0.0      # longest packing + launch of a batch
        self.max_complete_s = 0.0   # longest hand-back of a batch's results
        self.batches = 0
        self.overflow_reruns = 0
        self.nomem_splits = 0
        self.bytes_scanned = 0

    def latency_stats(self) -> Dict[str, float]:
        lat = np.asarray(self.latencies, dtype=np.float64)
        if len(lat) == 0:
            return {}
        return {"requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "batches": self.batches,
                "max_loop_gap_ms": self.max_loop_gap_s * 1e3,
                "max_loop_gap_at_s": self.max_loop_gap_at,
                "max_loop_gap_parts": dict(self.max_loop_gap_parts),
                "max_batch_ms": self.max_batch_s * 1e3,
                "max_admit_ms": self.max_admit_s * 1e3,
                "max_complete_ms": self.max_complete_s * 1e3,
                "overflow_reruns": self.overflow_reruns, "nomem_splits": self.nomem_splits, **{
                    "residency_" + k: v for k, v in pfsm_get_stats(self.pf.ctx).items()}}


def replay(server: Server, arrivals: np.ndarray, auts: np.ndarray, texts, t0: Optional[float] = None):
    """Submit requests at their arrival offsets (seconds) in real time, from
    the calling thread; returns the futures. `texts[i]` is request i's text.
    (For load tests prefer ``Server.run_trace``, which admits arrivals from
    the scheduler's own loop and so measures the server, not a second
    Python thread competing for the interpreter.)"""
    t0 = time.perf_counter() if t0 is None else t0
    futs = []
    for i in range(len(arrivals)):
        due = t0 + float(arrivals[i])
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            time.sleep(min(due - now, 1e-3))
        futs.append(server.submit(int(auts[i]), texts[i], arrival=due))
    return futs
