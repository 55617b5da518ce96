"""CPU oracle for the PFSM scan. TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package. The CUDA library never imports, links or calls it, and
this package imports nothing from the library.

Three independent ways to compute the match set
M(t, A) = {(i, j, f) : i <= j < n, f in F, f in delta^({q0}, t[i..j])}:

* ``scan_dfa`` / ``scan_nfa`` / ``run_segment``: the paper's tagged-state
  procedure (Sec. III.B), in plain C (``pfsm_oracle.c``).
* ``brute_force``: the definition read directly, i.e. the acalculia procedure
  of Sec. II: restart the machine at every position and stop at every end,
  with sets of states and epsilon closures. Pure Python, tiny inputs only.
* ``literal_occurrences``: for a set of literal strings, M is the set of all
  their occurrences; found here with ``bytes.find``.

``pair_steps`` gives the work of the tagged-state procedure: the number of
(start, state) pairs it advances over a symbol, summed over the text
(``brute_force_pair_steps`` computes the same number by definition).

Matches are returned as uint32 arrays of shape (m, 3) holding
(start, end, state) rows sorted lexicographically; ``end`` is inclusive
(Fig. 2 of the paper lists "c" at [2-2]).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place with gcc (plain C99, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    P, I, U64, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
    lib.oracle_scan_dfa.restype = I64
    lib.oracle_scan_dfa.argtypes = [P, I, I, I, I, P, P, U64, U64, U64, P, I64, P]
    lib.oracle_scan_nfa.restype = I64
    lib.oracle_scan_nfa.argtypes = [P, I, I, I, P, P, U64, U64, U64, P, I64, P]
    lib.oracle_run_segment.restype = I64
    lib.oracle_run_segment.argtypes = [P, P, I, I, I, I, P, P, U64, U64, U64, U64,
                                       P, U64, P, I64, P, I64, P, P]
    lib.oracle_pair_steps.restype = I64
    lib.oracle_pair_steps.argtypes = [P, P, I, I, I, I, P, P, U64, U64, U64, P, P]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        _bind(lib)
        _lib = lib
    return _lib


class using_library:
    """Context manager: route the oracle calls through another build of
    ``pfsm_oracle.c`` (the tests use it to show that copies with planted
    mistakes fail the pins)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.prev = _lib
        lib = ctypes.CDLL(self.path)
        _bind(lib)
        _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev
        return False


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def sort_matches(m: np.ndarray) -> np.ndarray:
    m = np.asarray(m, dtype=np.uint32).reshape(-1, 3)
    if len(m) == 0:
        return m
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0]))
    return m[order]


def _call_scan(fn, args, cap_guess):
    cap = max(16, int(cap_guess))
    while True:
        out = np.empty((cap, 3), dtype=np.uint32)
        err = ctypes.c_int(0)
        cnt = fn(*args, _ptr(out), cap, ctypes.byref(err))
        if cnt < 0:
            raise ValueError("oracle error %d" % err.value)
        if cnt <= cap:
            return sort_matches(out[:cnt])
        cap = int(cnt)


def scan_dfa(delta: np.ndarray, q0: int, dead: int, final: np.ndarray, text: np.ndarray,
             s_lo: int = 0, s_hi: Optional[int] = None) -> np.ndarray:
    """Matches of a DFA-form table whose start lies in [s_lo, s_hi)."""
    delta = np.ascontiguousarray(delta, dtype=np.int16)
    final = np.ascontiguousarray(final, dtype=np.uint8)
    text = np.ascontiguousarray(text, dtype=np.uint8)
    Q, S = delta.shape
    n = len(text)
    s_hi = n if s_hi is None else s_hi
    args = (_ptr(delta), Q, S, q0, dead, _ptr(final), _ptr(text), n, s_lo, s_hi)
    return _call_scan(_load().oracle_scan_dfa, args, 2 * max(1, s_hi - s_lo))


def scan_nfa(bits: np.ndarray, q0: int, final: np.ndarray, text: np.ndarray,
             s_lo: int = 0, s_hi: Optional[int] = None) -> np.ndarray:
    """Matches of an NFA-form (bitset rows) table whose start lies in [s_lo, s_hi)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    final = np.ascontiguousarray(final, dtype=np.uint8)
    text = np.ascontiguousarray(text, dtype=np.uint8)
    Q, S, W = bits.shape
    assert W == (Q + 31) // 32
    n = len(text)
    s_hi = n if s_hi is None else s_hi
    args = (_ptr(bits), Q, S, q0, _ptr(final), _ptr(text), n, s_lo, s_hi)
    return _call_scan(_load().oracle_scan_nfa, args, 2 * max(1, s_hi - s_lo))


def scan(aut, text: np.ndarray, s_lo: int = 0, s_hi: Optional[int] = None) -> np.ndarray:
    """Either form, from an object with the attributes of ``workloads.Dfa``
    (delta, q0, dead, final) or ``workloads.Nfa`` (bits, q0, final, eps=None)."""
    if hasattr(aut, "delta"):
        return scan_dfa(aut.delta, aut.q0, aut.dead, aut.final, text, s_lo, s_hi)
    if getattr(aut, "eps", None) is not None:
        raise ValueError("the oracle takes epsilon-free machines; remove epsilon edges first")
    return scan_nfa(aut.bits, aut.q0, aut.final, text, s_lo, s_hi)


def run_segment(aut, text: np.ndarray, j_begin: int, j_end: int, reinit_lo: int,
                reinit_hi: int, in_pairs: Optional[np.ndarray] = None):
    """One segment of chained data partitioning (Sec. III.D.2).

    Processes positions [j_begin, j_end) reinitialising on
    [reinit_lo, reinit_hi), starting from ``in_pairs`` (k, 2) uint32 rows of
    (tag, state). Returns (matches, out_pairs) where out_pairs are the tagged
    states still active after position j_end - 1.
    """
    text = np.ascontiguousarray(text, dtype=np.uint8)
    final = np.ascontiguousarray(aut.final, dtype=np.uint8)
    if hasattr(aut, "delta"):
        delta = np.ascontiguousarray(aut.delta, dtype=np.int16)
        bits = None
        Q, S = delta.shape
        dead = aut.dead
    else:
        delta = None
        bits = np.ascontiguousarray(aut.bits, dtype=np.uint32)
        Q, S, _ = bits.shape
        dead = -1
    if in_pairs is None:
        in_pairs = np.zeros((0, 2), dtype=np.uint32)
    in_pairs = np.ascontiguousarray(in_pairs, dtype=np.uint32).reshape(-1, 2)
    lib = _load()
    cap = max(16, 2 * (j_end - j_begin))
    acap = max(16, 4 * len(in_pairs) + 64)
    while True:
        out = np.empty((cap, 3), dtype=np.uint32)
        act = np.empty((acap, 2), dtype=np.uint32)
        n_act = ctypes.c_int64(0)
        err = ctypes.c_int(0)
        cnt = lib.oracle_run_segment(_ptr(delta), _ptr(bits), Q, S, aut.q0, dead, _ptr(final),
                                     _ptr(text), j_begin, j_end, reinit_lo, reinit_hi,
                                     _ptr(in_pairs), len(in_pairs), _ptr(out), cap, _ptr(act),
                                     acap, ctypes.byref(n_act), ctypes.byref(err))
        if cnt < 0:
            raise ValueError("oracle error %d" % err.value)
        if cnt <= cap and n_act.value <= acap:
            return sort_matches(out[:cnt]), act[:n_act.value].copy()
        cap = max(cap, int(cnt))
        acap = max(acap, int(n_act.value))


def pair_steps(aut, text: np.ndarray, s_lo: int = 0, s_hi: Optional[int] = None):
    """Work of the tagged-state procedure (Sec. III.B) for the starts in
    [s_lo, s_hi): (pair_steps, matches), where pair_steps counts the (tag,
    state) pairs advanced over a symbol, summed over the positions, and
    matches is the size of the match set (not stored)."""
    text = np.ascontiguousarray(text, dtype=np.uint8)
    final = np.ascontiguousarray(aut.final, dtype=np.uint8)
    if getattr(aut, "eps", None) is not None:
        raise ValueError("the oracle takes epsilon-free machines; remove epsilon edges first")
    if hasattr(aut, "delta"):
        delta = np.ascontiguousarray(aut.delta, dtype=np.int16)
        bits = None
        Q, S = delta.shape
        dead = aut.dead
    else:
        delta = None
        bits = np.ascontiguousarray(aut.bits, dtype=np.uint32)
        Q, S, _ = bits.shape
        dead = -1
    n = len(text)
    s_hi = n if s_hi is None else s_hi
    work = ctypes.c_uint64(0)
    err = ctypes.c_int(0)
    cnt = _load().oracle_pair_steps(_ptr(delta), _ptr(bits), Q, S, aut.q0, dead, _ptr(final),
                                    _ptr(text), n, s_lo, s_hi, ctypes.byref(work),
                                    ctypes.byref(err))
    if cnt < 0:
        raise ValueError("oracle error %d" % err.value)
    return int(work.value), int(cnt)


# ----------------------------------------------------------------------------
# The definition, read directly (Sec. II, acalculia by exhaustive restarts)
# ----------------------------------------------------------------------------
def _succ_sets(aut):
    """delta as Python sets: succ[q][a] -> set of states; eps[q] -> set."""
    if hasattr(aut, "delta"):
        Q, S = aut.delta.shape
        succ = [[{int(aut.delta[q, a])} for a in range(S)] for q in range(Q)]
        return Q, S, succ, [set() for _ in range(Q)]
    Q, S, W = aut.bits.shape
    succ = [[set() for _ in range(S)] for _ in range(Q)]
    for q in range(Q):
        for a in range(S):
            for w in range(W):
                v = int(aut.bits[q, a, w])
                for b in range(32):
                    if v >> b & 1:
                        succ[q][a].add(32 * w + b)
    eps = [set() for _ in range(Q)]
    if getattr(aut, "eps", None) is not None:
        for q in range(Q):
            for w in range(W):
                v = int(aut.eps[q, w])
                for b in range(32):
                    if v >> b & 1:
                        eps[q].add(32 * w + b)
    return Q, S, succ, eps


def brute_force(aut, text: Sequence[int]) -> np.ndarray:
    """M(t, A) by definition: for every start i run the set simulation
    delta^({q0}, t[i..j]) (with epsilon closures) for every end j, and record
    each final state in the set. The dead state of the DFA form is an ordinary
    state here; it is non-final and absorbing, so it never adds a match.
    Quadratic in n: tiny inputs only."""
    Q, S, succ, eps = _succ_sets(aut)
    fin = {q for q in range(Q) if aut.final[q]}

    def close(states):
        st = list(states)
        seen = set(states)
        while st:
            p = st.pop()
            for t in eps[p]:
                if t not in seen:
                    seen.add(t)
                    st.append(t)
        return seen

    n = len(text)
    out = []
    for i in range(n):
        cur = close({aut.q0})
        for j in range(i, n):
            a = int(text[j])
            nxt = set()
            for q in cur:
                nxt |= succ[q][a]
            cur = close(nxt)
            for f in sorted(cur & fin):
                out.append((i, j, f))
            if not cur:
                break
    return sort_matches(np.array(out, dtype=np.uint32).reshape(-1, 3))


def brute_force_pair_steps(aut, text: Sequence[int], s_lo: int = 0,
                           s_hi: Optional[int] = None) -> int:
    """The work count by definition: for every start i in [s_lo, s_hi), the
    size of the instance's state set before each symbol t[j] ({q0} before
    t[i], then delta^({q0}, t[i..j-1])), summed over j = i .. n - 1 while the
    set is non-empty. The DFA form's dead state and missing transitions hold
    no instance. Epsilon-free machines; quadratic in n: tiny inputs only."""
    Q, S, succ, eps = _succ_sets(aut)
    if any(eps):
        raise ValueError("epsilon-free machines only")
    dead = getattr(aut, "dead", -1)
    n = len(text)
    s_hi = n if s_hi is None else s_hi
    total = 0
    for i in range(s_lo, s_hi):
        cur = {aut.q0}
        for j in range(i, n):
            total += len(cur)
            nxt = set()
            for q in cur:
                nxt |= succ[q][int(text[j])]
            cur = {q for q in nxt if 0 <= q < Q and q != dead}
            if not cur:
                break
    return total


def literal_occurrences(sigs: Iterable[bytes], final_of: dict, text: np.ndarray) -> np.ndarray:
    """All occurrences of every literal signature, by repeated ``bytes.find``:
    (i, i + len(s) - 1, final_of[s]) for each i with text[i:i+len(s)] == s."""
    tb = np.ascontiguousarray(text, dtype=np.uint8).tobytes()
    out = set()
    for s in set(sigs):
        f = final_of[s]
        k = tb.find(s)
        while k >= 0:
            out.add((k, k + len(s) - 1, f))
            k = tb.find(s, k + 1)
    return sort_matches(np.array(sorted(out), dtype=np.uint32).reshape(-1, 3))


def labelled(matches: np.ndarray, labels: dict):
    """Map (start, end, state) rows to sorted (label, start, end) tuples."""
    return sorted((labels[int(f)], int(i), int(j)) for i, j, f in matches)
