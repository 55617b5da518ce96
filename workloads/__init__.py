"""Seeded synthetic inputs for the PFSM scan: automata tables and texts.

This module builds inputs only. It holds none of the scan's arithmetic (no
tagged-state stepping, no match reporting); both the CPU oracle and the CUDA
path consume what it returns. Everything is drawn from numpy's PCG64
``Generator`` seeded explicitly, so the same seed gives the same bytes on x86
and Arm.

Automaton model (Sec. III.A): a PFSM is (Sigma, Q, q0, delta, F, L, l) with an
NFA-like delta: Q x Sigma -> P(Q). Symbols are the integers 0..S-1, states
0..Q-1. Two table forms are produced:

* ``Dfa``: ``delta`` int16 [Q][S] (one successor per entry), an optional
  absorbing non-final ``dead`` state (-1 = none), ``final`` uint8 [Q].
* ``Nfa``: ``bits`` uint32 [Q][S][W], W = ceil(Q/32): bit (q' % 32) of word
  q' // 32 of row (q, a) is set iff q' is in delta(q, a). An optional ``eps``
  uint32 [Q][W] holds epsilon edges (only the Sec. III.A union construction
  uses them; ``eps_free`` removes them before a scan).

Workload shapes (one generator per shape):

* ``dfa_random``: random DNA DFA, 64 states, dead state 63, finals 1..8.
* ``motif_set`` + ``motif_nfa``: position NFA of DNA motifs with degenerate
  positions and bounded any-symbol gaps; ``plant_motifs`` writes instances.
* ``signature_set`` + ``trie_dfa``: byte trie of literal signatures with a
  dead state and no failure links; ``plant_signatures`` writes occurrences,
  overlapping and nested ones included.
* ``batch_workload`` and ``serve_workload``: the many-texts and the
  request-stream mixes built from the generators above.
"""
from __future__ import annotations

import dataclasses
import functools
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

DNA = "ACGT"  # symbol k <-> DNA[k]


# ----------------------------------------------------------------------------
# Table containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Dfa:
    delta: np.ndarray          # int16 [Q][S]
    q0: int
    dead: int                  # -1 = no dead state
    final: np.ndarray          # uint8 [Q]
    labels: Optional[dict] = None   # final state -> label (host-side l: F -> L)

    @property
    def Q(self) -> int:
        return int(self.delta.shape[0])

    @property
    def S(self) -> int:
        return int(self.delta.shape[1])

    kind = "dfa"


@dataclasses.dataclass
class Nfa:
    bits: np.ndarray           # uint32 [Q][S][W]
    q0: int
    final: np.ndarray          # uint8 [Q]
    eps: Optional[np.ndarray] = None   # uint32 [Q][W] or None
    labels: Optional[dict] = None

    @property
    def Q(self) -> int:
        return int(self.bits.shape[0])

    @property
    def S(self) -> int:
        return int(self.bits.shape[1])

    kind = "nfa"


def words(Q: int) -> int:
    return (Q + 31) // 32


def nfa_from_edges(Q: int, S: int, q0: int, edges, finals, eps_edges=(),
                   labels=None) -> Nfa:
    """Build an ``Nfa`` from (q, a, q') edge triples."""
    W = words(Q)
    bits = np.zeros((Q, S, W), dtype=np.uint32)
    for q, a, t in edges:
        bits[q, a, t >> 5] |= np.uint32(1 << (t & 31))
    eps = None
    if eps_edges:
        eps = np.zeros((Q, W), dtype=np.uint32)
        for q, t in eps_edges:
            eps[q, t >> 5] |= np.uint32(1 << (t & 31))
    fin = np.zeros(Q, dtype=np.uint8)
    for f in finals:
        fin[f] = 1
    return Nfa(bits=bits, q0=q0, final=fin, eps=eps, labels=labels)


def live_core_nfa(K: int, seed: int, p: float = 0.3) -> Nfa:
    """An NFA whose instances that start with symbol 0 never die: q0 --0-->
    a core of K states (1..K) in which every state has a successor on every
    symbol, plus random extra edges with probability p (the live set fills
    most of the core); core state 1 --1--> G --2--> F, the only final state,
    which has no successors. Over uniform DNA each live instance reports at
    about one position in 16: some n^2 / 128 matches for a text of n
    symbols, nearly all from instances that run far past their start."""
    rng = np.random.default_rng(seed)
    S = 4
    G, F = K + 1, K + 2
    edges = [(0, 0, 1)]
    for q in range(1, K + 1):
        for x in range(S):
            ts = {int(rng.integers(1, K + 1))} | {t for t in range(1, K + 1) if rng.random() < p}
            edges += [(q, x, t) for t in ts]
    edges += [(1, 1, G), (G, 2, F)]
    return nfa_from_edges(K + 3, S, 0, edges, [F])


def dfa_as_nfa(d: Dfa) -> Nfa:
    """The same machine with delta returning singletons (dead edges dropped)."""
    edges = []
    for q in range(d.Q):
        if q == d.dead:
            continue
        for a in range(d.S):
            t = int(d.delta[q, a])
            if t != d.dead:
                edges.append((q, a, t))
    fin = [q for q in range(d.Q) if d.final[q]]
    return nfa_from_edges(d.Q, d.S, d.q0, edges, fin, labels=d.labels)


def nfa_succ(n: Nfa, q: int, a: int) -> List[int]:
    row = n.bits[q, a]
    out = []
    for w in np.nonzero(row)[0]:
        v = int(row[w])
        while v:
            b = (v & -v).bit_length() - 1
            out.append(int(w) * 32 + b)
            v &= v - 1
    return out


def eps_free(n: Nfa) -> Nfa:
    """Standard epsilon removal: delta'(q,a) = E(U_{p in E(q)} delta(p,a)).

    E is the epsilon closure. Targets are closed, so a final state reached
    through epsilon edges after a consumed symbol is a member of the target set
    itself and F' = F. Zero-length matches do not exist in this form.
    """
    if n.eps is None:
        return n
    Q, S, W = n.bits.shape

    def eps_succ(q):
        row = n.eps[q]
        out = []
        for w in np.nonzero(row)[0]:
            v = int(row[w])
            while v:
                b = (v & -v).bit_length() - 1
                out.append(int(w) * 32 + b)
                v &= v - 1
        return out

    closure = []
    for q in range(Q):
        seen = {q}
        stack = [q]
        while stack:
            p = stack.pop()
            for t in eps_succ(p):
                if t not in seen:
                    seen.add(t)
                    stack.append(t)
        closure.append(sorted(seen))
    edges = []
    for q in range(Q):
        for a in range(S):
            tgt = set()
            for p in closure[q]:
                for t in nfa_succ(n, p, a):
                    tgt.update(closure[t])
            edges.extend((q, a, t) for t in tgt)
    fin = [q for q in range(Q) if n.final[q]]
    return nfa_from_edges(Q, S, n.q0, edges, fin, labels=n.labels)


# ----------------------------------------------------------------------------
# Sec. III.A worked example: union of "a*c", "ac", "a(ca)*b"
# ----------------------------------------------------------------------------
FIG1_ALPHABET = "abc"   # a=0, b=1, c=2


def fig1_union() -> Nfa:
    """The Sec. III.A example machine, rebuilt from its three expressions.

    The figure itself is missing, so the machine is reconstructed as the text
    describes it: one DFA per expression and an ancillary initial state with
    epsilon edges to each DFA's initial state; final states carry the label of
    their expression.

      state 0       ancillary initial state
      states 1-2    a*c      : 1 -a-> 1, 1 -c-> 2 (final)
      states 3-5    ac       : 3 -a-> 4 -c-> 5 (final)
      states 6-9    a(ca)*b  : 6 -a-> 7, 7 -c-> 8, 8 -a-> 7, 7 -b-> 9 (final)
    """
    a, b, c = 0, 1, 2
    edges = [(1, a, 1), (1, c, 2),
             (3, a, 4), (4, c, 5),
             (6, a, 7), (7, c, 8), (8, a, 7), (7, b, 9)]
    labels = {2: "a*c", 5: "ac", 9: "a(ca)*b"}
    return nfa_from_edges(10, 3, 0, edges, [2, 5, 9],
                          eps_edges=[(0, 1), (0, 3), (0, 6)], labels=labels)


def encode(s: str, alphabet: str) -> np.ndarray:
    return np.frombuffer(bytes(alphabet.index(ch) for ch in s), dtype=np.uint8).copy()


# ----------------------------------------------------------------------------
# Random DFA (DNA alphabet, dead state)
# ----------------------------------------------------------------------------
def dfa_random(seed: int, Q: int = 64, S: int = 4, dead: Optional[int] = None,
               finals: Optional[Sequence[int]] = None, p_dead: float = 0.3) -> Dfa:
    """Random DFA: every (q, a) with q != dead goes to ``dead`` with
    probability ``p_dead``, else to a state uniform over the non-dead states.
    The dead state is absorbing and non-final. Defaults: 64 states, dead 63,
    q0 0, finals 1..8 (for other sizes: finals 1..max(1, (Q-1)//8))."""
    rng = np.random.default_rng(seed)
    if dead is None:
        dead = Q - 1
    live = Q - 1 if dead >= 0 else Q
    if finals is None:
        finals = range(1, 1 + max(1, (Q - 1) // 8)) if Q != 64 else range(1, 9)
    to_dead = rng.random((Q, S)) < p_dead
    tgt = rng.integers(0, live, size=(Q, S))
    if dead >= 0:
        # live ids are 0..Q-1 without `dead`
        tgt = np.where(tgt >= dead, tgt + 1, tgt)
        tgt = np.where(to_dead, dead, tgt)
        tgt[dead, :] = dead
    delta = tgt.astype(np.int16)
    fin = np.zeros(Q, dtype=np.uint8)
    fin[list(finals)] = 1
    if dead >= 0:
        fin[dead] = 0
    return Dfa(delta=delta, q0=0, dead=dead, final=fin)


# ----------------------------------------------------------------------------
# Texts
# ----------------------------------------------------------------------------
def text_uniform(n: int, S: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, S, size=n, dtype=np.uint8)


_GC40 = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 3], dtype=np.uint8)


def text_dna(n: int, seed: int, gc: float = 0.4) -> np.ndarray:
    """i.i.d. DNA symbols; gc=0.4 gives P(A)=P(T)=0.3, P(C)=P(G)=0.2."""
    rng = np.random.default_rng(seed)
    if abs(gc - 0.4) < 1e-12:
        return _GC40[rng.integers(0, 10, size=n, dtype=np.uint8)]
    p = np.array([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
    return rng.choice(4, size=n, p=p).astype(np.uint8)


# ----------------------------------------------------------------------------
# Position NFA from DNA motifs
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Motif:
    classes: List[int]      # 4-bit masks over {A,C,G,T}, one per position
    gaps: List[bool]        # gaps[k]: a bounded gap x(0,3) between positions k and k+1

    def regex(self) -> str:
        out = []
        for k, m in enumerate(self.classes):
            bases = [DNA[b] for b in range(4) if m >> b & 1]
            out.append(bases[0] if len(bases) == 1 else "[" + "".join(bases) + "]")
            if k < len(self.gaps) and self.gaps[k]:
                out.append(".{0,3}")
        return "".join(out)


def motif_set(seed: int, n_motifs: int = 256, len_lo: int = 12, len_hi: int = 24,
              p_degenerate: float = 0.15, p_gap: float = 0.05) -> List[Motif]:
    """Motifs of U[len_lo, len_hi] positions. A position is degenerate with
    probability p_degenerate (a class of 2-4 distinct bases), else one base
    uniform over ACGT. Each of the L-1 boundaries carries a bounded gap of
    0-3 any-symbol steps with probability p_gap."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_motifs):
        L = int(rng.integers(len_lo, len_hi + 1))
        classes = []
        for _k in range(L):
            if rng.random() < p_degenerate:
                size = int(rng.integers(2, 5))
                bases = rng.choice(4, size=size, replace=False)
                classes.append(int(sum(1 << int(b) for b in bases)))
            else:
                classes.append(1 << int(rng.integers(0, 4)))
        gaps = [bool(rng.random() < p_gap) for _ in range(L - 1)]
        out.append(Motif(classes, gaps))
    return out


def motif_nfa(motifs: Sequence[Motif]) -> Tuple[Nfa, List[int]]:
    """Position NFA without determinisation (Sec. II, NFA form).

    State 0 is q0. Motif position k gets a state entered by consuming a symbol
    of class k. A gap x(0,3) after position k adds states g1, g2, g3, each
    entered by any symbol: P_k -> g1 -> g2 -> g3 along any symbol, and each of
    P_k, g1, g2, g3 also reaches P_{k+1} on class k+1 (gap length 0..3). The
    last position of each motif is its single final state and has no outgoing
    edges. Returns the machine and the final state of each motif.
    """
    edges = []
    finals = []
    nxt = 1
    for m in motifs:
        L = len(m.classes)
        pos = []
        gap_states = {}
        for k in range(L):
            pos.append(nxt)
            nxt += 1
            if k < L - 1 and m.gaps[k]:
                gap_states[k] = [nxt, nxt + 1, nxt + 2]
                nxt += 3
        # q0 -> first position
        for a in range(4):
            if m.classes[0] >> a & 1:
                edges.append((0, a, pos[0]))
        for k in range(L - 1):
            cls = m.classes[k + 1]
            srcs = [pos[k]] + gap_states.get(k, [])
            for s in srcs:
                for a in range(4):
                    if cls >> a & 1:
                        edges.append((s, a, pos[k + 1]))
            if k in gap_states:
                g = gap_states[k]
                chain = [pos[k]] + g
                for i in range(3):
                    for a in range(4):
                        edges.append((chain[i], a, chain[i + 1]))
        finals.append(pos[-1])
    Q = nxt
    labels = {f: i for i, f in enumerate(finals)}
    return nfa_from_edges(Q, 4, 0, edges, finals, labels=labels), finals


def motif_instance(m: Motif, rng: np.random.Generator) -> np.ndarray:
    out = []
    for k, cls in enumerate(m.classes):
        bases = [b for b in range(4) if cls >> b & 1]
        out.append(bases[int(rng.integers(0, len(bases)))])
        if k < len(m.gaps) and m.gaps[k]:
            g = int(rng.integers(0, 4))
            out.extend(int(x) for x in rng.integers(0, 4, size=g))
    return np.array(out, dtype=np.uint8)


def plant_motifs(text: np.ndarray, motifs: Sequence[Motif], every: int, seed: int):
    """Write one random instance of a random motif roughly every ``every``
    symbols (uniform jitter of +-every/4). Returns [(pos, motif, length)]."""
    rng = np.random.default_rng(seed)
    n = len(text)
    plants = []
    pos = int(rng.integers(0, max(1, every)))
    while True:
        mi = int(rng.integers(0, len(motifs)))
        inst = motif_instance(motifs[mi], rng)
        if pos + len(inst) > n:
            break
        text[pos:pos + len(inst)] = inst
        plants.append((pos, mi, len(inst)))
        pos += every + int(rng.integers(-(every // 4), every // 4 + 1))
    return plants


# ----------------------------------------------------------------------------
# Byte trie of literal signatures
# ----------------------------------------------------------------------------
def signature_set(seed: int, n_sigs: int = 1000, len_lo: int = 8, len_hi: int = 32,
                  S: int = 256, frac_nested: float = 0.03,
                  frac_overlap: float = 0.03) -> List[bytes]:
    """Random literal signatures of U[len_lo, len_hi] symbols. A fraction are
    built to nest (a slice of an earlier signature, so planting the outer one
    plants the inner) and a fraction to overlap (they begin with a suffix of
    an earlier signature, so the two can be planted overlapping)."""
    rng = np.random.default_rng(seed)
    sigs: List[bytes] = []
    for i in range(n_sigs):
        r = rng.random()
        L = int(rng.integers(len_lo, len_hi + 1))
        if i >= 8 and r < frac_nested:
            src = sigs[int(rng.integers(0, len(sigs)))]
            if len(src) > len_lo:
                ln = int(rng.integers(len_lo, len(src)))
                off = int(rng.integers(0, len(src) - ln + 1))
                sigs.append(src[off:off + ln])
                continue
        if i >= 8 and r < frac_nested + frac_overlap:
            src = sigs[int(rng.integers(0, len(sigs)))]
            ov = int(rng.integers(1, min(len(src), L)))
            tail = rng.integers(0, S, size=L - ov, dtype=np.uint8).tobytes()
            sigs.append(src[len(src) - ov:] + tail)
            continue
        sigs.append(rng.integers(0, S, size=L, dtype=np.uint8).tobytes())
    return sigs


def trie_dfa(sigs: Sequence[bytes], S: int = 256) -> Tuple[Dfa, dict]:
    """Trie DFA with a dead state and no failure links. Node ids follow
    insertion order (root = 0); the dead state is the last id. Duplicate
    signatures share one final state; a signature that is a prefix of another
    makes an internal node final. Returns the DFA and {signature: final}."""
    children = [dict()]
    final_of = {}
    for s in sigs:
        node = 0
        for ch in s:
            nxt = children[node].get(ch)
            if nxt is None:
                nxt = len(children)
                children[node][ch] = nxt
                children.append(dict())
            node = nxt
        final_of[s] = node
    Q = len(children) + 1
    dead = Q - 1
    if Q > 32767:
        raise ValueError("trie too large for int16 state ids")
    delta = np.full((Q, S), dead, dtype=np.int16)
    for q, ch in enumerate(children):
        for a, t in ch.items():
            delta[q, a] = t
    fin = np.zeros(Q, dtype=np.uint8)
    for f in final_of.values():
        fin[f] = 1
    labels = {}
    for s, f in final_of.items():
        labels.setdefault(f, s)
    return Dfa(delta=delta, q0=0, dead=dead, final=fin, labels=labels), final_of


@functools.lru_cache(maxsize=64)
def _prefix_index(sigs: Tuple[bytes, ...]) -> dict:
    """Which signatures begin with a given proper prefix (used to plant
    overlapping pairs)."""
    by_prefix = {}
    for j, s in enumerate(sigs):
        for ln in range(1, len(s)):
            by_prefix.setdefault(s[:ln], []).append(j)
    return by_prefix


def plant_signatures(text: np.ndarray, sigs: Sequence[bytes], every: int, seed: int):
    """Plant one signature per ``every`` bytes at a random offset inside each
    block. One block in eight plants an overlapping pair: a second signature
    written so that it starts inside the first (when one of the set begins
    with a suffix of the first, that one is chosen, so both stay intact).
    Returns [(pos, signature index)] of everything written."""
    rng = np.random.default_rng(seed)
    n = len(text)
    by_prefix = _prefix_index(tuple(sigs))
    plants = []
    for blk in range(0, n, every):
        i = int(rng.integers(0, len(sigs)))
        s = sigs[i]
        room = min(every, n - blk) - 2 * 32
        if room <= 0:
            continue
        pos = blk + int(rng.integers(0, room))
        text[pos:pos + len(s)] = np.frombuffer(s, dtype=np.uint8)
        plants.append((pos, i))
        if rng.random() < 0.125:
            cands = []
            for ov in range(len(s) - 1, 0, -1):
                cands = by_prefix.get(s[len(s) - ov:], [])
                if cands:
                    break
            if cands:
                j = cands[int(rng.integers(0, len(cands)))]
                p2 = pos + len(s) - ov
            else:
                j = int(rng.integers(0, len(sigs)))
                p2 = pos + int(rng.integers(1, len(s)))
            s2 = sigs[j]
            if p2 + len(s2) <= n:
                text[p2:p2 + len(s2)] = np.frombuffer(s2, dtype=np.uint8)
                plants.append((p2, j))
    return plants


# ----------------------------------------------------------------------------
# Named workloads (sizes of the five scan configurations)
# ----------------------------------------------------------------------------
def workload_dna_dfa(seed: int = 0, n: int = 1 << 20):
    """Random 64-state DNA DFA, text of n uniform symbols (default 1 MiB)."""
    d = dfa_random(seed)
    t = text_uniform(n, 4, seed + 1000)
    return d, t


def workload_motif_nfa(seed: int = 0, n: int = 64 << 20, n_motifs: int = 256,
                       every: int = 10_000):
    """Position NFA of 256 DNA motifs (~5.3k states); GC=0.4 text of n
    symbols (default 64 MiB) with a motif instance planted every ~10 kB."""
    motifs = motif_set(seed, n_motifs=n_motifs)
    nfa, finals = motif_nfa(motifs)
    t = text_dna(n, seed + 1000)
    plants = plant_motifs(t, motifs, every, seed + 2000)
    return nfa, t, motifs, plants


def workload_byte_trie(seed: int = 0, n: int = 1 << 30, n_sigs: int = 1000,
                       every: int = 1 << 16):
    """Trie DFA of 1000 byte signatures; n uniform random bytes (default
    1 GiB) with one signature planted per 64 KiB, overlaps and nests included."""
    sigs = signature_set(seed, n_sigs=n_sigs)
    dfa, final_of = trie_dfa(sigs)
    t = text_uniform(n, 256, seed + 1000)
    plants = plant_signatures(t, sigs, every, seed + 2000)
    return dfa, t, sigs, final_of, plants


def loguniform_lengths(rng, k: int, lo: int, hi: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=k)).astype(np.int64)


@dataclasses.dataclass
class BatchWorkload:
    automata: list            # Dfa | Nfa
    alphabet: List[int]       # S per automaton
    job_aut: np.ndarray       # int32 [k] automaton index of each text
    offsets: np.ndarray       # int64 [k+1] text i = data[offsets[i]:offsets[i+1]]
    data: np.ndarray          # uint8 concatenated texts


def batch_workload(seed: int = 0, n_texts: int = 10_000, lo: int = 100,
                   hi: int = 1 << 20, n_nfa: int = 8, n_trie: int = 8,
                   nfa_motifs: int = 256, trie_sigs: int = 1000) -> BatchWorkload:
    """Many texts of log-uniform length in [lo, hi] paired uniformly with one
    of n_nfa motif NFAs and n_trie byte tries (new seeds). Each text is drawn
    in its automaton's alphabet: GC=0.4 DNA for NFAs, uniform bytes for tries,
    with the automaton's patterns planted at the usual densities."""
    rng = np.random.default_rng(seed)
    automata, alph, pats = [], [], []
    for i in range(n_nfa):
        motifs = motif_set(seed * 1000 + 100 + i, n_motifs=nfa_motifs)
        automata.append(motif_nfa(motifs)[0])
        alph.append(4)
        pats.append(("motif", motifs))
    for i in range(n_trie):
        sigs = signature_set(seed * 1000 + 200 + i, n_sigs=trie_sigs)
        automata.append(trie_dfa(sigs)[0])
        alph.append(256)
        pats.append(("sig", sigs))
    lengths = loguniform_lengths(rng, n_texts, lo, hi)
    job_aut = rng.integers(0, len(automata), size=n_texts).astype(np.int32)
    offsets = np.zeros(n_texts + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    data = np.empty(int(offsets[-1]), dtype=np.uint8)
    for i in range(n_texts):
        a = int(job_aut[i])
        n = int(lengths[i])
        sub_seed = seed * 1_000_003 + i
        if alph[a] == 4:
            t = text_dna(n, sub_seed)
            plant_motifs(t, pats[a][1], 10_000, sub_seed + 7)
        else:
            t = text_uniform(n, 256, sub_seed)
            plant_signatures(t, pats[a][1], 1 << 16, sub_seed + 7)
        data[offsets[i]:offsets[i + 1]] = t
    return BatchWorkload(automata, alph, job_aut, offsets, data)


@dataclasses.dataclass
class ServeWorkload:
    automata: list
    alphabet: List[int]
    arrivals: np.ndarray      # float64 [k] seconds since start
    req_aut: np.ndarray       # int32 [k]
    lengths: np.ndarray       # int64 [k]
    text_seeds: np.ndarray    # int64 [k]


def serve_automaton(seed: int, kind: int, size: int):
    """One automaton of about ``size`` states from the DFA (kind 0), motif NFA
    (kind 1) or byte trie (kind 2) generator."""
    if kind == 0:
        return dfa_random(seed, Q=max(8, size), p_dead=0.3), 4
    if kind == 1:
        n_motifs = max(1, size // 19)
        return motif_nfa(motif_set(seed, n_motifs=n_motifs))[0], 4
    n_sigs = max(1, size // 20)
    return trie_dfa(signature_set(seed, n_sigs=n_sigs))[0], 256


def serve_workload(seed: int = 0, n_req: int = 100_000, rate_hz: float = 1000.0,
                   n_aut: int = 64, size_lo: int = 64, size_hi: int = 16384,
                   zipf_s: float = 1.1, median_len: int = 4096, sigma: float = 1.5,
                   max_len: int = 4 << 20) -> ServeWorkload:
    """Poisson arrivals at ``rate_hz``; text length lognormal (median 4 KiB,
    sigma 1.5, truncated at 4 MiB); automaton Zipf(1.1) over 64 automata of
    log-uniform size 64-16,384 states from the three generators."""
    rng = np.random.default_rng(seed)
    sizes = loguniform_lengths(rng, n_aut, size_lo, size_hi)
    kinds = rng.integers(0, 3, size=n_aut)
    automata, alph = [], []
    for i in range(n_aut):
        a, s = serve_automaton(seed * 7919 + i, int(kinds[i]), int(sizes[i]))
        automata.append(a)
        alph.append(s)
    gaps = rng.exponential(1.0 / rate_hz, size=n_req)
    arrivals = np.cumsum(gaps)
    ranks = np.arange(1, n_aut + 1, dtype=np.float64)
    pz = ranks ** (-zipf_s)
    pz /= pz.sum()
    req_aut = rng.choice(n_aut, size=n_req, p=pz).astype(np.int32)
    lengths = np.minimum(np.exp(rng.normal(math.log(median_len), sigma, size=n_req)),
                         max_len).astype(np.int64)
    lengths = np.maximum(lengths, 1)
    text_seeds = rng.integers(0, 2**62, size=n_req, dtype=np.int64)
    return ServeWorkload(automata, alph, arrivals, req_aut, lengths, text_seeds)


def serve_text(w: ServeWorkload, i: int) -> np.ndarray:
    S = w.alphabet[int(w.req_aut[i])]
    n = int(w.lengths[i])
    if S == 4:
        return text_dna(n, int(w.text_seeds[i]))
    return text_uniform(n, 256, int(w.text_seeds[i]))
