"""The CPU oracle pinned to things other than itself.

* the paper's worked examples (Fig. 2, Fig. 3 caption) as golden fixtures;
* the definition by exhaustive restarts (acalculia procedure, Sec. II) on
  every short text and on random longer ones;
* Python's ``re`` on every substring, for machines built from expressions;
* literal search (``bytes.find``) for signature tries;
* invariants: finals only, i <= j < n, one state per (i, j) for a DFA, the
  n(n+1)/2 |F| bound (Sec. III.C), independence from lazy and chained data
  partitioning (Sec. III.D.2), dead-state dropping, DFA vs NFA form.
"""
import itertools
import re

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import read_golden


def fig1():
    return W.eps_free(W.fig1_union())


# ---------------------------------------------------------------- worked examples
@pytest.mark.parametrize("fixture", ["fig2_aacacab.txt", "fig3_ac.txt"])
def test_paper_worked_examples(fixture):
    text, want = read_golden(fixture)
    m = fig1()
    got = oracle.labelled(oracle.scan(m, W.encode(text, W.FIG1_ALPHABET)), m.labels)
    assert got == want


@pytest.mark.parametrize("fixture", ["fig2_aacacab.txt", "fig3_ac.txt"])
def test_worked_examples_by_definition_on_epsilon_machine(fixture):
    """The definition run on the machine with its epsilon edges gives the
    same sets, which also pins the epsilon removal."""
    text, want = read_golden(fixture)
    m = W.fig1_union()
    got = oracle.labelled(oracle.brute_force(m, W.encode(text, W.FIG1_ALPHABET)), m.labels)
    assert got == want


def test_fig3_nothing_ends_at_zero():
    m = fig1()
    r = oracle.scan(m, W.encode("ac", W.FIG1_ALPHABET))
    assert (r[:, 1] == 1).all() and len(r) == 3


FIG1_RES = {"a*c": r"a*c", "ac": r"ac", "a(ca)*b": r"a(ca)*b"}


def test_fig1_machine_vs_re_on_random_texts():
    m = fig1()
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 40, 120):
        t = rng.integers(0, 3, size=n, dtype=np.uint8)
        s = "".join(W.FIG1_ALPHABET[x] for x in t)
        want = sorted((lab, i, j) for lab, rx in FIG1_RES.items()
                      for i in range(n) for j in range(i, n) if re.fullmatch(rx, s[i:j + 1]))
        assert oracle.labelled(oracle.scan(m, t), m.labels) == want


# ---------------------------------------------------------------- definition
def small_machines():
    out = []
    for seed in range(4):
        out.append(("dfa_dead%d" % seed, W.dfa_random(100 + seed, Q=9, S=4, p_dead=0.3)))
    for seed in range(2):
        d = W.dfa_random(200 + seed, Q=7, S=3, dead=-1, finals=[1, 2], p_dead=0.0)
        out.append(("dfa_nodead%d" % seed, d))
    rng = np.random.default_rng(7)
    for seed in range(4):
        Q, S = 8, 4
        edges = [(q, a, t) for q in range(Q) for a in range(S) for t in range(Q)
                 if rng.random() < 0.18]
        fins = [q for q in range(1, Q) if rng.random() < 0.35] or [Q - 1]
        out.append(("nfa%d" % seed, W.nfa_from_edges(Q, S, 0, edges, fins)))
    # q0 final and q0 reachable again: no empty matches, both tags kept
    out.append(("q0final", W.nfa_from_edges(3, 2, 0, [(0, 0, 0), (0, 1, 1), (1, 0, 2), (2, 1, 0)],
                                            [0, 2])))
    return out


@pytest.mark.parametrize("name,m", small_machines(), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_equals_definition_exhaustively(name, m):
    """Every text of length <= 5 (<= 6 for 2-3 symbols) over the alphabet."""
    S = m.S
    maxlen = 5 if S >= 4 else 6
    for n in range(0, maxlen + 1):
        for t in itertools.product(range(S), repeat=n):
            t = np.array(t, dtype=np.uint8)
            got = oracle.scan(m, t)
            want = oracle.brute_force(m, t)
            assert np.array_equal(got, want), (name, t.tolist())


@pytest.mark.parametrize("name,m", small_machines(), ids=lambda x: x if isinstance(x, str) else "")
def test_oracle_equals_definition_random(name, m):
    rng = np.random.default_rng(11)
    for n in (17, 64, 150):
        t = rng.integers(0, m.S, size=n, dtype=np.uint8)
        assert np.array_equal(oracle.scan(m, t), oracle.brute_force(m, t))


def test_epsilon_machine_definition_equals_oracle_after_removal():
    """Union machines with an ancillary epsilon state (Sec. III.A) over random
    sub-machines: definition on the epsilon form == oracle on removed form."""
    rng = np.random.default_rng(3)
    for trial in range(6):
        Q, S = 9, 3
        edges = [(q, a, t) for q in range(1, Q) for a in range(S) for t in range(1, Q)
                 if rng.random() < 0.15]
        eps = [(0, 1), (0, 4)] + [(q, t) for q in range(1, Q) for t in range(1, Q)
                                  if q != t and rng.random() < 0.05]
        fins = [q for q in range(1, Q) if rng.random() < 0.3] or [Q - 1]
        m = W.nfa_from_edges(Q, S, 0, edges, fins, eps_edges=eps)
        mf = W.eps_free(m)
        for n in (1, 3, 9, 40):
            t = rng.integers(0, S, size=n, dtype=np.uint8)
            assert np.array_equal(oracle.scan(mf, t), oracle.brute_force(m, t))


# ---------------------------------------------------------------- library routines
def test_motif_nfa_vs_re():
    motifs = W.motif_set(9, n_motifs=12, len_lo=3, len_hi=6, p_degenerate=0.4, p_gap=0.4)
    assert any(any(m.gaps) for m in motifs)
    nfa, finals = W.motif_nfa(motifs)
    rng = np.random.default_rng(4)
    t = W.text_dna(300, 17)
    W.plant_motifs(t, motifs, 25, 18)
    s = "".join(W.DNA[x] for x in t)
    rx = [re.compile(m.regex()) for m in motifs]
    want = []
    for k, r in enumerate(rx):
        for i in range(len(s)):
            for j in range(i, min(len(s), i + 40)):
                if r.fullmatch(s, i, j + 1):
                    want.append((i, j, finals[k]))
    want = oracle.sort_matches(np.array(sorted(set(want)), dtype=np.uint32))
    got = oracle.scan(nfa, t)
    assert len(got) > 20
    assert np.array_equal(got, want)


def test_trie_vs_literal_search_small_alphabet():
    rng = np.random.default_rng(8)
    sigs = sorted({bytes(rng.integers(0, 4, size=int(rng.integers(2, 6)), dtype=np.uint8))
                   for _ in range(40)})
    d, final_of = W.trie_dfa(sigs, S=4)
    t = W.text_uniform(3000, 4, 12)
    got = oracle.scan(d, t)
    want = oracle.literal_occurrences(sigs, final_of, t)
    assert len(got) > 100
    assert np.array_equal(got, want)


def test_trie_vs_literal_search_signature_shape():
    """Byte trie of the signature generator (nested and overlapping
    signatures, overlapping plants) against bytes.find, on 1 MiB."""
    sigs = W.signature_set(21)
    d, final_of = W.trie_dfa(sigs)
    t = W.text_uniform(1 << 20, 256, 22)
    plants = W.plant_signatures(t, sigs, 4096, 23)
    got = oracle.scan(d, t)
    want = oracle.literal_occurrences(sigs, final_of, t)
    assert np.array_equal(got, want)
    # every planted occurrence that is still intact is reported
    tb = t.tobytes()
    for pos, i in plants:
        s = sigs[i]
        if tb[pos:pos + len(s)] == s:
            row = (pos, pos + len(s) - 1, final_of[s])
            k = np.searchsorted(got[:, 0], pos)
            assert any(tuple(got[x]) == row for x in range(k, min(len(got), k + 64)))
    # nested signatures exist and produce nested matches
    assert len(got) > len(plants)


# ---------------------------------------------------------------- invariants
def test_invariants_random_dfa_full_size():
    d, t = W.workload_dna_dfa(0, n=1 << 18)
    m = oracle.scan(d, t)
    n = len(t)
    assert (m[:, 0] <= m[:, 1]).all() and (m[:, 1] < n).all()
    assert d.final[m[:, 2]].all()
    # DFA: at most one state per (start, end)
    key = m[:, 0].astype(np.uint64) << np.uint64(32) | m[:, 1].astype(np.uint64)
    assert len(np.unique(key)) == len(key)
    nF = int(d.final.sum())
    assert len(m) <= n * (n + 1) // 2 * nF


def test_matches_reach_final_by_delta():
    """Each reported (i, j, f) of a DFA: walking delta from q0 over t[i..j]
    ends in f without passing the dead state (sampled)."""
    d, t = W.workload_dna_dfa(1, n=1 << 16)
    m = oracle.scan(d, t)
    for i, j, f in m[:: max(1, len(m) // 500)]:
        q = d.q0
        for x in t[i:j + 1]:
            q = int(d.delta[q, x])
            assert q != d.dead
        assert q == f


@pytest.mark.parametrize("kind", ["dfa", "nfa"])
def test_lazy_partitioning_independence(kind):
    if kind == "dfa":
        a, t = W.workload_dna_dfa(2, n=20000)
    else:
        a, t, _, _ = W.workload_motif_nfa(2, n=20000, n_motifs=40, every=500)
    full = oracle.scan(a, t)
    n = len(t)
    for k in (1, 777, 4096, 10001, n - 1):
        parts = np.concatenate([oracle.scan(a, t, 0, k), oracle.scan(a, t, k, n)])
        assert np.array_equal(oracle.sort_matches(parts), full)
    cuts = [0, 1000, 1003, 5000, 12000, n]
    parts = np.concatenate([oracle.scan(a, t, lo, hi) for lo, hi in zip(cuts, cuts[1:])])
    assert np.array_equal(oracle.sort_matches(parts), full)


@pytest.mark.parametrize("kind", ["dfa", "nfa", "nodead"])
def test_chained_partitioning_independence(kind):
    """Sec. III.D.2 chained form: each segment finds the matches inside it and
    passes its tagged active states on; the receiver continues them without
    reinitialising, cycle after cycle, until nothing is passed on."""
    if kind == "dfa":
        a, t = W.workload_dna_dfa(3, n=6000)
    elif kind == "nfa":
        a, t, _, _ = W.workload_motif_nfa(3, n=6000, n_motifs=40, every=300)
    else:
        a = W.dfa_random(5, Q=6, S=4, dead=-1, finals=[1, 2], p_dead=0.0)
        t = W.text_uniform(300, 4, 6)
    full = oracle.scan(a, t)
    n = len(t)
    cuts = [0, n // 5, n // 5 + 1, n // 2, 3 * n // 4, n]
    segs = list(zip(cuts, cuts[1:]))
    got = []
    carry = [None] * len(segs)
    for s, (lo, hi) in enumerate(segs):
        m, act = oracle.run_segment(a, t, lo, hi, lo, hi)
        got.append(m)
        if s + 1 < len(segs):
            carry[s + 1] = act
    # cycles: pass survivors forward until none are left
    for s in range(1, len(segs)):
        pairs = carry[s]
        for s2 in range(s, len(segs)):
            if pairs is None or len(pairs) == 0:
                break
            lo, hi = segs[s2]
            m, pairs = oracle.run_segment(a, t, lo, hi, lo, lo, pairs)
            got.append(m)
    assert np.array_equal(oracle.sort_matches(np.concatenate(got)), full)


def test_dead_state_drop_does_not_change_result():
    d = W.dfa_random(31, Q=12, S=4, p_dead=0.3)
    t = W.text_uniform(500, 4, 32)
    keep = W.Dfa(delta=d.delta, q0=d.q0, dead=-1, final=d.final)
    assert np.array_equal(oracle.scan(d, t), oracle.scan(keep, t))


def test_dfa_and_nfa_forms_agree():
    d, t = W.workload_dna_dfa(4, n=30000)
    assert np.array_equal(oracle.scan(d, t), oracle.scan(W.dfa_as_nfa(d), t))


def test_reinitialisation_keeps_existing_tags():
    """q0 is re-entered by a transition while a new instance starts there
    (reading A6): both instances live on."""
    # q0 -a-> q0 and q0 -b-> 1 (final); on "aab": starts 0, 1, 2 all end at 2
    m = W.nfa_from_edges(2, 2, 0, [(0, 0, 0), (0, 1, 1)], [1])
    r = oracle.scan(m, np.array([0, 0, 1], dtype=np.uint8))
    assert r.tolist() == [[0, 2, 1], [1, 2, 1], [2, 2, 1]]


def test_nfa_two_paths_one_match():
    """One start reaching one final state along two paths is one match (tags
    form a set, Sec. III.B)."""
    m = W.nfa_from_edges(4, 1, 0, [(0, 0, 1), (0, 0, 2), (1, 0, 3), (2, 0, 3)], [3])
    r = oracle.scan(m, np.zeros(2, dtype=np.uint8))
    assert r.tolist() == [[0, 1, 3]]


def test_empty_and_invalid_inputs():
    d = W.dfa_random(1, Q=8, S=4)
    assert oracle.scan(d, np.zeros(0, dtype=np.uint8)).shape == (0, 3)
    with pytest.raises(ValueError):
        oracle.scan(d, np.array([0, 7], dtype=np.uint8))


# ---------------------------------------------------------------- work (pair-steps)
def test_pair_steps_closed_forms():
    """Closed forms of the number of (start, state) pairs advanced over a
    symbol (Sec. III.B): a complete DFA keeps every start alive, so position
    j advances j + 1 pairs (n(n+1)/2 in all); a DFA whose every move enters
    the dead state advances only the new start (n); an NFA with
    q0 -> {q0, q1}, q1 -> {q1} on every symbol holds two states per older
    start (1 + 2j at position j, n^2 in all)."""
    for n in (0, 1, 7, 300):
        t = W.text_uniform(n, 3, n + 1)
        full = W.dfa_random(5, Q=7, S=3, dead=-1, finals=[1, 2], p_dead=0.0)
        assert oracle.pair_steps(full, t)[0] == n * (n + 1) // 2
        delta = np.full((4, 3), 3, dtype=np.int16)
        alldead = W.Dfa(delta=delta, q0=0, dead=3, final=np.array([0, 1, 0, 0], np.uint8))
        assert oracle.pair_steps(alldead, t) == (n, 0)
        two = W.nfa_from_edges(2, 3, 0, [(0, a, 0) for a in range(3)] + [(0, a, 1) for a in range(3)]
                               + [(1, a, 1) for a in range(3)], [1])
        # every start i reaches the final q1 at every end j >= i
        assert oracle.pair_steps(two, t) == (n * n, n * (n + 1) // 2)


@pytest.mark.parametrize("name,m", small_machines(), ids=lambda x: x if isinstance(x, str) else "")
def test_pair_steps_equal_definition(name, m):
    """The tagged-state procedure's count equals the count by definition
    (per start, the size of its set before every symbol), on every short
    text and on random longer ones, for whole texts and start windows."""
    maxlen = 4 if m.S >= 4 else 5
    for n in range(0, maxlen + 1):
        for t in itertools.product(range(m.S), repeat=n):
            t = np.array(t, dtype=np.uint8)
            assert oracle.pair_steps(m, t)[0] == oracle.brute_force_pair_steps(m, t), t.tolist()
    rng = np.random.default_rng(13)
    for n in (40, 150):
        t = rng.integers(0, m.S, size=n, dtype=np.uint8)
        w, cnt = oracle.pair_steps(m, t)
        assert w == oracle.brute_force_pair_steps(m, t)
        assert cnt == len(oracle.brute_force(m, t))
        lo, hi = 13, 101
        assert oracle.pair_steps(m, t, lo, hi)[0] == oracle.brute_force_pair_steps(m, t, lo, hi)


def test_pair_steps_additive_over_start_windows():
    """Lazy data partitioning (Sec. III.D.2) splits the work exactly: the
    windows' counts add up to the whole text's."""
    nfa, text, _, _ = W.workload_motif_nfa(3, n=1 << 14, n_motifs=24)
    whole = oracle.pair_steps(nfa, text)
    cuts = [0, 1, 999, 5000, 5001, 1 << 14]
    parts = [oracle.pair_steps(nfa, text, cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1)]
    assert whole == (sum(p[0] for p in parts), sum(p[1] for p in parts))
    assert whole[1] == len(oracle.scan(nfa, text))
