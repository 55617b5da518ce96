"""Epsilon edges followed at scan time (step 2 of Sec. III.B).

A machine loaded with pfsm_load_nfa_eps keeps its epsilon edges; the scan
closes every state set under them after each symbol. The match set equals
that of the epsilon-free machine (standard epsilon removal), which the
oracle scans: pinned on the paper's own union machine (Fig. 1, its worked
examples of Fig. 2 and Fig. 3) and on random machines with epsilon cycles,
epsilon edges into final states and out of q0.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from conftest import read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_1716_gb300 as P  # noqa: E402


@pytest.fixture(scope="module")
def pf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = P.Pfsm(0)
    yield p
    p.close()


def gpu_matches(pf, aut_id, text, cap=None):
    return oracle.sort_matches(pf.scan_numpy(aut_id, text, cap))


@pytest.mark.parametrize("fixture", ["fig2_aacacab.txt", "fig3_ac.txt"])
def test_paper_union_machine_with_its_epsilon_edges(pf, fixture):
    text, want = read_golden(fixture)
    m = W.fig1_union()            # ancillary state 0 with epsilon edges, not removed
    assert m.eps is not None
    a = pf.load(m)
    got = gpu_matches(pf, a, W.encode(text, W.FIG1_ALPHABET))
    assert oracle.labelled(got, m.labels) == want


def random_eps_nfa(seed, Q=16, S=4):
    rng = np.random.default_rng(seed)
    edges = [(q, x, t) for q in range(Q) for x in range(S) for t in range(Q)
             if (t > q or q == 0) and rng.random() < 0.18]
    eps = [(q, t) for q in range(Q) for t in range(q + 1, Q) if rng.random() < 0.06]
    eps += [(0, 5), (12, 14), (14, 12)]      # out of q0 (into a final), a cycle
    return W.nfa_from_edges(Q, S, 0, edges, [5, 9, 13], eps_edges=eps)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 1, 3])
def test_random_machines_with_epsilon_cycles(pf, seed, k):
    m = random_eps_nfa(seed)
    ref = W.eps_free(m)
    a = pf.load(m)
    if k:
        P.pfsm_set_params(pf.ctx, a, {"prefix_k": k, "tile": 4096, "halo": 16})
    for n in (0, 1, 2, 5, 17, 300, 4095, 4096, 4097, 9001):
        t = W.text_uniform(n, 4, 1000 * seed + n)
        assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(ref, t)), (seed, k, n)


def test_union_machine_loaded_as_it_is(pf):
    motifs = W.motif_set(91, n_motifs=24, len_lo=6, len_hi=10)
    parts = [W.motif_nfa(motifs)[0], W.dfa_as_nfa(W.dfa_random(92, Q=20, S=4))]
    S = 4
    edges, finals, eps = [], [], []
    q = 1
    for n in parts:
        for s in range(n.Q):
            for x in range(S):
                for t in W.nfa_succ(n, s, x):
                    edges.append((q + s, x, q + t))
        finals += [q + f for f in np.nonzero(n.final)[0]]
        eps.append((0, q + n.q0))
        q += n.Q
    u = W.nfa_from_edges(q, S, 0, edges, finals, eps_edges=eps)
    a = pf.load(u)
    t = W.text_dna(40_000, 93)
    W.plant_motifs(t, motifs, 400, 94)
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(W.eps_free(u), t))


def test_prefix_table_stays_on(pf):
    a = pf.load(random_eps_nfa(4))
    assert P.pfsm_get_params(pf.ctx, a)["prefix_k"] >= 1
    with pytest.raises(P.PfsmError):
        P.pfsm_set_params(pf.ctx, a, {"prefix_k": -1})


def test_epsilon_machine_in_a_batch(pf):
    ms = [random_eps_nfa(5), W.dfa_random(6, Q=20, S=4), random_eps_nfa(7)]
    ids = [pf.load(m) for m in ms]
    texts = [W.text_uniform(3000 + 1111 * i, 4, 50 + i) for i in range(6)]
    jobs = [(ids[i % 3], t) for i, t in enumerate(texts)]
    got, counts = pf.scan_batch(jobs)
    m = got.cpu().numpy().view(np.uint32)
    for j, (mi, t) in enumerate(zip([i % 3 for i in range(6)], texts)):
        ref = ms[mi] if isinstance(ms[mi], W.Dfa) else W.eps_free(ms[mi])
        want = oracle.scan(ref, t)
        assert int(counts[j]) == len(want), j
        assert np.array_equal(oracle.sort_matches(m[m[:, 0] == j][:, 1:]), want), j
