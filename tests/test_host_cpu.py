"""Host-side logic that needs no GPU: generators, tuner bookkeeping."""
import json
import os

import numpy as np

import workloads as W


def test_generators_are_deterministic():
    a = W.workload_motif_nfa(3, n=5000, n_motifs=20, every=300)
    b = W.workload_motif_nfa(3, n=5000, n_motifs=20, every=300)
    assert np.array_equal(a[0].bits, b[0].bits) and np.array_equal(a[1], b[1])
    d1, t1 = W.workload_dna_dfa(2, n=1000)
    d2, t2 = W.workload_dna_dfa(2, n=1000)
    assert np.array_equal(d1.delta, d2.delta) and np.array_equal(t1, t2)
    s1 = W.signature_set(5, n_sigs=50)
    assert s1 == W.signature_set(5, n_sigs=50)


def test_generator_shapes_match_the_workload_definitions():
    d = W.dfa_random(0)
    assert d.Q == 64 and d.dead == 63 and (d.delta[63] == 63).all()
    assert list(np.nonzero(d.final)[0]) == list(range(1, 9))
    live_targets = d.delta[:63][d.delta[:63] != 63]
    assert live_targets.max() <= 62
    nfa, finals = W.motif_nfa(W.motif_set(0))
    assert 4500 < nfa.Q < 6000 and len(finals) == 256 and nfa.final.sum() == 256
    t = W.text_dna(200_000, 1)
    frac = np.bincount(t, minlength=4) / len(t)
    assert abs(frac[0] - 0.3) < 0.01 and abs(frac[1] - 0.2) < 0.01
    trie, fo = W.trie_dfa(W.signature_set(0))
    assert 4000 < trie.Q < 32767 and trie.final.sum() == len(set(fo.values()))


def test_batch_and_serve_workloads_have_the_stated_shape():
    w = W.batch_workload(seed=1, n_texts=50, lo=100, hi=5000, n_nfa=1, n_trie=1,
                         nfa_motifs=8, trie_sigs=20)
    lens = np.diff(w.offsets)
    assert len(lens) == 50 and lens.min() >= 100 and lens.max() <= 5000
    assert set(np.unique(w.job_aut)) <= {0, 1}
    s = W.serve_workload(seed=1, n_req=2000, n_aut=6, size_lo=64, size_hi=256)
    assert len(s.automata) == 6 and (np.diff(s.arrivals) >= 0).all()
    assert s.lengths.max() <= 4 << 20 and s.lengths.min() >= 1
    counts = np.bincount(s.req_aut, minlength=6)
    assert counts[0] > counts[-1]          # Zipf: the first machine is the most popular


def test_tuner_candidates_and_cache(tmp_path, monkeypatch):
    from paper_1110_1716_gb300 import tune
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "cache.json"))
    c = tune.candidates("nfa", 4, 6)
    assert c and all(1 <= x["prefix_k"] <= 8 for x in c)
    assert all(x["threads"] in (256, 512) for x in c)
    tune._store("nfa/Q10/S4/gpu", {"prefix_k": 6}, 1.5)
    assert json.load(open(tmp_path / "cache.json"))["nfa/Q10/S4/gpu"]["params"] == {"prefix_k": 6}
