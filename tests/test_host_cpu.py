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


def test_tuner_axes_and_cache(tmp_path, monkeypatch):
    from paper_1110_1716_gb300 import tune
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "sub" / "cache.json"))
    ax = tune.axes("nfa", 4, 8)
    assert ax["prefix_k"] and all(1 <= k <= 8 for k in ax["prefix_k"])
    assert set(ax["spt"]) == {8, 32} and set(ax["threads"]) == {256, 512}
    assert set(ax["settle"]) == {8, 16} and "table_smem" not in ax
    dfa = tune.axes("dfa", 256, 2)
    assert set(dfa["table_smem"]) == {-1, 0, 1} and "settle" not in dfa
    assert max(dfa["prefix_k"]) == 2            # 8-bit symbols: 16 bits of index
    c = tune.candidates("dfa", 4, 6)
    assert len(c) == np.prod([len(v) for v in tune.axes("dfa", 4, 6).values()])
    tune._store("nfa/Q10/S4/gpu", {"prefix_k": 6}, 1.5)
    assert json.load(open(tmp_path / "sub" / "cache.json"))["nfa/Q10/S4/gpu"]["params"] == {"prefix_k": 6}
    # the default cache sits outside the package directory
    import paper_1110_1716_gb300 as pkg
    assert not tune._default_cache_path().startswith(os.path.dirname(pkg.__file__))


def test_tuner_descent_finds_the_minimum_axis_by_axis():
    from paper_1110_1716_gb300 import tune
    cost = {"a": {0: 5.0, 1: 3.0, 2: 4.0}, "b": {0: 2.0, 1: 1.0}}
    calls = []

    def timer(p):
        calls.append(dict(p))
        return cost["a"][p["a"]] + cost["b"][p["b"]]

    best, ms, evals = tune._descend({"a": 0, "b": 0}, {"a": [0, 1, 2], "b": [0, 1]}, timer)
    assert best == {"a": 1, "b": 1} and ms == 4.0
    assert evals == len(calls) and len({json.dumps(c, sort_keys=True) for c in calls}) == evals


def test_tuner_descent_keeps_the_start_unless_a_candidate_wins_by_the_margin():
    """A candidate replaces the best only when it takes less than `gain`
    times its time: a 2 % gain is noise for the batch tuner (gain 0.97) and
    a win for the single-scan tuner (gain 0.99)."""
    from paper_1110_1716_gb300 import tune
    cost = {0: 1.00, 1: 0.98, 2: 0.90}

    def timer(p):
        return cost[p["a"]] if p["a"] != 2 else None   # 2 does not fit

    assert tune._descend({"a": 0}, {"a": [0, 1, 2]}, timer, gain=0.97)[0] == {"a": 0}
    assert tune._descend({"a": 0}, {"a": [0, 1, 2]}, timer, gain=0.99)[0] == {"a": 1}


# ---------------------------------------------------------------- serving: batch packing
class _Req:
    def __init__(self, aut, n):
        self.aut = aut
        self.text = bytes(n)


def _pack(reqs, **kw):
    import collections
    from paper_1110_1716_gb300.serve import pack_batch
    q = collections.deque(reqs)
    args = dict(max_jobs=8, text_bytes=1 << 20, aut_bytes=[100] * 8, budget=1 << 30,
                one_machine=False)
    args.update(kw)
    got, used = pack_batch(q, **args)
    return got, used, list(q)


def test_pack_batch_in_order_with_job_and_arena_limits():
    rs = [_Req(i % 3, 10 + i) for i in range(12)]
    got, used, left = _pack(rs, max_jobs=5)
    assert got == rs[:5] and left == rs[5:]
    assert used == sum((len(r.text) + 15) & ~15 for r in rs[:5])
    # texts start on 16-byte boundaries; the first one that does not fit the
    # arena ends the batch (10, 11, 12, 13 bytes fill 64; 14 more do not fit)
    got, used, left = _pack(rs, text_bytes=64)
    assert got == rs[:4] and left == rs[4:] and used == 64


def test_pack_batch_keeps_machines_within_the_budget():
    sizes = [60, 50, 30, 10]
    rs = [_Req(0, 5), _Req(1, 5), _Req(0, 5), _Req(2, 5), _Req(3, 5), _Req(1, 5)]
    got, used, left = _pack(rs, aut_bytes=sizes, budget=100)
    # machine 0 (60) then 2 (30) then 3 (10) fit; machine 1 (50) does not: its
    # requests stay at the front, in order, for the next batch
    assert [r.aut for r in got] == [0, 0, 2, 3]
    assert left == [rs[1], rs[5]]
    # a machine larger than the budget alone is still taken (the library
    # reports E_NOMEM if it cannot be made resident)
    got, used, left = _pack([_Req(1, 5), _Req(0, 5)], aut_bytes=sizes, budget=40)
    assert [r.aut for r in got] == [1] and [r.aut for r in left] == [0]


def test_pack_batch_one_machine():
    rs = [_Req(2, 5), _Req(1, 5), _Req(2, 5), _Req(3, 5), _Req(2, 5)]
    got, used, left = _pack(rs, one_machine=True)
    assert [r.aut for r in got] == [2, 2, 2] and [r.aut for r in left] == [1, 3]


def test_bench_work_rate_counts_pair_steps():
    """The bench's work figure: the oracle's pair-step count over the whole
    text (here a complete DFA: n(n+1)/2) per second of kernel time, reported
    as a rate with no machine peak beside it."""
    import bench
    import oracle
    import workloads as W
    d = W.dfa_random(5, Q=7, S=3, dead=-1, finals=[1, 2], p_dead=0.0)
    text = W.text_uniform(3000, 3, 9)
    res = {"aut": d, "text": text, "kernel_ms": 2.0, "matches": len(oracle.scan(d, text))}
    w = bench.work_rate(res)
    assert w["pair_steps"] == 3000 * 3001 // 2
    assert w["matches_agree"] and w["oracle_matches"] == res["matches"]
    assert w["achieved"] == w["pair_steps"] / 2e-3
    assert "frac" not in w and "peak" not in w


def test_bench_compact_configs_keep_every_config():
    """The one-line summary at the end of the bench line has an entry per
    configuration (c0-c4 and both lazy/chained comparisons), with the
    scheduler's longest pass and its on-CPU time per load."""
    import bench

    def scan(gbps):
        return {"gbps": gbps, "kernel_ms": 0.1, "roofline": {"frac": 0.1},
                "e2e": {"value": 1.0}, "matches": 7, "load_ms": 3.0, "device_bytes": 2e6}

    loads = {k: {"p99_ms": 2.0, "max_loop_gap_ms": 9.0,
                 "max_loop_gap_parts": {"thread_cpu_ms": 8.5}} for k in ("0.25", "0.5")}
    others = {
        "dna_dfa_1mib": scan(20.0), "byte_trie_1gib": scan(1400.0),
        "batch_10k_texts": {"gbps": 240.0, "device_gbps": 260.0, "roofline": {"frac": 0.04},
                            "e2e": {"value": 110.0}, "plain_gbps": 3.4, "speedup_vs_plain": 70.0,
                            "params_source": "autotuner", "tuned_batch": {"threads": 0},
                            "default_params_device_ms": 4.3, "device_ms": 4.3},
        "long_lived_dfa_16kib": {"lazy": {"ms": 160.0}, "chained": {"ms": 12.0}, "matches": 5},
        "long_lived_nfa_16kib": {"lazy": {"ms": 860.0}, "chained": {"ms": 100.0}, "matches": 6},
        "serving": {"p50_ms": 1.0, "p99_ms": 5.0, "offered_load": 0.5, "served_gbps": 0.3,
                    "burst_req_per_s": 5e4, "plain_req_per_s": 1e4, "loads": loads,
                    "small_budget": {"p50_ms": 1.5, "p99_ms": 10.0, "evictions": 3}},
    }
    out = bench.compact_configs("motif_nfa_64mib", scan(300.0), others, {"main": {}})
    assert list(out) == ["c0_dna_dfa_1mib", "c1_motif_nfa_64mib", "c2_byte_trie_1gib",
                         "c3_batch_10k_texts", "f2_long_lived_dfa_16kib",
                         "f2_long_lived_nfa_16kib", "c4_serving"]
    assert out["f2_long_lived_nfa_16kib"] == {"lazy_ms": 860.0, "chained_ms": 100.0, "matches": 6}
    assert out["c4_serving"]["max_pass_ms_by_load"]["0.25"] == [9.0, 8.5]
    assert out["c3_batch_10k_texts"]["params_source"] == "autotuner"
