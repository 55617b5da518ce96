"""GPU parity of the batched scan (one persistent launch over many texts,
each with its own machine) against the CPU oracle, per text."""
import numpy as np
import pytest

import oracle
import workloads as W

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


def split_by_text(m: np.ndarray, k: int):
    m = np.asarray(m, dtype=np.uint32).reshape(-1, 4)
    out = []
    order = np.argsort(m[:, 0], kind="stable")
    m = m[order]
    bounds = np.searchsorted(m[:, 0], np.arange(k + 1))
    for i in range(k):
        out.append(oracle.sort_matches(m[bounds[i]:bounds[i + 1], 1:]))
    return out


def machines():
    sigs = W.signature_set(77, n_sigs=150)
    trie, _ = W.trie_dfa(sigs)
    motifs = W.motif_set(78, n_motifs=64)
    nfa, _ = W.motif_nfa(motifs)
    rng = np.random.default_rng(79)
    Q = 12
    edges = [(q, x, t) for q in range(Q) for x in range(4) for t in range(Q)
             if (t > q or q == 0) and rng.random() < 0.25]
    fwd = W.nfa_from_edges(Q, 4, 0, edges, [3, 7, 11])
    return [("dna_dfa", W.dfa_random(5), 4), ("trie", trie, 256), ("motif_nfa", nfa, 4),
            ("fwd_nfa", fwd, 4), ("small_dfa", W.dfa_random(6, Q=20, S=17, p_dead=0.2), 17)]


LENGTHS = [0, 1, 15, 100, 4095, 16384, 16385, 50000, 120001]


def make_jobs(ms, seed, lengths=LENGTHS, plants=True):
    rng = np.random.default_rng(seed)
    jobs = []
    for i, n in enumerate(lengths * 2):
        mi = int(rng.integers(0, len(ms)))
        name, m, S = ms[mi]
        if S == 4:
            t = W.text_dna(n, seed * 1000 + i)
        else:
            t = W.text_uniform(n, S, seed * 1000 + i)
        jobs.append((mi, t))
    return jobs


def test_batch_matches_oracle_per_text(pf):
    ms = machines()
    ids = [pf.load(m) for _, m, _ in ms]
    jobs = make_jobs(ms, 1)
    got, counts = pf.scan_batch([(ids[mi], t) for mi, t in jobs])
    per = split_by_text(got.cpu().numpy().view(np.uint32), len(jobs))
    for j, (mi, t) in enumerate(jobs):
        want = oracle.scan(ms[mi][1], t)
        assert int(counts[j]) == len(want), (j, ms[mi][0], len(t))
        assert np.array_equal(per[j], want), (j, ms[mi][0], len(t))


def test_batch_equals_single_scans_on_mixed_workload(pf):
    w = W.batch_workload(seed=3, n_texts=120, lo=100, hi=1 << 18, n_nfa=2, n_trie=2,
                         nfa_motifs=128, trie_sigs=300)
    ids = [pf.load(a) for a in w.automata]
    data = pf.to_device(w.data)
    jobs = []
    for i in range(len(w.job_aut)):
        lo, hi = int(w.offsets[i]), int(w.offsets[i + 1])
        jobs.append((ids[int(w.job_aut[i])], data[lo:hi], hi - lo))
    out = torch.empty((200_000, 4), dtype=torch.int32, device="cuda")
    st, counts, total = P.pfsm_scan_batch(pf.ctx, jobs, out)
    assert st == P.PFSM_OK
    per = split_by_text(out[:total].cpu().numpy().view(np.uint32), len(jobs))
    for i, (aid, tt, n) in enumerate(jobs):
        single = oracle.sort_matches(pf.scan_numpy(aid, tt))
        assert np.array_equal(per[i], single), i
    # and a sample against the oracle
    for i in range(0, len(jobs), 17):
        lo, hi = int(w.offsets[i]), int(w.offsets[i + 1])
        assert np.array_equal(per[i], oracle.scan(w.automata[int(w.job_aut[i])], w.data[lo:hi]))


def test_batch_overflow_and_async_status(pf):
    ms = machines()
    ids = [pf.load(m) for _, m, _ in ms]
    jobs = make_jobs(ms, 2)
    dj = [(ids[mi], pf.to_device(t), len(t)) for mi, t in jobs]
    want = [len(oracle.scan(ms[mi][1], t)) for mi, t in jobs]
    out = torch.empty((5, 4), dtype=torch.int32, device="cuda")
    st, counts, total = P.pfsm_scan_batch(pf.ctx, dj, out)
    assert st == P.PFSM_E_OVERFLOW and total == sum(want)
    assert [int(c) for c in counts] == want
    s = torch.cuda.Stream()
    out = torch.empty((total + 1, 4), dtype=torch.int32, device="cuda")
    status = torch.zeros(len(dj) + 2, dtype=torch.int64, device="cuda")
    P.pfsm_scan_batch_async(pf.ctx, dj, out, status, stream=s)
    s.synchronize()
    stv = status.cpu().numpy()
    assert stv[0] == total and stv[1] == 0 and list(stv[2:]) == want


def test_graph_replay_across_batches(pf):
    ms = machines()
    ids = [pf.load(m) for _, m, _ in ms]
    for seed in (4, 5, 6):
        jobs = make_jobs(ms, seed, lengths=[300, 7000, 33333])
        got, counts = pf.scan_batch([(ids[mi], t) for mi, t in jobs])
        per = split_by_text(got.cpu().numpy().view(np.uint32), len(jobs))
        for j, (mi, t) in enumerate(jobs):
            assert np.array_equal(per[j], oracle.scan(ms[mi][1], t))


def test_batch_errors(pf):
    d = W.dfa_random(1)
    a = pf.load(d)
    t = pf.to_device(W.text_uniform(1000, 4, 1))
    out = torch.empty((10, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(P.PfsmError) as e:
        P.pfsm_scan_batch(pf.ctx, [(a, t, 1000), (123456, t, 1000)], out)
    assert e.value.status == P.PFSM_E_NOENT
    bad = W.text_uniform(1000, 4, 2)
    bad[500] = 9
    with pytest.raises(P.PfsmError) as e:
        P.pfsm_scan_batch(pf.ctx, [(a, pf.to_device(bad), 1000)], out)
    assert e.value.status == P.PFSM_E_INVAL
    st, counts, total = P.pfsm_scan_batch(pf.ctx, [], out)
    assert st == P.PFSM_OK and total == 0


def test_batch_under_small_budget_reloads(pf):
    autos = [W.dfa_random(60 + i, Q=64, S=4) for i in range(6)]
    sizes = []
    for x in autos:
        before = P.pfsm_get_stats(pf.ctx)["resident_bytes"]
        a = pf.load(x)
        sizes.append(P.pfsm_get_stats(pf.ctx)["resident_bytes"] - before)
        P.pfsm_unload(pf.ctx, a)
    budget = int(3.5 * max(sizes))     # any three fit together, all six do not
    assert budget < sum(sizes)
    small = P.Pfsm(0, budget_bytes=budget)
    try:
        ids = [small.load(x) for x in autos]
        texts = [W.text_uniform(20_000, 4, 70 + i) for i in range(6)]
        for rnd in range(2):
            for grp in ([0, 1, 2], [3, 4, 5], [1, 3, 5]):
                got, counts = small.scan_batch([(ids[g], texts[g]) for g in grp])
                per = split_by_text(got.cpu().numpy().view(np.uint32), len(grp))
                for j, g in enumerate(grp):
                    assert np.array_equal(per[j], oracle.scan(autos[g], texts[g]))
        st = P.pfsm_get_stats(small.ctx)
        assert st["evictions"] > 0 and st["reloads"] > 0
    finally:
        small.close()


def test_batch_mixes_lazy_and_chained_machines(pf):
    """Long-lived DFA instances in one batch: one machine continues them in
    place (lazy), the other through the carry queue (chained)."""
    ms = [W.dfa_random(20 + i, Q=6, S=4, dead=-1, finals=[1, 3], p_dead=0.0) for i in range(2)]
    ids = [pf.load(m) for m in ms]
    P.pfsm_set_params(pf.ctx, ids[0], {"partition": 1})
    P.pfsm_set_params(pf.ctx, ids[1], {"partition": 2})
    texts = [W.text_uniform(5000 + 700 * i, 4, 30 + i) for i in range(4)]
    jobs = [(ids[i % 2], t) for i, t in enumerate(texts)]
    want = [oracle.scan(ms[i % 2], t) for i, t in enumerate(texts)]
    P.pfsm_set_batch_params(pf.ctx, {"tile": 4096})
    try:
        got, counts = pf.scan_batch(jobs)
    finally:
        P.pfsm_set_batch_params(pf.ctx, None)
    per = split_by_text(got.cpu().numpy().view(np.uint32), len(jobs))
    for j in range(len(jobs)):
        assert int(counts[j]) == len(want[j]), j
        assert np.array_equal(per[j], want[j]), j
