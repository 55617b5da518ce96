"""The continuous-batching server: every request's result in the mix equals
the same text scanned alone, and the oracle on a sample."""
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_1716_gb300 as P  # noqa: E402
from paper_1110_1716_gb300.serve import Server, replay  # noqa: E402


def small_fleet(seed):
    rng = np.random.default_rng(seed)
    autos, alph = [], []
    for i in range(12):
        kind = i % 3
        size = int(np.exp(rng.uniform(np.log(64), np.log(2048))))
        a, S = W.serve_automaton(seed * 100 + i, kind, size)
        autos.append(a)
        alph.append(S)
    return autos, alph


def requests(autos, alph, k, seed, median=2048, max_len=256 << 10):
    rng = np.random.default_rng(seed)
    auts = rng.integers(0, len(autos), size=k)
    lens = np.minimum(np.exp(rng.normal(np.log(median), 1.5, size=k)), max_len).astype(int) + 1
    texts = []
    for i in range(k):
        S = alph[auts[i]]
        texts.append(W.text_dna(int(lens[i]), seed * 7919 + i) if S == 4
                     else W.text_uniform(int(lens[i]), 256, seed * 7919 + i))
    return auts, texts


@pytest.fixture(scope="module")
def fleet():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return small_fleet(3)


def alone(pf, ids, auts, texts):
    return [oracle.sort_matches(pf.scan_numpy(ids[a], t)) for a, t in zip(auts, texts)]


def test_mix_equals_alone_burst(fleet):
    autos, alph = fleet
    auts, texts = requests(autos, alph, 300, 11)
    with P.Pfsm(0) as pf:
        srv = Server(pf, autos, slots=3, slot_bytes=1 << 20, out_rows=1 << 18, max_jobs=64)
        with srv:
            futs = [srv.submit(int(a), t) for a, t in zip(auts, texts)]
            got = [oracle.sort_matches(f.result(timeout=120)) for f in futs]
        assert srv.batches > 3   # requests were split over several concurrent batches
        ref = alone(pf, srv.ids, auts, texts)
        for i in range(len(texts)):
            assert np.array_equal(got[i], ref[i]), i
        for i in range(0, len(texts), 25):
            assert np.array_equal(got[i], oracle.scan(autos[auts[i]], texts[i])), i
        st = srv.latency_stats()
        assert st["requests"] == len(texts) and st["p99_ms"] >= st["p50_ms"] > 0


def fleet_bytes(autos):
    """Device bytes of each machine, read from the residency counters."""
    sizes = []
    with P.Pfsm(0) as pf:
        for a in autos:
            before = P.pfsm_get_stats(pf.ctx)["resident_bytes"]
            pf.load(a)
            sizes.append(P.pfsm_get_stats(pf.ctx)["resident_bytes"] - before)
    return sizes


def test_mix_equals_alone_poisson_with_evictions(fleet):
    autos, alph = fleet
    auts, texts = requests(autos, alph, 400, 12, median=1024)
    sizes = fleet_bytes(autos)
    budget = max(2 * max(sizes), sum(sizes) // 2)
    assert budget < sum(sizes)
    with P.Pfsm(0, budget_bytes=budget) as pf:
        srv = Server(pf, autos, slots=3, slot_bytes=1 << 20, out_rows=1 << 18, max_jobs=32)
        arrivals = np.cumsum(np.random.default_rng(5).exponential(1 / 4000.0, size=len(texts)))
        with srv:
            futs = replay(srv, arrivals, auts, texts)
            got = [oracle.sort_matches(f.result(timeout=120)) for f in futs]
        st = srv.latency_stats()
        assert st["residency_evictions"] > 0 and st["residency_reloads"] > 0
        ref = alone(pf, srv.ids, auts, texts)
        for i in range(len(texts)):
            assert np.array_equal(got[i], ref[i]), i


def test_overflowing_batch_is_rerun(fleet):
    d = W.dfa_random(1)
    texts = [W.text_uniform(30_000, 4, 40 + i) for i in range(6)]
    with P.Pfsm(0) as pf:
        srv = Server(pf, [d], slots=2, slot_bytes=1 << 20, out_rows=1000, max_jobs=8)
        with srv:
            futs = [srv.submit(0, t) for t in texts]
            got = [oracle.sort_matches(f.result(timeout=60)) for f in futs]
        assert srv.overflow_reruns > 0
        for t, g in zip(texts, got):
            assert np.array_equal(g, oracle.scan(d, t))
