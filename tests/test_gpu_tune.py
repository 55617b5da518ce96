"""The autotuner on the GPU: the parameters it chooses are valid, are the
ones the library then reports, and keep the match set equal to the oracle's
(for single scans and for a batch)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_1716_gb300 as P  # noqa: E402
from paper_1110_1716_gb300 import tune  # noqa: E402


@pytest.fixture(scope="module")
def pf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = P.Pfsm(0)
    yield p
    p.close()


def machines():
    d = W.dfa_random(31)
    nfa, _ = W.motif_nfa(W.motif_set(32, n_motifs=64))
    sigs = W.signature_set(33, n_sigs=200)
    trie, _ = W.trie_dfa(sigs)
    return [("dna_dfa", d, W.text_uniform(1 << 20, 4, 34)),
            ("motif_nfa", nfa, W.text_dna(2 << 20, 35)),
            ("trie", trie, W.text_uniform(2 << 20, 256, 36))]


@pytest.mark.parametrize("which", [0, 1, 2])
def test_tune_keeps_parity(pf, which, tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE_PATH", str(tmp_path / "cache.json"))
    name, m, t = machines()[which]
    aid = pf.load(m)
    td = pf.to_device(t)
    chosen = tune.tune(pf.ctx, aid, m, td, reps=1, sweeps=1)
    assert chosen == P.pfsm_get_params(pf.ctx, aid)
    want = oracle.scan(m, t)
    got = oracle.sort_matches(pf.scan_numpy(aid, td))
    assert np.array_equal(got, want), (name, chosen)
    # the cached choice is applied as it was stored
    P.pfsm_set_params(pf.ctx, aid, None)
    again = tune.tune(pf.ctx, aid, m, td)
    assert again == chosen
    P.pfsm_unload(pf.ctx, aid)


def test_tune_batch_keeps_parity(pf):
    ms = machines()
    ids = [pf.load(m) for _, m, _ in ms]
    kinds = {ids[i]: ("nfa" if name == "motif_nfa" else "dfa") for i, (name, _, _) in enumerate(ms)}
    rng = np.random.default_rng(40)
    texts, jobs = [], []
    for i in range(60):
        mi = int(rng.integers(0, len(ms)))
        n = int(np.exp(rng.uniform(np.log(100), np.log(300_000))))
        S = ms[mi][1].S
        t = W.text_dna(n, 500 + i) if S == 4 else W.text_uniform(n, S, 500 + i)
        texts.append((mi, t))
        jobs.append((ids[mi], pf.to_device(t), n))
    res = tune.tune_batch(pf.ctx, jobs, reps=1, machines=kinds)
    assert set(res["batch"]) == {"threads", "ctas_per_sm", "tile"}
    assert set(res["machines"]) == set(kinds)
    out, counts = pf.scan_batch([(ids[mi], t) for mi, t in texts])
    m = out.cpu().numpy().view(np.uint32)
    for k, (mi, t) in enumerate(texts):
        got = oracle.sort_matches(m[m[:, 0] == k][:, 1:])
        assert np.array_equal(got, oracle.scan(ms[mi][1], t)), k
    P.pfsm_set_batch_params(pf.ctx, None)
    for a in ids:
        P.pfsm_unload(pf.ctx, a)
