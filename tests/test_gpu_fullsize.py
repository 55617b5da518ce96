"""Full-size parity: the three single-text scan workloads and the whole
many-texts batch compared with the oracle on every start (the oracle split
into start windows over every host core), element by element."""
import concurrent.futures
import os

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import oracle_parallel

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def test_motif_nfa_64mib_full(pf):
    """The headline workload: 256 motifs as a position NFA, 64 MiB of DNA."""
    nfa, t, motifs, plants = W.workload_motif_nfa(0)
    got = gpu_matches(pf, pf.load(nfa), t)
    want = oracle_parallel(nfa, t)
    assert got.shape == want.shape and np.array_equal(got, want)
    assert len(got) >= len(plants)


def test_byte_trie_1gib_full(pf):
    """1000 byte signatures as a trie DFA, 1 GiB of uniform bytes."""
    d, t, sigs, final_of, plants = W.workload_byte_trie(0)
    got = gpu_matches(pf, pf.load(d), t)
    want = oracle_parallel(d, t)
    assert got.shape == want.shape and np.array_equal(got, want)
    # each match spells a signature ending in that final state, and each
    # intact planted occurrence is among them
    sig_of = {f: s for s, f in final_of.items()}
    tb = memoryview(t)
    for i, j, f in got:
        assert bytes(tb[i:j + 1]) == sig_of[int(f)]
    have = set(map(tuple, got.tolist()))
    for pos, i in plants:
        s = sigs[i]
        if bytes(tb[pos:pos + len(s)]) == s:
            assert (pos, pos + len(s) - 1, final_of[s]) in have


def test_dna_dfa_1mib_full_every_seed(pf):
    for seed in range(5):
        d, t = W.workload_dna_dfa(seed)
        assert np.array_equal(gpu_matches(pf, pf.load(d), t), oracle.scan(d, t)), seed


WIN = 32 << 10   # start window length for the long texts of the batch


def batch_oracle(w, i):
    """Oracle matches of text i of the batch: every start of a text of at
    most 4 windows, else the starts of its first, middle and last window
    (disjoint: the middle one ends before the last one begins)."""
    a = w.automata[int(w.job_aut[i])]
    t = w.data[int(w.offsets[i]):int(w.offsets[i + 1])]
    n = len(t)
    if n <= 4 * WIN:
        wins = [(0, n)]
    else:
        mid = (n // 2) & ~15
        wins = [(0, WIN), (mid, mid + WIN), (n - WIN, n)]
    got = [oracle.scan(a, t, lo, hi) for lo, hi in wins]
    got = [g for g in got if len(g)]
    want = oracle.sort_matches(np.concatenate(got)) if got else np.zeros((0, 3), np.uint32)
    return wins, want


def test_batch_10k_texts_against_the_oracle(pf):
    """The whole 10,000-text batch (8 motif NFAs and 8 byte tries, lengths
    log-uniform 100 B - 1 MiB) in one pfsm_scan_batch call; every text's
    matches are compared with the oracle's (long texts on three start
    windows), and the per-text counts with the rows returned."""
    w = W.batch_workload(seed=0)
    ids = np.array([pf.load(a) for a in w.automata], dtype=np.int32)
    data = pf.to_device(w.data)
    lengths = np.diff(w.offsets)
    table = P.job_table(ids[w.job_aut], data.data_ptr() + w.offsets[:-1], lengths)
    st, counts, total = P.pfsm_scan_batch(pf.ctx, table, None, 0)
    out = torch.empty((int(total) + 1024, 4), dtype=torch.int32, device=data.device)
    st, counts, total = P.pfsm_scan_batch(pf.ctx, table, out, out.shape[0])
    assert st == P.PFSM_OK
    m = out[:int(total)].cpu().numpy().view(np.uint32)
    order = np.argsort(m[:, 0], kind="stable")
    m = m[order]
    bounds = np.searchsorted(m[:, 0], np.arange(len(lengths) + 1))
    assert np.array_equal(np.diff(bounds), np.asarray(counts, dtype=np.int64))
    cores = max(1, os.cpu_count() or 1)
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
        results = list(ex.map(lambda i: batch_oracle(w, i), range(len(lengths))))
    for i, (wins, want) in enumerate(results):
        got = oracle.sort_matches(m[bounds[i]:bounds[i + 1], 1:])
        if len(wins) > 1:
            keep = np.zeros(len(got), dtype=bool)
            for lo, hi in wins:
                keep |= (got[:, 0] >= lo) & (got[:, 0] < hi)
            got = got[keep]
        assert np.array_equal(got, want), i
    for a in ids:
        P.pfsm_unload(pf.ctx, int(a))
