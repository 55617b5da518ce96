"""Texts that do not start on a 16-byte boundary: every tile is copied from
the boundary below its first byte and moved down in shared memory. Parity
with the oracle for every shift 1..15, for single scans and for batches
whose texts are packed back to back at arbitrary offsets."""
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


def cases():
    motifs = W.motif_set(91, n_motifs=48)
    nfa, _ = W.motif_nfa(motifs)
    t_nfa = W.text_dna(23_001, 92)
    W.plant_motifs(t_nfa, motifs, 700, 93)
    sigs = W.signature_set(94, n_sigs=120)
    trie, _ = W.trie_dfa(sigs)
    t_trie = W.text_uniform(21_003, 256, 95)
    W.plant_signatures(t_trie, sigs, 500, 96)
    dfa = W.dfa_random(97)
    t_dfa = W.text_uniform(9_005, 4, 98)
    return [("motif_nfa", nfa, t_nfa), ("trie", trie, t_trie), ("dna_dfa", dfa, t_dfa)]


@pytest.mark.parametrize("which", [0, 1, 2])
def test_single_scan_every_shift(pf, which):
    name, m, t = cases()[which]
    a = pf.load(m)
    # several tiles and a ragged tail at every shift
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 2048})
    want = oracle.scan(m, t)
    assert len(want) > 0
    out = torch.empty((len(want) + 1024, 3), dtype=torch.int32, device="cuda")
    for sh in range(1, 16):
        buf = pf.to_device(np.concatenate([np.full(sh, 7, np.uint8), t, np.full(5, 3, np.uint8)]))
        view = buf[sh:sh + len(t)]
        assert view.data_ptr() % 16 == sh % 16
        st, cnt = P.pfsm_scan(pf.ctx, a, view, len(t), out)
        assert st == P.PFSM_OK
        got = oracle.sort_matches(out[:cnt].cpu().numpy().view(np.uint32))
        assert np.array_equal(got, want), (name, sh)


def test_batch_packed_at_every_shift(pf):
    cs = cases()
    ids = [pf.load(m) for _, m, _ in cs]
    rng = np.random.default_rng(99)
    pieces, jobs, want = [], [], []
    off = 0
    for i in range(48):
        ci = i % 3
        name, m, t = cs[ci]
        # a prefix of the case's text, of a length that spans zero to several tiles
        n = int(rng.integers(0, len(t) + 1)) if i % 5 else len(t)
        pad = int(rng.integers(0, 16))   # next text starts at an arbitrary offset
        pieces.append(np.full(pad, 1, np.uint8))
        off += pad
        pieces.append(t[:n])
        jobs.append((ci, off, n))
        off += n
        want.append(oracle.scan(m, t[:n]))
    data = pf.to_device(np.concatenate(pieces + [np.zeros(16, np.uint8)]))
    shifts = {(data.data_ptr() + o) % 16 for _, o, n in jobs if n}
    assert len(shifts) >= 12
    table = P.job_table([ids[ci] for ci, _, _ in jobs], [data.data_ptr() + o for _, o, _ in jobs],
                        [n for _, _, n in jobs])
    P.pfsm_set_batch_params(pf.ctx, {"tile": 4096})
    try:
        st, counts, total = P.pfsm_scan_batch(pf.ctx, table, None, 0)
        out = torch.empty((int(total) + 16, 4), dtype=torch.int32, device="cuda")
        st, counts, total = P.pfsm_scan_batch(pf.ctx, table, out)
    finally:
        P.pfsm_set_batch_params(pf.ctx, None)
    assert st == P.PFSM_OK
    m = out[:total].cpu().numpy().view(np.uint32)
    m = m[np.argsort(m[:, 0], kind="stable")]
    bounds = np.searchsorted(m[:, 0], np.arange(len(jobs) + 1))
    for j in range(len(jobs)):
        got = oracle.sort_matches(m[bounds[j]:bounds[j + 1], 1:])
        assert int(counts[j]) == len(want[j]), j
        assert np.array_equal(got, want[j]), (j, cs[jobs[j][0]][0], jobs[j][2])
