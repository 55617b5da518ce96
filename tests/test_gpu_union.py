"""Union machines (Sec. III.A) and changing them while scans run.

A union of automata through an ancillary initial state with epsilon edges
to every component's q0 reports exactly the union of the components' match
sets. `pfsm_scan_union` runs the components as one batch over the same text;
the oracle scans the union machine itself, built here the paper's way and
made epsilon-free, and its final states are mapped back to (component, state).
"""
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


def as_nfa(a):
    return W.dfa_as_nfa(a) if isinstance(a, W.Dfa) else a


def union_machine(components):
    """Ancillary state 0 with epsilon edges to each component's q0; component
    i's states are shifted by offset[i]. Returns (epsilon-free union, offsets)."""
    S = components[0].S
    offsets, edges, finals, eps = [], [], [], []
    q = 1
    for c in components:
        n = as_nfa(c)
        offsets.append(q)
        for s in range(n.Q):
            for a in range(S):
                for t in W.nfa_succ(n, s, a):
                    edges.append((q + s, a, q + t))
        finals += [q + f for f in np.nonzero(n.final)[0]]
        eps.append((0, q + n.q0))
        q += n.Q
    u = W.nfa_from_edges(q, S, 0, edges, finals, eps_edges=eps)
    return W.eps_free(u), offsets


def components():
    motifs = W.motif_set(81, n_motifs=32, len_lo=6, len_hi=10)
    nfa = W.motif_nfa(motifs)[0]
    rng = np.random.default_rng(82)
    Q = 12
    edges = [(q, x, t) for q in range(Q) for x in range(4) for t in range(Q)
             if (t > q or q == 0) and rng.random() < 0.25]
    fwd = W.nfa_from_edges(Q, 4, 0, edges, [3, 7, 11])
    return [W.dfa_random(83, Q=32, S=4), nfa, fwd, W.dfa_random(84, Q=20, S=4, p_dead=0.5)], motifs


def to_union_states(rows, offsets):
    rows = np.asarray(rows, dtype=np.uint32).reshape(-1, 4)
    off = np.asarray(offsets, dtype=np.uint32)[rows[:, 0]]
    return oracle.sort_matches(np.stack([rows[:, 1], rows[:, 2], rows[:, 3] + off], 1))


def test_union_scan_equals_the_union_machine(pf):
    comps, motifs = components()
    u, offsets = union_machine(comps)
    t = W.text_dna(30_000, 85)
    W.plant_motifs(t, motifs, 500, 86)
    want = oracle.scan(u, t)
    ids = [pf.load(c) for c in comps]
    tt = pf.to_device(t)
    st, counts, total = P.pfsm_scan_union(pf.ctx, ids, tt, None, None, 0)
    out = torch.empty((int(total) + 16, 4), dtype=torch.int32, device="cuda")
    st, counts, total = P.pfsm_scan_union(pf.ctx, ids, tt, None, out)
    assert st == P.PFSM_OK and total == len(want)
    assert np.array_equal(to_union_states(out[:total].cpu().numpy(), offsets), want)
    # per-component counts are the components' own match counts
    for i, c in enumerate(comps):
        assert int(counts[i]) == len(oracle.scan(c, t)), i


def test_components_change_while_scans_run():
    """Remove one component and add another while scans that read it are
    still queued on another stream: the queued scans keep their images, the
    new union sees the new set, and the unload does not wait for the first
    stream (the image is retired and freed after its last scan)."""
    comps, motifs = components()
    t = W.text_dna(200_000, 87)
    W.plant_motifs(t, motifs, 500, 88)
    want = [oracle.scan(c, t) for c in comps[:3]]
    extra = W.dfa_random(89, Q=24, S=4)
    want_extra = oracle.scan(extra, t)
    pf = P.Pfsm(0)
    try:
        ids = [pf.load(c) for c in comps[:3]]
        tt = pf.to_device(t)
        st, counts, total = P.pfsm_scan_union(pf.ctx, ids, tt, None, None, 0)
        reps = 12
        outs = [torch.empty((int(total) + 16, 4), dtype=torch.int32, device="cuda")
                for _ in range(reps)]
        stats = torch.zeros((reps, 5), dtype=torch.int64, device="cuda")
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        for r in range(reps):
            P.pfsm_scan_union_async(pf.ctx, ids, tt, None, outs[r], stats[r], stream=s1)
        # change the union at once: drop component 2 (its scans are queued), add one
        P.pfsm_unload(pf.ctx, ids[2])
        new_ids = [ids[0], ids[1], pf.load(extra)]
        st2, _, total2 = P.pfsm_scan_union(pf.ctx, new_ids, tt, None, None, 0, stream=s2)
        out2 = torch.empty((int(total2) + 16, 4), dtype=torch.int32, device="cuda")
        st2, counts2, total2 = P.pfsm_scan_union(pf.ctx, new_ids, tt, None, out2, stream=s2)
        assert st2 == P.PFSM_OK
        torch.cuda.synchronize()
        s = stats.cpu().numpy()
        for r in range(reps):
            assert s[r, 1] == 0 and list(s[r, 2:5]) == [len(w) for w in want], r
        rows = outs[-1][:int(s[-1, 0])].cpu().numpy().view(np.uint32)
        for i in range(3):
            assert np.array_equal(oracle.sort_matches(rows[rows[:, 0] == i][:, 1:]), want[i]), i
        rows2 = out2[:total2].cpu().numpy().view(np.uint32)
        for i, w in enumerate([want[0], want[1], want_extra]):
            assert np.array_equal(oracle.sort_matches(rows2[rows2[:, 0] == i][:, 1:]), w), i
        with pytest.raises(P.PfsmError):
            P.pfsm_aut_bytes(pf.ctx, ids[2])
        # every scan is done: only the three live machines hold device memory
        live = sum(P.pfsm_aut_bytes(pf.ctx, a)[0] for a in new_ids)
        assert P.pfsm_get_stats(pf.ctx)["resident_bytes"] == live
    finally:
        pf.close()
