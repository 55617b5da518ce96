"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Match sets are compared as sorted (start, end, state) arrays, element by
element (bit-exact: the scan is integer work). Sizes span several tiles and
a ragged tail; the full-size workloads are in test_gpu_fullsize.py (every
start, with the oracle split into start windows on every host core).
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


def in_window(m, lo, hi):
    sel = (m[:, 0] >= lo) & (m[:, 0] < hi)
    return m[sel]


# ---------------------------------------------------------------- worked examples
@pytest.mark.parametrize("fixture", ["fig2_aacacab.txt", "fig3_ac.txt"])
def test_paper_examples_on_gpu(pf, fixture):
    text, want = read_golden(fixture)
    m = W.eps_free(W.fig1_union())
    a = pf.load(m)
    got = gpu_matches(pf, a, W.encode(text, W.FIG1_ALPHABET))
    assert oracle.labelled(got, m.labels) == want


# ---------------------------------------------------------------- text ends
@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_nfa_starts_near_the_end_of_the_text(pf, k):
    """Starts with fewer than k symbols left read the short-gram table; texts
    of every length up to 3k + 2 put each j < k at the end of a text (and of
    a tile), with matches of length 1 (a*c, ac) among them."""
    m = W.eps_free(W.fig1_union())
    a = pf.load(m)
    P.pfsm_set_params(pf.ctx, a, {"prefix_k": k})
    for n in range(0, 3 * k + 3):
        for rep in range(3):
            t = W.text_uniform(n, m.S, 77_000 + 100 * n + rep)
            assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(m, t)), (k, n, rep)
    # a long text whose last tile ends in every phase
    t = W.text_uniform(4096 * 3 + 5, m.S, 78_000 + k)
    P.pfsm_set_params(pf.ctx, a, {"prefix_k": k, "tile": 4096, "halo": 16})
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(m, t)), k


# ---------------------------------------------------------------- small machines, ragged sizes
SIZES = [0, 1, 2, 7, 15, 16, 17, 100, 4095, 4096, 4097, 16383, 16384, 16385, 70001]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_dfa_sizes(pf, seed):
    d = W.dfa_random(300 + seed, Q=12, S=4, p_dead=0.25)
    a = pf.load(d)
    for n in SIZES:
        t = W.text_uniform(n, 4, 1000 * seed + n)
        assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(d, t)), n


def forward_nfa(seed, Q=14, S=4, p=0.25):
    """Random NFA whose edges only go to higher states (q0 excepted), so every
    instance dies within Q steps."""
    rng = np.random.default_rng(seed)
    edges = [(q, x, t) for q in range(Q) for x in range(S) for t in range(Q)
             if (t > q or q == 0) and rng.random() < p]
    fins = [q for q in range(1, Q) if rng.random() < 0.3] or [Q - 1]
    return W.nfa_from_edges(Q, S, 0, edges, fins)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_nfa_sizes(pf, seed):
    m = forward_nfa(40 + seed)
    a = pf.load(m)
    for n in SIZES:
        t = W.text_uniform(n, 4, 77 * seed + n)
        assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(m, t)), n


def test_cyclic_nfa_long_lived_sets(pf):
    """Cycles everywhere: state sets live to the end of the text, past every
    tile's staged bytes (lazy partitioning reads the global text)."""
    rng = np.random.default_rng(41)
    Q, S = 14, 4
    edges = [(q, x, t) for q in range(Q) for x in range(S) for t in range(Q) if rng.random() < 0.12]
    m = W.nfa_from_edges(Q, S, 0, edges, [3, 7, 11])
    a = pf.load(m)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16})
    t = W.text_uniform(700, 4, 2)
    want = oracle.scan(m, t)
    assert len(want) > 100_000
    assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 8), want)


def test_byte_alphabet_and_odd_alphabets(pf):
    for S, seed, pdead in ((2, 22, 0.35), (3, 31, 0.3), (5, 5, 0.3), (17, 17, 0.2),
                           (200, 200, 0.2), (256, 256, 0.2)):
        d = W.dfa_random(seed, Q=20, S=S, p_dead=pdead)
        a = pf.load(d)
        t = W.text_uniform(30011, S, S + 1)
        want = oracle.scan(d, t)
        assert len(want) > 0, S
        assert np.array_equal(gpu_matches(pf, a, t), want), S


# ---------------------------------------------------------------- launch parameters
PARAMS = [
    {"prefix_k": -1},
    {"prefix_k": 1},
    {"prefix_k": 3, "tile": 4096, "halo": 16},
    {"threads": 128, "tile": 8192},
    {"threads": 256, "table_smem": 0},
    {"threads": 512, "tile": 32768, "halo": 4096, "ctas_per_sm": 1},
    {"settle": -1},
    {"settle": 2, "prefix_k": 4},
    {"spt": 32},                                # 32 starts per thread on a short text
    {"spt": 8, "threads": 512, "tile": 4096},   # 8 per thread, several rounds per tile
    {"spt": 8, "partition": 1},
]


@pytest.mark.parametrize("params", PARAMS, ids=lambda p: ",".join("%s=%s" % kv for kv in p.items()))
def test_params_do_not_change_dfa_result(pf, params):
    d, t = W.workload_dna_dfa(1, n=300_000)
    a = pf.load(d)
    P.pfsm_set_params(pf.ctx, a, params)
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(d, t))


@pytest.mark.parametrize("params", PARAMS[:4] + PARAMS[6:],
                         ids=lambda p: ",".join("%s=%s" % kv for kv in p.items()))
def test_params_do_not_change_nfa_result(pf, params):
    nfa, t, _, _ = W.workload_motif_nfa(5, n=150_000, n_motifs=64, every=1500)
    a = pf.load(nfa)
    P.pfsm_set_params(pf.ctx, a, params)
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(nfa, t))


def test_nfa_warp_sets(pf):
    """Without the prefix table the first step from q0 reaches ~85 states, more
    than a lane holds: every instance runs on the warp-cooperative bitset path."""
    nfa, t, _, _ = W.workload_motif_nfa(6, n=40_000, n_motifs=256, every=1000)
    a = pf.load(nfa)
    P.pfsm_set_params(pf.ctx, a, {"prefix_k": -1})
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(nfa, t))


# ---------------------------------------------------------------- full-size workloads
@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_dna_dfa_1mib(pf, seed):
    d, t = W.workload_dna_dfa(seed)
    got = gpu_matches(pf, pf.load(d), t)
    want = oracle.scan(d, t)
    assert np.array_equal(got, want)


def test_motif_nfa_4mib_full(pf):
    nfa, t, _, plants = W.workload_motif_nfa(0, n=4 << 20)
    got = gpu_matches(pf, pf.load(nfa), t)
    assert np.array_equal(got, oracle.scan(nfa, t))
    assert len(got) >= len(plants)


def test_byte_trie_16mib_full(pf):
    d, t, sigs, final_of, plants = W.workload_byte_trie(0, n=16 << 20)
    got = gpu_matches(pf, pf.load(d), t)
    assert np.array_equal(got, oracle.scan(d, t))


# ---------------------------------------------------------------- protocol and errors
def test_overflow_reports_required_count(pf):
    d, t = W.workload_dna_dfa(1, n=100_000)
    a = pf.load(d)
    want = oracle.scan(d, t)
    tt = pf.to_device(t)
    out = torch.empty((10, 3), dtype=torch.int32, device="cuda")
    st, cnt = P.pfsm_scan(pf.ctx, a, tt, None, out)
    assert st == P.PFSM_E_OVERFLOW and cnt == len(want)
    out = torch.empty((cnt, 3), dtype=torch.int32, device="cuda")
    st, cnt2 = P.pfsm_scan(pf.ctx, a, tt, None, out)
    assert st == P.PFSM_OK and cnt2 == cnt
    got = oracle.sort_matches(out.cpu().numpy().view(np.uint32))
    assert np.array_equal(got, want)


def test_zero_capacity_counts(pf):
    d, t = W.workload_dna_dfa(2, n=50_000)
    a = pf.load(d)
    st, cnt = P.pfsm_scan(pf.ctx, a, pf.to_device(t), None, None, 0)
    assert cnt == len(oracle.scan(d, t))
    assert st == (P.PFSM_OK if cnt == 0 else P.PFSM_E_OVERFLOW)


def test_bad_symbol_is_rejected(pf):
    d = W.dfa_random(3, Q=10, S=4)
    a = pf.load(d)
    t = W.text_uniform(50_000, 4, 1)
    t[33_333] = 4
    out = torch.empty((100_000, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(P.PfsmError) as e:
        P.pfsm_scan(pf.ctx, a, pf.to_device(t), None, out)
    assert e.value.status == P.PFSM_E_INVAL


def test_unknown_automaton_and_bad_tables(pf):
    out = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    t = pf.to_device(np.zeros(8, dtype=np.uint8))
    with pytest.raises(P.PfsmError) as e:
        P.pfsm_scan(pf.ctx, 987654, t, None, out)
    assert e.value.status == P.PFSM_E_NOENT
    d = W.dfa_random(1, Q=8, S=4)
    bad = d.delta.copy()
    bad[2, 1] = 8
    with pytest.raises(P.PfsmError):
        P.pfsm_load_dfa(pf.ctx, bad, 0, d.dead, d.final)
    nonabs = d.delta.copy()
    nonabs[d.dead, 0] = 1
    with pytest.raises(P.PfsmError):
        P.pfsm_load_dfa(pf.ctx, nonabs, 0, d.dead, d.final)
    finaldead = d.final.copy()
    finaldead[d.dead] = 1
    with pytest.raises(P.PfsmError):
        P.pfsm_load_dfa(pf.ctx, d.delta, 0, d.dead, finaldead)


def test_unaligned_text_pointer(pf):
    d, t = W.workload_dna_dfa(2, n=100_003)
    a = pf.load(d)
    big = pf.to_device(np.concatenate([np.zeros(3, np.uint8), t]))
    view = big[3:]
    assert view.data_ptr() % 16 != 0
    out = torch.empty((400_000, 3), dtype=torch.int32, device="cuda")
    st, cnt = P.pfsm_scan(pf.ctx, a, view, None, out)
    assert st == P.PFSM_OK
    got = oracle.sort_matches(out[:cnt].cpu().numpy().view(np.uint32))
    assert np.array_equal(got, oracle.scan(d, t))


def test_instances_outliving_tiles_use_the_carry_queue(pf):
    """No dead state: every instance lives to the end of the text, so most of
    them leave their tile's staged bytes (chained partitioning)."""
    d = W.dfa_random(8, Q=6, S=4, dead=-1, finals=[1], p_dead=0.0)
    a = pf.load(d)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "prefix_k": 2})
    t = W.text_uniform(9000, 4, 3)
    want = oracle.scan(d, t)
    assert len(want) > 1_000_000
    assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 16), want)


@pytest.mark.parametrize("partition", [1, 2])
def test_lazy_and_chained_partitioning(pf, partition):
    """Sec. III.D.2 both ways on instances that never die: lazy (continue on
    the global text in place) and chained (carry queue, second kernel)."""
    d = W.dfa_random(18, Q=6, S=4, dead=-1, finals=[1, 4], p_dead=0.0)
    a = pf.load(d)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "prefix_k": 2, "partition": partition})
    assert P.pfsm_get_params(pf.ctx, a)["partition"] == partition
    t = W.text_uniform(9000, 4, 19)
    want = oracle.scan(d, t)
    assert len(want) > 1_000_000
    assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 16), want)


def test_nfa_partition_default_is_lazy(pf):
    a = pf.load(W.eps_free(W.fig1_union()))
    assert P.pfsm_get_params(pf.ctx, a)["partition"] == 1
    P.pfsm_set_params(pf.ctx, a, {"partition": 2})
    assert P.pfsm_get_params(pf.ctx, a)["partition"] == 2
    with pytest.raises(P.PfsmError):
        P.pfsm_set_params(pf.ctx, a, {"partition": 3})


@pytest.mark.parametrize("partition", [1, 2])
@pytest.mark.parametrize("K", [5, 24])
@pytest.mark.parametrize("spt", [8, 32])
def test_nfa_lazy_and_chained_partitioning(pf, partition, K, spt):
    """Sec. III.D.2 for NFAs on instances that never die. Chained: a live
    instance leaves its tile as (start, position, state set), inline for a
    core of 5 states (sets of at most 8 held by one lane), in the carry pool
    for a core of 24 (sets run by the whole warp), and the carry kernel
    continues it; lazy: it continues in place on the global text."""
    m = W.live_core_nfa(K, 7)
    a = pf.load(m)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "spt": spt, "partition": partition})
    t = W.text_uniform(6000, 4, 11)
    want = oracle.scan(m, t)
    assert len(want) > 200_000
    assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 16), want)


@pytest.mark.parametrize("K", [5, 24])
def test_nfa_chained_partitioning_with_a_full_carry_queue(pf, K):
    """A carry queue of 100 entries and a pool of 64 states: the instances
    that find no room (entries or pool) continue in place, and the match set
    is unchanged."""
    m = W.live_core_nfa(K, 8)
    a = pf.load(m)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "partition": 2})
    t = W.text_uniform(9000, 4, 12)
    want = oracle.scan(m, t)
    P.pfsm_test_carry_cap(pf.ctx, 100, 64)
    try:
        got = gpu_matches(pf, a, t, cap=len(want) + 16)
    finally:
        P.pfsm_test_carry_cap(pf.ctx, 0, 0)
    assert np.array_equal(got, want)


def test_nfa_chained_partitioning_with_bitsets_in_global_memory(pf):
    """The live core of 24 states padded with unreachable states to Q =
    12,288: the warp-wide bitsets (2 x 384 words per warp) no longer fit the
    tile kernel's shared memory, so they and the carry kernel's live in a
    global scratch sized for both kernels' warps; a short text (few tile-kernel
    CTAs, a full grid of carry CTAs) against the oracle."""
    core = W.live_core_nfa(24, 9)
    Q = 12_288
    bits = np.zeros((Q, core.S, Q // 32), dtype=np.uint32)
    bits[:core.Q, :, :core.bits.shape[2]] = core.bits
    fin = np.zeros(Q, dtype=np.uint8)
    fin[:core.Q] = core.final
    m = W.Nfa(bits=bits, q0=core.q0, final=fin)
    a = pf.load(m)
    P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "partition": 2})
    t = W.text_uniform(6000, 4, 13)
    want = oracle.scan(core, t)
    assert len(want) > 100_000
    assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 16), want)
    P.pfsm_unload(pf.ctx, a)


def test_nfa_chained_partitioning_on_cyclic_sets(pf):
    """Random cyclic NFAs (sets grow and shrink; seeds picked so that
    thousands of matches come from instances that crossed the first tile's
    end) chained against the oracle, one of them following epsilon edges at
    run time."""
    for seed in (102, 109, 110, 126):
        rng = np.random.default_rng(seed)
        Q, S = 12 + (seed % 4) * 4, 4
        edges = [(q, x, u) for q in range(Q) for x in range(S) for u in range(Q)
                 if rng.random() < 0.06]
        eps = [(q, u) for q in range(Q) for u in range(Q) if q != u and rng.random() < 0.03]
        with_eps = seed % 2 == 1
        m = W.nfa_from_edges(Q, S, 0, edges, [3], eps_edges=eps if with_eps else ())
        a = pf.load(m)
        P.pfsm_set_params(pf.ctx, a, {"tile": 4096, "halo": 16, "partition": 2})
        t = W.text_uniform(4800, 4, seed)
        want = oracle.scan(W.eps_free(m) if with_eps else m, t)
        assert ((want[:, 0] < 4096) & (want[:, 1] >= 4112)).sum() > 2000, seed
        assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 16), want), seed
        P.pfsm_unload(pf.ctx, a)


def test_eviction_and_reload(pf):
    autos = [W.dfa_random(50 + i, Q=64, S=4) for i in range(3)]
    autos.append(W.workload_motif_nfa(3, n=10, n_motifs=40)[0])
    sizes = []
    for x in autos:
        before = P.pfsm_get_stats(pf.ctx)["resident_bytes"]
        a = pf.load(x)
        sizes.append(P.pfsm_get_stats(pf.ctx)["resident_bytes"] - before)
        P.pfsm_unload(pf.ctx, a)
    budget = max(sizes) + min(sizes)      # never room for all of them
    assert budget < sum(sizes)
    small = P.Pfsm(0, budget_bytes=budget)
    try:
        ids = [small.load(x) for x in autos]
        t = W.text_uniform(60_000, 4, 5)
        for rnd in range(2):
            for x, i in zip(autos, ids):
                assert np.array_equal(gpu_matches(small, i, t), oracle.scan(x, t))
        st = P.pfsm_get_stats(small.ctx)
        assert st["evictions"] > 0 and st["reloads"] > 0
        assert st["resident_bytes"] <= budget
        P.pfsm_evict(small.ctx, ids[0])
        assert np.array_equal(gpu_matches(small, ids[0], t), oracle.scan(autos[0], t))
        P.pfsm_unload(small.ctx, ids[1])
        with pytest.raises(P.PfsmError):
            P.pfsm_scan(small.ctx, ids[1], small.to_device(t), None, None, 0)
    finally:
        small.close()


def test_eviction_orders_after_scans_in_flight_on_other_streams(pf):
    """Room for one machine only: every scan evicts the other machine, whose
    scan may still be running on the other stream. The eviction is ordered
    after that scan (its use event) and the reload after the eviction, all
    without a host synchronisation; both match sets stay exact."""
    motifs = W.motif_set(61, n_motifs=64)
    nfa = W.motif_nfa(motifs)[0]
    dfa = W.dfa_random(62, Q=64, S=4)
    t_n = W.text_dna(400_000, 63)
    W.plant_motifs(t_n, motifs, 2_000, 64)
    t_d = W.text_uniform(150_000, 4, 65)
    want_n, want_d = oracle.scan(nfa, t_n), oracle.scan(dfa, t_d)
    probe = P.Pfsm(0)
    try:
        sizes = [P.pfsm_aut_bytes(probe.ctx, probe.load(x))[0] for x in (nfa, dfa)]
    finally:
        probe.close()
    small = P.Pfsm(0, budget_bytes=max(sizes) + 256)
    try:
        ids = [small.load(nfa), small.load(dfa)]
        assert P.pfsm_aut_bytes(small.ctx, ids[0]) == (sizes[0], False)   # evicted by the second load
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        tn, td = small.to_device(t_n), small.to_device(t_d)
        outs = [torch.empty((len(want_n) + 64, 3), dtype=torch.int32, device="cuda") for _ in range(3)]
        outd = [torch.empty((len(want_d) + 64, 3), dtype=torch.int32, device="cuda") for _ in range(3)]
        sts = torch.zeros((6, 2), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        for r in range(3):
            P.pfsm_scan_async(small.ctx, ids[0], tn, None, outs[r], sts[2 * r], stream=s1)
            P.pfsm_scan_async(small.ctx, ids[1], td, None, outd[r], sts[2 * r + 1], stream=s2)
        torch.cuda.synchronize()
        st = sts.cpu().numpy()
        for r in range(3):
            assert st[2 * r, 1] == 0 and st[2 * r + 1, 1] == 0
            got_n = oracle.sort_matches(outs[r][:st[2 * r, 0]].cpu().numpy().view(np.uint32))
            got_d = oracle.sort_matches(outd[r][:st[2 * r + 1, 0]].cpu().numpy().view(np.uint32))
            assert np.array_equal(got_n, want_n), r
            assert np.array_equal(got_d, want_d), r
        stats = P.pfsm_get_stats(small.ctx)
        assert stats["evictions"] >= 5 and stats["reloads"] >= 5
        assert stats["resident_bytes"] <= max(sizes) + 256
    finally:
        small.close()


def test_async_status_and_stream(pf):
    d, t = W.workload_dna_dfa(2, n=200_000)
    a = pf.load(d)
    want = oracle.scan(d, t)
    s = torch.cuda.Stream()
    tt = pf.to_device(t)
    out = torch.empty((len(want) + 5, 3), dtype=torch.int32, device="cuda")
    status = torch.zeros(2, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        P.pfsm_scan_async(pf.ctx, a, tt, None, out, status, stream=s)
    s.synchronize()
    cnt, err = status.tolist()
    assert err == 0 and cnt == len(want)
    assert np.array_equal(oracle.sort_matches(out[:cnt].cpu().numpy().view(np.uint32)), want)


# ---------------------------------------------------------------- second-level prefix records
def twin_chain_nfa(seed, H=100, L=16, p_die=0.08, p_fin=0.04):
    """Two independent chains run side by side from q0: chain c has states
    (c, d, h) for depth d = 1..L and hash h < H, and symbol a moves (c, d, h)
    to (c, d + 1, f_c(d, h, a)) or nowhere (probability p_die). The state set
    after d symbols holds at most one state per chain, so the sets met after
    8 symbols are pairs of hashes: about H^2 of them, more than the 4096 sets
    that get second-level tables. Finals are scattered over depths 9..L.
    Returns the machine and the set of (h1, h2) pairs met after 8 symbols by
    starts that have met no final state (counted by direct simulation)."""
    rng = np.random.default_rng(seed)
    S = 4
    Q = 1 + 2 * L * H
    sid = lambda c, d, h: 1 + (c * L + (d - 1)) * H + h
    f = rng.integers(0, H, size=(2, L + 1, H, S))
    die = rng.random((2, L + 1, H, S)) < p_die
    edges = []
    for c in range(2):
        for a in range(S):
            h0 = int(f[c, 0, 0, a])
            if not die[c, 0, 0, a]:
                edges.append((0, a, sid(c, 1, h0)))
            for d in range(1, L):
                for h in range(H):
                    if not die[c, d, h, a]:
                        edges.append((sid(c, d, h), a, sid(c, d + 1, int(f[c, d, h, a]))))
    fins = [sid(c, d, h) for c in range(2) for d in range(9, L + 1) for h in range(H)
            if rng.random() < p_fin]
    m = W.nfa_from_edges(Q, S, 0, edges, fins)
    # the sets after 8 symbols, over every 8-gram (no final before depth 9)
    grams = np.arange(1 << 16)
    hs, alive = [], []
    for c in range(2):
        h = np.zeros(len(grams), dtype=np.int64)
        ok = np.ones(len(grams), dtype=bool)
        for d in range(8):
            a = (grams >> (2 * d)) & 3
            ok &= ~die[c, d, h if d else 0, a]
            h = f[c, d, h if d else 0, a]
        hs.append(np.where(ok, h, -1))
    pairs = {(int(x), int(y)) for x, y in zip(hs[0], hs[1]) if x >= 0 or y >= 0}
    return m, pairs


def test_second_level_records_beyond_the_table_cap(pf):
    """More survivor sets after k = 8 symbols than get second-level tables:
    starts on the first 4096 sets take the second level (empty entries
    dismiss them, others settle from k + 5 symbols or take the exact path),
    the rest settle from k symbols. Every start must still report exactly
    the oracle's matches, near text ends too."""
    m, pairs = twin_chain_nfa(7)
    assert len(pairs) > 4096
    a = pf.load(m)
    for n, seed in ((200_000, 1), (16_399, 2), (13, 3), (9, 4)):
        t = W.text_uniform(n, 4, 900 + seed)
        want = oracle.scan(m, t)
        if n > 1000:
            assert len(want) > 100
        assert np.array_equal(gpu_matches(pf, a, t, cap=len(want) + 8), want), n
    for k in (3, 7):
        P.pfsm_set_params(pf.ctx, a, {"prefix_k": k})
        t = W.text_uniform(50_000, 4, 950 + k)
        assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(m, t)), k


# ---------------------------------------------------------------- bounded waits
def test_bounded_waits_end_a_held_scan_with_timeout(pf):
    """Every wait of the scan kernel is bounded: with the producer warp
    handing no tile over (a test hook; nothing faults and nothing spins
    without a limit), the filtering warps' waits run out, the scan reports
    E_TIMEOUT within seconds, and the next scan on the same context is
    exact."""
    import time
    nfa, t, _, _ = W.workload_motif_nfa(2, n=8 << 20, n_motifs=32)
    a = pf.load(nfa)
    P.pfsm_set_params(pf.ctx, a, {"spt": 32})   # tiles staged by a producer warp
    P.pfsm_test_hold_tiles(pf.ctx, True)
    try:
        t0 = time.time()
        with pytest.raises(P.PfsmError) as err:
            gpu_matches(pf, a, t)
        assert err.value.status == P.PFSM_E_TIMEOUT
        assert time.time() - t0 < 30
    finally:
        P.pfsm_test_hold_tiles(pf.ctx, False)
    assert np.array_equal(gpu_matches(pf, a, t), oracle.scan(nfa, t))
