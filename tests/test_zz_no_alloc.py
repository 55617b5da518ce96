"""The allocation-free DFA scan, for callers that cannot allocate device
memory: a plugin that is only handed buffers, a process whose device memory
belongs to another allocator, a loop that must never stall on cudaMalloc or
cudaFree. It works on the buffers the caller passes plus one fixed array
inside the library. These tests check, on two calls in a row, that it gives
the oracle's match set and the same set as the regular scan, including a
machine without a dead state whose instances overflow the array's carry
region, an unaligned text and the error paths. This file is collected last so
that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_1716_gb300 as P  # noqa: E402


def noalloc_scan(lib, d, text_dev, cap, delta=None):
    """One call through the C ABI; returns (matches as uint32 rows, count,
    error bits)."""
    dev = torch.device("cuda", 0)
    tab = d.delta if delta is None else delta
    delta_t = torch.from_numpy(np.ascontiguousarray(tab, dtype=np.int16)).to(dev)
    fin = torch.from_numpy(np.ascontiguousarray(d.final, dtype=np.uint8)).to(dev)
    out = torch.empty((max(1, cap), 3), dtype=torch.int32, device=dev)
    status = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    Q, S = tab.shape
    st = lib.pfsm_scan_dfa_noalloc(
        ctypes.c_void_p(delta_t.data_ptr()), Q, S, d.q0, d.dead, ctypes.c_void_p(fin.data_ptr()),
        ctypes.c_void_p(text_dev.data_ptr()), text_dev.numel(), ctypes.c_void_p(out.data_ptr()),
        cap, ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == P.PFSM_OK, P.strerror(st)
    stream.synchronize()
    cnt, err = status.tolist()
    rows = out[:min(cnt, cap)].cpu().numpy().view(np.uint32)
    return oracle.sort_matches(rows), cnt, err


def no_dead_state_dfa():
    """Every instance lives to the end of the text (no dead state), but each
    reports at most once: A -> final 1; another symbol then C -> final 4;
    everything else falls into state 3, absorbing and not final."""
    Q, S = 5, 4
    delta = np.full((Q, S), 3, dtype=np.int16)
    delta[0, :] = 2
    delta[0, 0] = 1          # A
    delta[2, 1] = 4          # C after a non-A first symbol
    fin = np.zeros(Q, dtype=np.uint8)
    fin[[1, 4]] = 1
    return W.Dfa(delta=delta, q0=0, dead=-1, final=fin)


def windows_oracle(d, t, windows):
    return oracle.sort_matches(np.concatenate([oracle.scan(d, t, lo, hi) for lo, hi in windows]))


def in_windows(m, windows):
    keep = np.zeros(len(m), dtype=bool)
    for lo, hi in windows:
        keep |= (m[:, 0] >= lo) & (m[:, 0] < hi)
    return m[keep]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("which", ["dna_dfa", "byte_trie"])
def test_noalloc_equals_oracle_and_regular_scan_twice(which):
    need_gpu()
    lib = P.load_library()
    if which == "dna_dfa":
        d, t = W.workload_dna_dfa(1, n=1 << 20)
    else:
        sigs = W.signature_set(4, n_sigs=60)   # 1212 states x 256: a 620 KB table
        d, _ = W.trie_dfa(sigs)
        t = W.text_uniform(3 << 20, 256, 5)
        W.plant_signatures(t, sigs, 4096, 6)
    want = oracle.scan(d, t)
    with P.Pfsm(0) as pf:
        tdev = pf.to_device(t)
        regular = oracle.sort_matches(pf.scan_numpy(pf.load(d), tdev))
        assert np.array_equal(regular, want)
        for call in range(2):
            got, cnt, err = noalloc_scan(lib, d, tdev, len(want) + 64)
            assert err == 0 and cnt == len(want), call
            assert np.array_equal(got, want), call


def test_noalloc_unaligned_text():
    need_gpu()
    lib = P.load_library()
    d, t = W.workload_dna_dfa(2, n=300_001)
    with P.Pfsm(0) as pf:
        base = pf.to_device(np.concatenate([np.zeros(3, np.uint8), t]))
        tdev = base[3:]                      # 3 bytes past a 16-byte boundary
        want = oracle.scan(d, t)
        for call in range(2):
            got, cnt, err = noalloc_scan(lib, d, tdev, len(want) + 64)
            assert err == 0 and cnt == len(want), call
            assert np.array_equal(got, want), call


def test_noalloc_without_dead_state_overflows_its_carry_region():
    """Instances outlive their tiles, and there are more of them than the
    array's carry region holds (about 196k entries): the rest continue in
    place on the global text. Compared with the regular scan on every start
    and with the oracle on start windows (the whole oracle run is O(n^2))."""
    need_gpu()
    lib = P.load_library()
    d = no_dead_state_dfa()
    n = 256 << 10
    t = W.text_uniform(n, 4, 23)
    windows = [(0, 1500), (n // 2, n // 2 + 1500), (n - 1500, n)]
    want_w = windows_oracle(d, t, windows)
    with P.Pfsm(0) as pf:
        tdev = pf.to_device(t)
        regular = oracle.sort_matches(pf.scan_numpy(pf.load(d), tdev))
        assert np.array_equal(in_windows(regular, windows), want_w)
        for call in range(2):
            got, cnt, err = noalloc_scan(lib, d, tdev, len(regular) + 64)
            assert err == 0 and cnt == len(regular), call
            assert np.array_equal(got, regular), call
            assert np.array_equal(in_windows(got, windows), want_w), call


def test_noalloc_reports_bad_tables_and_symbols():
    need_gpu()
    lib = P.load_library()
    d, t = W.workload_dna_dfa(3, n=100_000)
    with P.Pfsm(0) as pf:
        tdev = pf.to_device(t)
        bad = d.delta.copy()
        bad[5, 2] = d.Q              # a target outside [0, Q)
        _, _, err = noalloc_scan(lib, d, tdev, 1 << 20, delta=bad)
        assert err & 1
        t2 = t.copy()
        t2[77_777] = 4               # a symbol >= S
        _, _, err = noalloc_scan(lib, d, pf.to_device(t2), 1 << 20)
        assert err & 1
        # the next good call is exact again
        want = oracle.scan(d, t)
        got, cnt, err = noalloc_scan(lib, d, tdev, len(want) + 64)
        assert err == 0 and np.array_equal(got, want)


def test_noalloc_second_call_takes_no_device_memory():
    need_gpu()
    lib = P.load_library()
    d, t = W.workload_dna_dfa(1, n=1 << 20)
    tdev = torch.from_numpy(t).cuda()
    dev = torch.device("cuda", 0)
    delta_t = torch.from_numpy(np.ascontiguousarray(d.delta, dtype=np.int16)).to(dev)
    fin = torch.from_numpy(np.ascontiguousarray(d.final, dtype=np.uint8)).to(dev)
    out = torch.empty((2 << 20, 3), dtype=torch.int32, device=dev)
    status = torch.zeros(2, dtype=torch.int64, device=dev)
    args = (ctypes.c_void_p(delta_t.data_ptr()), d.Q, d.S, d.q0, d.dead,
            ctypes.c_void_p(fin.data_ptr()), ctypes.c_void_p(tdev.data_ptr()), tdev.numel(),
            ctypes.c_void_p(out.data_ptr()), out.shape[0], ctypes.c_void_p(status.data_ptr()),
            None)
    assert lib.pfsm_scan_dfa_noalloc(*args) == P.PFSM_OK   # may load the library's module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert lib.pfsm_scan_dfa_noalloc(*args) == P.PFSM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(status[1].item()) == 0


def test_noalloc_rejects_tables_above_its_limit():
    need_gpu()
    lib = P.load_library()
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # Q * S = 4096 * 256 entries would need 2 MiB of encoded table
    st = lib.pfsm_scan_dfa_noalloc(p, 4096, 256, 0, -1, p, p, 0, p, 0, p, None)
    assert st == P.PFSM_E_INVAL
