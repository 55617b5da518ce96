"""The allocation-free DFA scan (for callers that cannot allocate device
memory: it works only on buffers they pass in plus a fixed array inside the
library) gives the same match set as the regular scan, on two calls in a
row. This file is collected last so that a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1110_1716_gb300 as P  # noqa: E402


def noalloc_scan(lib, d, text_dev, cap):
    dev = torch.device("cuda", 0)
    delta = torch.from_numpy(np.ascontiguousarray(d.delta, dtype=np.int16)).to(dev)
    fin = torch.from_numpy(np.ascontiguousarray(d.final, dtype=np.uint8)).to(dev)
    out = torch.empty((cap, 3), dtype=torch.int32, device=dev)
    status = torch.zeros(2, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    Q, S = d.delta.shape
    st = lib.pfsm_scan_dfa_noalloc(
        ctypes.c_void_p(delta.data_ptr()), Q, S, d.q0, d.dead, ctypes.c_void_p(fin.data_ptr()),
        ctypes.c_void_p(text_dev.data_ptr()), text_dev.numel(), ctypes.c_void_p(out.data_ptr()),
        cap, ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == P.PFSM_OK, P.strerror(st)
    stream.synchronize()
    cnt, err = status.tolist()
    return out, cnt, err


@pytest.mark.parametrize("which", ["dna_dfa", "byte_trie"])
def test_noalloc_matches_regular_scan_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = P.load_library()
    if which == "dna_dfa":
        d, t = W.workload_dna_dfa(1, n=1 << 20)
    else:
        sigs = W.signature_set(4, n_sigs=60)   # 1212 states x 256: a 620 KB table
        d, _ = W.trie_dfa(sigs)
        t = W.text_uniform(3 << 20, 256, 5)
        W.plant_signatures(t, sigs, 4096, 6)
    with P.Pfsm(0) as pf:
        tdev = pf.to_device(t)
        want = oracle.sort_matches(pf.scan_numpy(pf.load(d), tdev))
        for call in range(2):
            out, cnt, err = noalloc_scan(lib, d, tdev, len(want) + 64)
            assert err == 0 and cnt == len(want), call
            got = oracle.sort_matches(out[:cnt].cpu().numpy().view(np.uint32))
            assert np.array_equal(got, want), call


def test_noalloc_rejects_tables_above_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = P.load_library()
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # Q * S = 4096 * 256 entries would need 2 MiB of encoded table
    st = lib.pfsm_scan_dfa_noalloc(p, 4096, 256, 0, -1, p, p, 0, p, 0, p, None)
    assert st == P.PFSM_E_INVAL
