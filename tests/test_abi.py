"""The C ABI library builds, loads, and exports every function that
include/pfsm.h declares (CPU only: no call here touches a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pfsm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(pfsm_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1110_1716_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pfsm_load_dfa", "pfsm_load_nfa", "pfsm_scan", "pfsm_scan_batch", "pfsm_evict"):
        assert must in names


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_1110_1716_gb300 as P
    for name in declared_functions():
        assert name in P.EXPORTS and callable(getattr(P, name)), name


def test_strerror_covers_status_codes(lib):
    lib.pfsm_strerror.restype = ctypes.c_char_p
    texts = {lib.pfsm_strerror(i).decode() for i in range(7)}
    assert len(texts) == 7
    assert lib.pfsm_strerror(99).decode() == "unknown status"


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument checks happen before any CUDA call
    assert lib.pfsm_ctx_create(0, 0, None) == 1
    assert lib.pfsm_load_dfa(None, None, 0, 0, 0, 0, None, None) == 1
    assert lib.pfsm_scan(None, 0, None, 0, None, 0, None, None) == 1
    assert lib.pfsm_ctx_destroy(None) == 0
