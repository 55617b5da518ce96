"""The pins are sharp: copies of the oracle with one plausible mistake
planted each (compiled here, on the CPU) must fail at least one pin."""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "pfsm_oracle.c")

MUTANTS = {
    # step 1 forgets the new tag when q0 already holds one (reading A6)
    "reinit_drops_new_tag": ("uint32_t tag = (uint32_t)j;",
                             "uint32_t tag = (uint32_t)(t0->n ? t0->v[0] : j);"),
    # end index off by one (exclusive instead of inclusive end)
    "end_off_by_one": ("out[3 * count + 1] = (uint32_t)j;",
                       "out[3 * count + 1] = (uint32_t)(j + 1);"),
    # delta read transposed: delta[a][q] instead of delta[q][a]
    "delta_transposed": ("int t = delta[k];", "int t = delta[(k % S) * Q + k / S];"),
    # tags of a target overwritten instead of unioned (step 4)
    "tags_overwritten": ("if (ts_union(&nxt[t], &cur[q], &scratch, &scap)) {",
                         "if ((nxt[t].n = 0, ts_union(&nxt[t], &cur[q], &scratch, &scap))) {"),
    # reinitialisation range starts one late (a dropped start)
    "reinit_range": ("if (j >= reinit_lo && j < reinit_hi) {",
                     "if (j > reinit_lo && j < reinit_hi) {"),
    # report rule tests the source state instead of the target
    "report_source": ("if (!m->fin[t]) continue;", "if (!m->fin[t] || !m->fin[act[0]]) continue;"),
    # successor row read for the wrong symbol (previous one)
    # the work count takes one per active state instead of one per (tag, state) pair
    "work_counts_states": ("work += cur[q].n;", "work += 1;"),
    # the work count misses the pairs of the first active state
    "work_skips_first": ("work += cur[q].n;", "work += k ? cur[q].n : 0;"),
    "symbol_index": ("uint32_t lo = m->off[(size_t)q * m->S + a], hi = m->off[(size_t)q * m->S + a + 1];",
                     "uint32_t a2 = j ? text[j - 1] : a; uint32_t lo = m->off[(size_t)q * m->S + a2], "
                     "hi = m->off[(size_t)q * m->S + a2 + 1];"),
}


def battery():
    """Returns the names of the pins that fail."""
    failed = []
    m = W.eps_free(W.fig1_union())
    for fx in ("fig2_aacacab.txt", "fig3_ac.txt"):
        text, want = read_golden(fx)
        try:
            got = oracle.labelled(oracle.scan(m, W.encode(text, W.FIG1_ALPHABET)), m.labels)
        except Exception:
            got = None
        if got != want:
            failed.append(fx)
    rng = np.random.default_rng(1)
    for seed in range(3):
        d = W.dfa_random(100 + seed, Q=9, S=4)
        for n in (3, 8, 40):
            t = rng.integers(0, 4, size=n, dtype=np.uint8)
            try:
                ok = np.array_equal(oracle.scan(d, t), oracle.brute_force(d, t))
            except Exception:
                ok = False
            if not ok:
                failed.append("brute_dfa")
                break
    sigs = [b"\x00\x01\x02", b"\x01\x02", b"\x03\x03\x00\x01"]
    d, fo = W.trie_dfa(sigs, S=4)
    t = W.text_uniform(400, 4, 3)
    try:
        ok = np.array_equal(oracle.scan(d, t), oracle.literal_occurrences(sigs, fo, t))
    except Exception:
        ok = False
    if not ok:
        failed.append("literal")
    # the work count against its closed form and its definition
    try:
        full = W.dfa_random(5, Q=7, S=3, dead=-1, finals=[1, 2], p_dead=0.0)
        t3 = W.text_uniform(50, 3, 2)
        ok = oracle.pair_steps(full, t3)[0] == 50 * 51 // 2
        nfa = W.nfa_from_edges(4, 2, 0, [(0, 0, 1), (0, 0, 2), (1, 1, 3), (2, 1, 0), (3, 0, 3)], [3])
        t2 = W.text_uniform(60, 2, 4)
        ok = ok and oracle.pair_steps(nfa, t2)[0] == oracle.brute_force_pair_steps(nfa, t2)
    except Exception:
        ok = False
    if not ok:
        failed.append("pair_steps")
    return failed


def test_unmutated_oracle_passes_battery():
    assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("m_%s.c" % name)
    path.write_text(src.replace(old, new))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", str(path), "-o", str(so)])
    with oracle.using_library(str(so)):
        failed = battery()
    assert failed, "mutant %s passed every pin" % name
