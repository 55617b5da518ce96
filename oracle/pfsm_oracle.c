/*
 * Plain CPU oracle for the PFSM scan. TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the benchmark's CPU-baseline leg call it; the CUDA
 * library never does, and the two share no code.
 *
 * What it computes (Sec. III.A-B of Quesada, Berzal, Cortijo, "Treating
 * Insomnia, Amnesia, and Acalculia in Regular Expression Matching"):
 *
 *   M(t, A) = { (i, j, f) : 0 <= i <= j < n, f in F, f in delta^({q0}, t[i..j]) }
 *
 * It reaches M by the paper's own per-symbol procedure (Sec. III.B), not by a
 * shortcut. Each state carries a set of tags; a tag is the input position at
 * which the instance holding it was started. For every position j:
 *
 *   step 1  reinitialise: q0 is activated and tagged with j; states that are
 *           already active stay active with their tags;
 *   step 2  epsilon transitions: none, since automata are epsilon-free here;
 *           they are removed when the machine is built;
 *   step 3  consume t[j]: from each active state q take the transitions that
 *           match t[j];
 *   step 4  apply them: every target q' in delta(q, t[j]) receives all tags of
 *           q (tag sets are unioned, so one start reaching q' along two paths
 *           is one instance);
 *   report  for every final target f and every tag i on it, (i, j, f) is a
 *           match: start = tag, end = current position (Sec. III.B, last
 *           paragraph), and the state stands in for its label (l: F -> L is
 *           applied by the caller).
 *
 * An instance that enters the DFA's dead state is dropped (the dead state is
 * absorbing and non-final, so this does not change M); an NFA instance whose
 * set is empty has no tags left anywhere and disappears by itself.
 *
 * Lazy data partitioning (Sec. III.D.2): reinitialisation is limited to
 * positions in [reinit_lo, reinit_hi), and processing goes on past reinit_hi
 * until the text ends or no state is active. That yields exactly the matches
 * whose start lies in [reinit_lo, reinit_hi).
 *
 * Chained data partitioning (Sec. III.D.2): a run may start from a given set
 * of tagged active states and hand back the tagged active states left at its
 * end, so a segment's survivors can be continued on the next segment.
 *
 * Work (Sec. III.B): each position advances every (tag, state) pair active
 * after step 1 over one symbol; the number of such pair-steps, summed over
 * the positions, is the work of the procedure (a DFA instance is one pair;
 * an NFA instance is one pair per state of its set).
 *
 * Data structures are deliberately naive: one sorted, duplicate-free array of
 * tags per state, and a list of the active states. Transitions are read from
 * per-(state, symbol) successor lists built once from the caller's table (for
 * the NFA form, the bits of each delta row; for the DFA form, the one entry).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t *v;
    uint32_t n, cap;
} tagset;

typedef struct {
    int Q, S, q0, dead;
    uint32_t *off;      /* [Q*S + 1] start of the successors of (q, a) */
    int32_t *succ;      /* successor states */
    const uint8_t *fin; /* [Q] */
} machine;

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

static int ts_reserve(tagset *t, uint32_t need) {
    if (need <= t->cap) return 0;
    uint32_t c = t->cap ? t->cap : 4;
    while (c < need) c *= 2;
    uint32_t *nv = (uint32_t *)realloc(t->v, (size_t)c * sizeof(uint32_t));
    if (!nv) return -1;
    t->v = nv;
    t->cap = c;
    return 0;
}

/* dst := dst U src, both sorted ascending without duplicates */
static int ts_union(tagset *dst, const tagset *src, uint32_t **scratch, uint32_t *scap) {
    uint32_t need = dst->n + src->n;
    if (need > *scap) {
        uint32_t c = *scap ? *scap : 64;
        while (c < need) c *= 2;
        uint32_t *ns = (uint32_t *)realloc(*scratch, (size_t)c * sizeof(uint32_t));
        if (!ns) return -1;
        *scratch = ns;
        *scap = c;
    }
    uint32_t a = 0, b = 0, k = 0;
    uint32_t *o = *scratch;
    while (a < dst->n && b < src->n) {
        uint32_t x = dst->v[a], y = src->v[b];
        if (x < y) { o[k++] = x; a++; }
        else if (y < x) { o[k++] = y; b++; }
        else { o[k++] = x; a++; b++; }
    }
    while (a < dst->n) o[k++] = dst->v[a++];
    while (b < src->n) o[k++] = src->v[b++];
    if (ts_reserve(dst, k)) return -1;
    memcpy(dst->v, o, (size_t)k * sizeof(uint32_t));
    dst->n = k;
    return 0;
}

/*
 * The per-symbol procedure over text positions [j_begin, j_end).
 *   in_pairs   n_in (tag, state) pairs active before position j_begin
 *   out        up to cap matches as (start, end, state) triples
 *   out_active if not NULL, receives up to active_cap (tag, state) pairs left
 *              active after the last processed position; *n_active gets the
 *              full number
 *   pair_steps if not NULL, gets the number of (tag, state) pairs advanced
 *              over a symbol, summed over the processed positions
 * Returns the number of matches (which may exceed cap), or -1 on error with
 * *err set (OR_EINVAL: a symbol >= S; OR_ENOMEM).
 */
static int64_t run(const machine *m, const uint8_t *text, uint64_t j_begin, uint64_t j_end,
                   uint64_t reinit_lo, uint64_t reinit_hi, const uint32_t *in_pairs,
                   uint64_t n_in, uint32_t *out, int64_t cap, uint32_t *out_active,
                   int64_t active_cap, int64_t *n_active, uint64_t *pair_steps, int *err) {
    int Q = m->Q;
    tagset *cur = (tagset *)calloc((size_t)Q, sizeof(tagset));
    tagset *nxt = (tagset *)calloc((size_t)Q, sizeof(tagset));
    int32_t *act = (int32_t *)malloc((size_t)Q * sizeof(int32_t));
    int32_t *act2 = (int32_t *)malloc((size_t)Q * sizeof(int32_t));
    uint32_t *scratch = NULL, scap = 0;
    int64_t count = 0;
    uint64_t work = 0;
    int na = 0;
    *err = OR_OK;
    if (!cur || !nxt || !act || !act2) { *err = OR_ENOMEM; count = -1; goto done; }

    /* tagged states handed over from a previous segment (chained partitioning) */
    for (uint64_t k = 0; k < n_in; k++) {
        uint32_t tag = in_pairs[2 * k], q = in_pairs[2 * k + 1];
        if ((int)q >= Q) { *err = OR_EINVAL; count = -1; goto done; }
        if (cur[q].n == 0) act[na++] = (int32_t)q;
        tagset one = {&tag, 1, 1};
        if (ts_union(&cur[q], &one, &scratch, &scap)) { *err = OR_ENOMEM; count = -1; goto done; }
    }

    for (uint64_t j = j_begin; j < j_end; j++) {
        /* step 1: reinitialise */
        if (j >= reinit_lo && j < reinit_hi) {
            tagset *t0 = &cur[m->q0];
            if (t0->n == 0) act[na++] = m->q0;
            uint32_t tag = (uint32_t)j;
            tagset one = {&tag, 1, 1};
            if (ts_union(t0, &one, &scratch, &scap)) { *err = OR_ENOMEM; count = -1; goto done; }
        }
        if (na == 0) {
            if (j >= reinit_hi) break; /* nothing active and no more starts */
            continue;
        }
        /* step 2: no epsilon transitions in this form */
        uint32_t a = text[j];
        if ((int)a >= m->S) { *err = OR_EINVAL; count = -1; goto done; }
        /* steps 3 and 4: traverse the transitions that match t[j] and tag the targets */
        int nb = 0;
        for (int k = 0; k < na; k++) {
            int q = act[k];
            work += cur[q].n; /* every tag on q is advanced over t[j] */
            uint32_t lo = m->off[(size_t)q * m->S + a], hi = m->off[(size_t)q * m->S + a + 1];
            for (uint32_t e = lo; e < hi; e++) {
                int t = m->succ[e];
                if (t == m->dead) continue; /* instance dropped */
                if (nxt[t].n == 0) act2[nb++] = t;
                if (ts_union(&nxt[t], &cur[q], &scratch, &scap)) {
                    *err = OR_ENOMEM; count = -1; goto done;
                }
            }
            cur[q].n = 0;
        }
        /* report: a final target with tag i is the match (i, j, target) */
        for (int k = 0; k < nb; k++) {
            int t = act2[k];
            if (!m->fin[t]) continue;
            for (uint32_t x = 0; x < nxt[t].n; x++) {
                if (count < cap) {
                    out[3 * count + 0] = nxt[t].v[x];
                    out[3 * count + 1] = (uint32_t)j;
                    out[3 * count + 2] = (uint32_t)t;
                }
                count++;
            }
        }
        /* the targets are the active states for the next symbol */
        tagset *sw = cur; cur = nxt; nxt = sw;
        int32_t *sa = act; act = act2; act2 = sa;
        na = nb;
    }

    if (n_active) {
        int64_t k = 0;
        for (int x = 0; x < na; x++) {
            int q = act[x];
            for (uint32_t y = 0; y < cur[q].n; y++) {
                if (out_active && k < active_cap) {
                    out_active[2 * k] = cur[q].v[y];
                    out_active[2 * k + 1] = (uint32_t)q;
                }
                k++;
            }
        }
        *n_active = k;
    }

done:
    if (pair_steps) *pair_steps = work;
    if (cur) for (int q = 0; q < Q; q++) free(cur[q].v);
    if (nxt) for (int q = 0; q < Q; q++) free(nxt[q].v);
    free(cur); free(nxt); free(act); free(act2); free(scratch);
    return count;
}

static int machine_from_dfa(machine *m, const int16_t *delta, int Q, int S, int q0, int dead,
                            const uint8_t *fin) {
    m->Q = Q; m->S = S; m->q0 = q0; m->dead = dead; m->fin = fin;
    m->off = (uint32_t *)malloc(((size_t)Q * S + 1) * sizeof(uint32_t));
    m->succ = (int32_t *)malloc((size_t)Q * S * sizeof(int32_t));
    if (!m->off || !m->succ) return -1;
    uint32_t e = 0;
    for (size_t k = 0; k < (size_t)Q * S; k++) {
        m->off[k] = e;
        int t = delta[k];
        if (t < 0 || t >= Q) continue; /* no transition */
        m->succ[e++] = t;
    }
    m->off[(size_t)Q * S] = e;
    return 0;
}

static int machine_from_nfa(machine *m, const uint32_t *bits, int Q, int S, int q0,
                            const uint8_t *fin) {
    int W = (Q + 31) / 32;
    m->Q = Q; m->S = S; m->q0 = q0; m->dead = -1; m->fin = fin;
    size_t total = 0;
    for (size_t k = 0; k < (size_t)Q * S * W; k++) total += (size_t)__builtin_popcount(bits[k]);
    m->off = (uint32_t *)malloc(((size_t)Q * S + 1) * sizeof(uint32_t));
    m->succ = (int32_t *)malloc((total + 1) * sizeof(int32_t));
    if (!m->off || !m->succ) return -1;
    uint32_t e = 0;
    for (size_t k = 0; k < (size_t)Q * S; k++) {
        m->off[k] = e;
        const uint32_t *row = bits + k * W;
        for (int w = 0; w < W; w++)
            for (int b = 0; b < 32; b++)
                if (row[w] >> b & 1u) m->succ[e++] = w * 32 + b;
    }
    m->off[(size_t)Q * S] = e;
    return 0;
}

static void machine_free(machine *m) {
    free(m->off);
    free(m->succ);
}

/* ---------------------------------------------------------------- exports */

/* DFA form: delta int16 [Q][S] row-major; dead = -1 for none. Runs positions
 * [s_lo, n), reinitialising on [s_lo, s_hi): the matches starting in
 * [s_lo, s_hi). */
int64_t oracle_scan_dfa(const int16_t *delta, int Q, int S, int q0, int dead, const uint8_t *fin,
                        const uint8_t *text, uint64_t n, uint64_t s_lo, uint64_t s_hi,
                        uint32_t *out, int64_t cap, int *err) {
    machine m;
    if (machine_from_dfa(&m, delta, Q, S, q0, dead, fin)) { machine_free(&m); *err = OR_ENOMEM; return -1; }
    int64_t r = run(&m, text, s_lo, n, s_lo, s_hi, NULL, 0, out, cap, NULL, 0, NULL, NULL, err);
    machine_free(&m);
    return r;
}

/* NFA form: bits uint32 [Q][S][ceil(Q/32)]. Same positions as above. */
int64_t oracle_scan_nfa(const uint32_t *bits, int Q, int S, int q0, const uint8_t *fin,
                        const uint8_t *text, uint64_t n, uint64_t s_lo, uint64_t s_hi,
                        uint32_t *out, int64_t cap, int *err) {
    machine m;
    if (machine_from_nfa(&m, bits, Q, S, q0, fin)) { machine_free(&m); *err = OR_ENOMEM; return -1; }
    int64_t r = run(&m, text, s_lo, n, s_lo, s_hi, NULL, 0, out, cap, NULL, 0, NULL, NULL, err);
    machine_free(&m);
    return r;
}

/* One segment of chained data partitioning, either table form (bits == NULL
 * selects the DFA form): positions [j_begin, j_end), reinitialising on
 * [reinit_lo, reinit_hi), starting from the n_in tagged states in_pairs and
 * handing back the tagged states active at the end. */
int64_t oracle_run_segment(const int16_t *delta, const uint32_t *bits, int Q, int S, int q0,
                           int dead, const uint8_t *fin, const uint8_t *text, uint64_t j_begin,
                           uint64_t j_end, uint64_t reinit_lo, uint64_t reinit_hi,
                           const uint32_t *in_pairs, uint64_t n_in, uint32_t *out, int64_t cap,
                           uint32_t *out_active, int64_t active_cap, int64_t *n_active, int *err) {
    machine m;
    int bad = bits ? machine_from_nfa(&m, bits, Q, S, q0, fin)
                   : machine_from_dfa(&m, delta, Q, S, q0, dead, fin);
    if (bad) { machine_free(&m); *err = OR_ENOMEM; return -1; }
    int64_t r = run(&m, text, j_begin, j_end, reinit_lo, reinit_hi, in_pairs, n_in, out, cap,
                    out_active, active_cap, n_active, NULL, err);
    machine_free(&m);
    return r;
}

/* The work of the scan of either table form (bits == NULL selects the DFA
 * form) for the starts in [s_lo, s_hi): *pair_steps gets the number of
 * (tag, state) pairs advanced over a symbol. The matches are counted, not
 * stored; the count is returned (or -1 with *err set). */
int64_t oracle_pair_steps(const int16_t *delta, const uint32_t *bits, int Q, int S, int q0,
                          int dead, const uint8_t *fin, const uint8_t *text, uint64_t n,
                          uint64_t s_lo, uint64_t s_hi, uint64_t *pair_steps, int *err) {
    machine m;
    int bad = bits ? machine_from_nfa(&m, bits, Q, S, q0, fin)
                   : machine_from_dfa(&m, delta, Q, S, q0, dead, fin);
    if (bad) { machine_free(&m); *err = OR_ENOMEM; return -1; }
    int64_t r = run(&m, text, s_lo, n, s_lo, s_hi, NULL, 0, NULL, 0, NULL, 0, NULL, pair_steps,
                    err);
    machine_free(&m);
    return r;
}
