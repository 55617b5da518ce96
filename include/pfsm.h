/*
 * pfsm.h - C ABI of the GB300 PFSM scan library (libpfsm.so).
 *
 * The operation (Sec. III.A-B of Quesada, Berzal, Cortijo, "Treating Insomnia,
 * Amnesia, and Acalculia in Regular Expression Matching"): a Parallel Finite
 * State Machine (Sigma, Q, q0, delta, F, L, l) is reinitialised at every input
 * symbol, so an instance starts at q0 at every position i and carries i as its
 * tag; every live instance advances on each symbol through delta; whenever a
 * transition lands on a final state f, (start = tag, end = current position,
 * f) is a match. The library reports the full set
 *
 *     M(t, A) = { (i, j, f) : 0 <= i <= j < n, f in F, f in delta^({q0}, t[i..j]) }
 *
 * with 0-based, inclusive ends (Fig. 2: "c" is reported at [2-2]). Empty
 * matches are not reported (tables are epsilon-free; a final q0 does not match
 * the empty string). Labels l: F -> L stay with the caller: results carry the
 * final state, which the caller maps to its label.
 *
 * Conventions for every call:
 *   - every function returns an int status, PFSM_OK (0) on success;
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     device memory of the context's device (for example torch tensors);
 *   - tables passed at load are copied; the caller may free them on return;
 *   - texts and outputs are caller-owned device memory; the library never
 *     frees them;
 *   - streams are the caller's (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream). Work is ordered on that stream;
 *   - a context may be used from one host thread at a time, except that scans
 *     on different streams may be issued from different threads;
 *   - state ids are 0..Q-1 with Q <= 32767; symbols are the bytes 0..S-1 with
 *     1 <= S <= 256; positions are 32-bit, so texts are shorter than 2^32.
 */
#ifndef PFSM_H
#define PFSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define PFSM_OK 0
#define PFSM_E_INVAL 1    /* bad argument, bad table, or a text symbol >= S */
#define PFSM_E_NOMEM 2    /* device memory or the residency budget exhausted */
#define PFSM_E_OVERFLOW 3 /* more matches than the output capacity */
#define PFSM_E_NOENT 4    /* unknown or unloaded automaton id */
#define PFSM_E_TIMEOUT 5  /* a bounded device wait expired: a warp waited 2 s
                             for a tile, a buffer or the other warps of its
                             CTA while none of them was running continuation
                             work (which always ends) */
#define PFSM_E_CUDA 6     /* a CUDA runtime call failed */
#define PFSM_E_CHECK 7    /* a device-side bounds check failed: only the checked
                             build (libpfsm_checked.so, compiled with
                             PFSM_CHECKED) tests indices; an async status then
                             has error bit 3 set */

typedef struct pfsm_ctx pfsm_ctx;
typedef int32_t pfsm_aut;

/* One match: the instance started at `start` reached final state `state`
 * after consuming t[start..end] (inclusive). */
typedef struct {
    uint32_t start, end, state;
} pfsm_match;

/* One match of a batch: as pfsm_match, for text number `text` of the batch. */
typedef struct {
    uint32_t text, start, end, state;
} pfsm_bmatch;

/* One job of a batch: scan `n` bytes at device address `text` with `aut`. */
typedef struct {
    pfsm_aut aut;
    uint32_t reserved; /* must be 0 */
    const uint8_t *text;
    uint64_t n;
} pfsm_job;

/* Tunable launch parameters of one automaton (0 = library default). */
typedef struct {
    int32_t prefix_k;   /* depth of the start-prefix table: the first k steps of
                           every instance are looked up once per k-gram;
                           -1 = off (every instance steps from q0); 0 = the
                           deepest table of 16 bits of k-gram index for an
                           NFA (12 for a DFA over fewer than 256 symbols,
                           16 for bytes), lowered when an NFA's records
                           outgrow 16-bit offsets; an explicit k that does
                           not fit fails with E_INVAL, keeping the old table.
                           An NFA over at most 4 symbols with k + 5 <= 16
                           also gets second-level records: for each state
                           set that k symbols leave without a match (up to
                           4096 sets, at most 8 MB of device memory), the
                           outcome of the next 5 symbols */
    int32_t tile;       /* starts owned by one CTA tile (multiple of 4096, at
                           most 49152; 0 = automatic: 16384, smaller for short
                           texts) */
    int32_t halo;       /* text staged past the tile end (multiple of 16) */
    int32_t threads;    /* filtering threads per CTA: 128, 256 or 512 (a
                           scan with 32 starts per thread adds one producer
                           warp that stages the tiles) */
    int32_t spt;        /* consecutive starts each thread filters per round:
                           8 or 32; 0 = automatic (8 for texts too short to
                           give every SM 16 warps at 32, else 32) */
    int32_t table_smem; /* delta table in shared memory: 1 yes, 0 no, -1 auto */
    int32_t ctas_per_sm;/* persistent CTAs per SM (0 = occupancy maximum) */
    int32_t settle;     /* NFA: steps a surviving instance is advanced in the
                           filter before it is queued for the exact path,
                           counted from k symbols past its start (an instance
                           carried by a second-level record starts at step
                           5); 0 = library default (8), -1 = queue at once */
    int32_t partition;  /* instances alive past their tile's staged text
                           (Sec. III.D.2): 1 = lazy (continue in place on the
                           global text), 2 = chained (hand the instance, a
                           DFA's (start, position, state) or an NFA's (start,
                           position, state set), to a carry queue that a
                           second kernel finishes; when the queue is full the
                           rest continue in place); 0 = default (DFA chained,
                           NFA lazy). In pfsm_scan_batch NFA machines are
                           always lazy. */
} pfsm_params;

/* Residency counters of a context. */
typedef struct {
    uint64_t resident_bytes, budget_bytes;
    uint64_t loads, evictions, reloads;
    int32_t resident, loaded;
} pfsm_stats;

/* ------------------------------------------------------------------ context */
/* Create a context on CUDA device `device`. `budget_bytes` bounds the device
 * memory held by resident automata (0 = 8 GiB); scans reload evicted
 * automata and evict the least recently used ones to stay inside it (the
 * device form of the paper's treatment of insomnia, Sec. I-II). Errors:
 * E_INVAL (bad device), E_CUDA, E_NOMEM. */
int pfsm_ctx_create(int device, uint64_t budget_bytes, pfsm_ctx **out);

/* Release every automaton and scratch buffer of the context. Waits for the
 * context's own work to finish. NULL is accepted. */
int pfsm_ctx_destroy(pfsm_ctx *ctx);

/* ------------------------------------------------------------------ automata */
/* Load a DFA-form machine (Sec. II: delta: Q x Sigma -> Q).
 *   delta     host, int16 [Q][S] row-major, every entry in [0, Q)
 *   q0        initial state
 *   dead      an absorbing non-final state (every entry of its row is `dead`,
 *             and it is not final); instances entering it are dropped.
 *             -1 = no dead state: instances then live to the end of the text
 *   is_final  host, uint8 [Q], nonzero = final
 * The table is copied to the device (charged to the budget) along with a
 * start-prefix table derived from it. Errors: E_INVAL (Q outside 1..32767,
 * S outside 1..256, q0/dead out of range, an entry out of range, dead not
 * absorbing or final), E_NOMEM. */
int pfsm_load_dfa(pfsm_ctx *ctx, const int16_t *delta, int32_t Q, int32_t S, int32_t q0,
                  int32_t dead, const uint8_t *is_final, pfsm_aut *out_id);

/* Load an NFA-form machine, run without determinisation (Sec. II: delta:
 * Q x Sigma -> P(Q); Sec. III.A: a PFSM's delta is NFA-like).
 *   delta_bits  host, uint32 [Q][S][W], W = ceil(Q/32): bit (q' % 32) of word
 *               q' / 32 of row (q, a) is set iff q' is in delta(q, a)
 *   q0, is_final as for pfsm_load_dfa
 * An instance whose state set becomes empty is dropped. The machine must be
 * epsilon-free (remove epsilon edges first; the union construction of
 * Sec. III.A is epsilon-free after that). Errors: E_INVAL, E_NOMEM. */
int pfsm_load_nfa(pfsm_ctx *ctx, const uint32_t *delta_bits, int32_t Q, int32_t S, int32_t q0,
                  const uint8_t *is_final, pfsm_aut *out_id);

/* Load an NFA that keeps its epsilon edges for the scan to follow at run
 * time (step 2 of Sec. III.B): after every symbol, and for the instance
 * started at q0, the state set is closed under epsilon edges; a final state
 * reached through them reports at the position of the symbol just consumed,
 * and no empty match is reported. The union machine of Sec. III.A (an
 * ancillary initial state with epsilon edges to each component) loads as it
 * is. delta_bits as for pfsm_load_nfa; eps_bits host [Q][ceil(Q/32)], bit t
 * of row q set iff q -epsilon-> t. delta itself is kept as given; the loader
 * lists, for every state, the states its epsilon edges reach (the closure
 * the scan applies). The prefix depth stays >= 1 for such a machine
 * (prefix_k = -1 is E_INVAL). Result: the same match set as
 * pfsm_load_nfa on the epsilon-free machine. Errors: E_INVAL, E_NOMEM. */
int pfsm_load_nfa_eps(pfsm_ctx *ctx, const uint32_t *delta_bits, const uint32_t *eps_bits,
                      int32_t Q, int32_t S, int32_t q0, const uint8_t *is_final,
                      pfsm_aut *out_id);

/* Drop the device copy of an automaton (its host copy stays); the next scan
 * that names it reloads it. This is the device form of the paper's remedy for
 * insomnia (Sec. I-II: a machine too large for fast memory keeps only its hot
 * part there): cold automata leave device memory and come back on use.
 * Waits for the scans already enqueued that read the copy. Errors: E_NOENT. */
int pfsm_evict(pfsm_ctx *ctx, pfsm_aut aut);

/* Forget an automaton entirely; its id becomes invalid (removing one regular
 * expression from a resident set, Sec. III.A and IV: the other automata keep
 * running). Scans already enqueued that read it keep their copy, which is
 * freed when the last of them completes. Errors: E_NOENT. */
int pfsm_unload(pfsm_ctx *ctx, pfsm_aut aut);

/* Launch parameters of an automaton (the autotuner sets them). `p` may be
 * NULL to restore the defaults. Errors: E_NOENT, E_INVAL. */
int pfsm_set_params(pfsm_ctx *ctx, pfsm_aut aut, const pfsm_params *p);
int pfsm_get_params(pfsm_ctx *ctx, pfsm_aut aut, pfsm_params *out);

/* ------------------------------------------------------------------ scanning */
/* Report every match of `aut` in the text (Sec. III.B; the result is the set
 * M above, in unspecified order).
 *   text_dev   device, n bytes, every byte < S (a byte >= S fails with
 *              E_INVAL after the scan; the output is then unspecified)
 *   out_dev    device, room for `cap` pfsm_match entries
 *   n_matches  host; receives |M| on PFSM_OK and on PFSM_E_OVERFLOW (when
 *              |M| > cap: the first contents of out_dev are unspecified and
 *              the caller retries with cap >= *n_matches)
 *   stream     cudaStream_t or NULL
 * Blocks until the scan has finished on `stream`. n = 0 yields 0 matches.
 * Errors: E_NOENT, E_INVAL (n >= 2^32, NULL pointers with n > 0 or cap > 0,
 * bad symbol), E_OVERFLOW, E_NOMEM (reload), E_TIMEOUT, E_CUDA. */
int pfsm_scan(pfsm_ctx *ctx, pfsm_aut aut, const uint8_t *text_dev, uint64_t n,
              pfsm_match *out_dev, uint64_t cap, uint64_t *n_matches, void *stream);

/* Asynchronous form of pfsm_scan (Sec. III.B, the same match set M): enqueues
 * the scan on `stream` and returns.
 * On completion, status_dev (device, 2 x uint64) holds { |M|, error bits }
 * where error bit 0 = a symbol >= S, bit 1 = a device wait timed out.
 * Capturable in a CUDA graph once the automaton is resident (a scan
 * of a non-resident automaton reloads it, which is a host-synchronous copy).
 * Errors detected on the host are returned directly. */
int pfsm_scan_async(pfsm_ctx *ctx, pfsm_aut aut, const uint8_t *text_dev, uint64_t n,
                    pfsm_match *out_dev, uint64_t cap, uint64_t *status_dev, void *stream);

/* Scan k texts, each with its own automaton, in one batch (the regex and
 * data partitioning of Sec. III.D combined). The automata are grouped into
 * classes (DFA or NFA, prefix-symbol width, DFA table in shared memory); each
 * class runs one persistent kernel over work units of a few consecutive tiles
 * of one text, and the class kernels of a batch run concurrently.
 *   jobs     host, k entries; texts are device pointers
 *   out_dev  device, room for `cap` pfsm_bmatch entries (text = job index)
 *   counts   host, k entries; receives |M| per job (may be NULL)
 *   total    host; receives the sum (also on PFSM_E_OVERFLOW)
 * Blocks until done. Errors: as pfsm_scan, per job. */
int pfsm_scan_batch(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, pfsm_bmatch *out_dev,
                    uint64_t cap, uint64_t *counts, uint64_t *total, void *stream);

/* A union machine (Sec. III.A): automata auts[0..k), DFAs and NFAs mixed,
 * over one device text. The union through an ancillary initial state with
 * epsilon edges to each component's q0 has exactly the union of the
 * components' match sets; here every component runs as one job of a batch
 * over the same text, and a match's `text` field is the index of its
 * component in auts (its `state` is that component's own state id).
 * Components are the caller's loaded automata: adding or removing one is a
 * pfsm_load_* or pfsm_unload between calls, and scans already enqueued keep
 * the images they read (an unloaded automaton still in use is freed when
 * its last scan completes). Arguments, output and errors as
 * pfsm_scan_batch / pfsm_scan_batch_async. */
int pfsm_scan_union(pfsm_ctx *ctx, const pfsm_aut *auts, int32_t k, const uint8_t *text_dev,
                    uint64_t n, pfsm_bmatch *out_dev, uint64_t cap, uint64_t *counts,
                    uint64_t *total, void *stream);
int pfsm_scan_union_async(pfsm_ctx *ctx, const pfsm_aut *auts, int32_t k,
                          const uint8_t *text_dev, uint64_t n, pfsm_bmatch *out_dev,
                          uint64_t cap, uint64_t *status_dev, void *stream);

/* Launch shape of batches on this context: `threads` (128, 256 or 512
 * filtering threads per CTA; the kernels add one producer warp, and NFA
 * classes keep 512 threads in all, so 512 means 480 filtering threads there),
 * `ctas_per_sm` (1 to 4) and `tile` (multiple of 4096, at most 32768; rounded
 * down to whole filter rounds of 32 starts per filtering thread) of *p are
 * used, other fields are ignored. 0 in a field, or a NULL p, selects the
 * default: 256 threads x 2 CTAs per SM for DFA classes, 480 x 1 for NFA
 * classes, tiles of 16384 (15360 for NFA classes). Per-machine parameters (prefix depth,
 * settling) still come from pfsm_set_params. The autotuner sets this.
 * Errors: E_INVAL (a value outside those ranges). */
int pfsm_set_batch_params(pfsm_ctx *ctx, const pfsm_params *p);

/* Asynchronous form of pfsm_scan_batch (Sec. III.B per text, Sec. III.D for
 * the batch): enqueues the batch on `stream` and returns. status_dev (device, k + 2 uint64) receives, when the stream
 * reaches it: [0] total matches, [1] error bits (as pfsm_scan_async),
 * [2 + i] matches of job i. The job array may be reused once the call
 * returns. Errors detected on the host are returned directly. */
int pfsm_scan_batch_async(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, pfsm_bmatch *out_dev,
                          uint64_t cap, uint64_t *status_dev, void *stream);

/* Allocation-free DFA scan. The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory (a plugin that is only
 * handed buffers, a process whose device memory belongs to another
 * allocator, a loop that must never stall on cudaMalloc/cudaFree). It needs
 * no context and allocates nothing; its working memory is one 4 MiB array
 * of device memory that every GPU loading the library holds until exit. The
 * driver reserves the array when it loads the library's module: with lazy
 * module loading (the CUDA default) that happens during the first call on a
 * device, so make that call before another allocator takes the device's
 * memory (CUDA_MODULE_LOADING=EAGER reserves it when the library loads).
 *   delta_dev     device, int16 [Q][S] row-major (entries in [0, Q))
 *   is_final_dev  device, uint8 [Q]
 *   q0, dead      as for pfsm_load_dfa (dead = -1: none)
 *   text_dev, n   device text, n < 2^32, every byte < S
 *   out_dev, cap  device, room for `cap` pfsm_match entries
 *   status_dev    device, 2 x uint64: { |M|, error bits } when the stream
 *                 reaches the end of the scan (bit 0: a symbol >= S or a
 *                 malformed table; |M| > cap means the output was truncated)
 * Limits: Q * S <= 524288 (the encoded table must fit 1 MiB of the array);
 * larger tables fail with E_INVAL. The result is the same match set as
 * pfsm_scan. Asynchronous on `stream`. Every call looks up the array's
 * device address (cudaGetSymbolAddress, which allocates nothing once the
 * module is loaded), so make the first call on a device before any stream
 * capture. Calls share the array: two calls whose
 * work overlaps on the GPU race, so issue them on one stream or wait in
 * between. Errors detected on the host are returned directly. */
int pfsm_scan_dfa_noalloc(const int16_t *delta_dev, int32_t Q, int32_t S, int32_t q0,
                          int32_t dead, const uint8_t *is_final_dev, const uint8_t *text_dev,
                          uint64_t n, pfsm_match *out_dev, uint64_t cap, uint64_t *status_dev,
                          void *stream);

/* ------------------------------------------------------------------ misc */
int pfsm_get_stats(pfsm_ctx *ctx, pfsm_stats *out);

/* Device bytes that automaton `aut` holds while resident (its encoded
 * tables; every automaton of one batch must fit the budget together), and
 * in *resident whether it is resident now (either pointer may be NULL).
 * The paper has no counterpart: this is a query for callers that pack
 * batches under a residency budget. Errors: E_INVAL, E_NOENT. */
int pfsm_aut_bytes(pfsm_ctx *ctx, pfsm_aut aut, uint64_t *bytes, int32_t *resident);

/* Test of the timeout path (no counterpart in the paper). While enabled,
 * single-text scans whose tiles are staged by a producer warp (32 starts per
 * thread) hand no tile to their filtering warps: every wait for a tile runs
 * into its bound (2 s), the kernel ends and the scan reports E_TIMEOUT, and
 * the context stays usable. Nothing faults or hangs; scans of other forms
 * are unaffected. For tests only. Errors: E_INVAL (NULL ctx). */
int pfsm_test_hold_tiles(pfsm_ctx *ctx, int32_t enable);

/* Test of a full carry queue (no counterpart in the paper). Caps the carry
 * queue of later chained single-text scans at `entries` instances and, for
 * NFAs, its pool at `pool_states` states of sets larger than 8; instances
 * that find no room continue in place (lazy), as they do when the real
 * queue fills. 0 restores the library's capacities (2^20 DFA entries;
 * 2^18 NFA entries and 2^21 pool states); values above them are clamped.
 * For tests only. Errors: E_INVAL (NULL ctx). */
int pfsm_test_carry_cap(pfsm_ctx *ctx, uint32_t entries, uint32_t pool_states);

/* Kernel timing: when enabled, every scan records CUDA events around its
 * tile kernel (a batch: around its graph) on the scan's stream;
 * pfsm_kernel_time returns the summed milliseconds and launch count since
 * timing was last enabled. */
int pfsm_set_timing(pfsm_ctx *ctx, int enable);
int pfsm_kernel_time(pfsm_ctx *ctx, double *ms, uint64_t *launches);

/* Static string for a status code. */
const char *pfsm_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PFSM_H */
