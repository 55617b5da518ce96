// Internal declarations of libpfsm: device table encodings, kernel arguments
// and launch helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pfsm.h"

namespace pfsm {

// ---- device encodings of a machine --------------------------------------
// DFA transition entry (uint16): target state in bits 0..14, bit 15 set when
// the target is final; the dead state is stored as DEAD16 so that the kernel
// drops an instance by comparing with a constant.
constexpr uint16_t DEAD16 = 0x7FFF;
constexpr uint16_t FINAL_BIT = 0x8000;
// NFA targets (uint16) use the same layout: state | FINAL_BIT if final.

// Start-prefix table entry (uint16), one per k-gram w (index
// sum_m w[m] << (m * sbits)): the outcome of the first k steps of an instance
// started at q0, computed once per k-gram at load time.
//   PT_SKIP  no instance survives k steps and none matches within them
//   PT_WALK  (DFA) a final state is met within k steps: step from q0
//   other    DFA: the state after k steps (no match on the way);
//            NFA: the word offset o of a record in `pool` holding the
//            matches within the k steps and the state set after them:
//              pool[o] = n_match | n_surv << 16
//              pool[o+1 .. o+n_match]       = step << 16 | final state
//              pool[o+1+n_match .. +n_surv] = surviving states after k steps
constexpr uint16_t PT_SKIP = 0xFFFF;
constexpr uint16_t PT_WALK = 0xFFFE;
// DFA: an entry with bit 15 set (below PT_WALK) is PT_REC | o, the word
// offset o of a record in `pool` in the NFA record format (the matches met
// within the k steps, then the surviving state if there is one: n_surv is 0
// or 1); a k-gram whose record does not fit stays PT_WALK.
constexpr uint16_t PT_REC = 0x8000;
constexpr uint32_t PT_REC_MAX = 0x7FFD;   // largest record offset

// NFA second-level records (2-bit alphabets with k + L2_SYMS <= 16): they
// carry a start L2_SYMS symbols past the prefix table. A first-level record
// with survivors and no matches holds one more word after its survivors,
// the index x of its survivor set (L2_NONE: no second level). Entry
// l2tab[x * 4^L2_SYMS + g], for the next L2_SYMS symbols g of the text
// (g = sum g[i] << 2i), is L2_EMPTY when no state of the set survives them
// and none meets a final state on the way, else the word offset in `pool2`
// of a record in the first-level format whose match steps count from the
// start (k .. k + L2_SYMS - 1) and whose survivors are the states after
// k + L2_SYMS symbols.
constexpr int L2_SYMS = 5;
constexpr uint32_t L2_GRAMS = 1u << (2 * L2_SYMS);
constexpr uint16_t L2_NONE = 0xFFFF;
constexpr uint16_t L2_EMPTY = 0xFFFF;
constexpr uint32_t L2_MAX_SETS = 4096;   // at most 8 MB of second-level tables
constexpr uint32_t L2_NO_REC = 0xFFFFFFFFu;   // (device) a start without a second-level record
// memox[w] (beside the prefix table, same index): the survivor-set index x
// of k-gram w's first-level record when that record has survivors, no
// matches and a second-level table, else L2_NONE. Read together with
// memo[w], it lets a start go to the second level without reading the
// record itself.

// NFA short-gram table: a start with only j < k symbols left before the end
// of its text has its whole future fixed by those j symbols: the matches it
// meets within them. Entry tail_base(j) + (index of the j-gram) holds
// PT_SKIP (no match) or the pool offset of a record with those matches and
// no survivors. tail_base(j) = sum of 2^(i * sbits) for 0 < i < j.
__host__ __device__ inline uint32_t tail_base(int j, int sbits) {
    uint32_t b = 0;
    for (int i = 1; i < j; ++i) b += 1u << (i * sbits);
    return b;
}

// NFA band image (alphabets of at most 4 symbols): Q uint32 rows followed by
// a final-state bitmap of ceil(Q/32) words. Byte a of row q is the mask of
// delta(q, a) within q+1..q+8 (bit d set iff q+1+d is a target). BAND_CSR
// marks a state with a target outside that window: its rows are read from
// the CSR arrays instead.
constexpr uint32_t BAND_CSR = 0xFFFFFFFFu;

// Survival bitmap (optional): one bit per m-gram, set when an instance
// started at q0 meets a final state within those m symbols or still holds a
// state after them; a clear bit settles the start without a lookup.

// Work-queue entry of the filter phase: the absolute start (uint32) and its
// prefix-table entry (uint16; PT_WALK when the instance steps from q0).

// ---- per-scan device state ---------------------------------------------
// status[0] = match count, status[1] = error bits (ERR_*).
constexpr unsigned long long ERR_SYMBOL = 1ull;
constexpr unsigned long long ERR_TIMEOUT = 2ull;
constexpr unsigned long long ERR_CHECK = 8ull;   // a device bounds check failed (PFSM_CHECKED builds)

constexpr int NFA_SLOT = 8;       // states one lane holds for a small NFA set
constexpr int STAGE = 128;        // largest per-warp match staging (entries)
constexpr int SETTLE_PAIRS = 128; // per-warp pool of (start, state) pairs being settled
constexpr int SETTLE_BURST = 4;   // symbols a lane advances its pair between warp syncs
constexpr int WARP_LIST = 1024;   // surviving starts a warp lists per round (32 lanes x 32)
// per-warp list area: the start offsets (uint16), the settling pool, the mark
// bits and the pool count
constexpr int WARP_LIST_BYTES = 2 * WARP_LIST + 4 * SETTLE_PAIRS + WARP_LIST / 8 + 16;
constexpr int FILTER_SPT = 32;    // starts per thread per filter round
constexpr int WARP_QUEUE = 256;   // per-warp queue of instances for the exact path
constexpr int DEEP_GROUP = 1;     // chunks of 32 list entries whose deep-bitmap loads are in flight together

struct ScanArgs {
    // text
    const uint8_t *text;
    uint32_t n;
    uint32_t ntiles;
    uint32_t tile;          // starts per tile
    uint32_t halo;          // bytes staged past the tile
    uint32_t text_buf;      // bytes per staging buffer (tile + halo + 32, rounded)
    uint32_t shift;         // text address mod 16 (tiles are staged from the
                            // 16-byte boundary below and moved down by it)
    // machine
    int32_t Q, S, q0, k, sbits;
    uint32_t memo_n;        // entries of the prefix table (0 when k == 0)
    const uint16_t *memo;   // prefix table (global copy, staged to smem)
    const uint16_t *tail;   // NFA: short-gram table for starts within k of the end, or null
    const uint32_t *ecl_off;// NFA with epsilon edges: closure lists (CSR by state), or null
    const uint16_t *ecl_tgt;
    const uint16_t *dtab;   // DFA: [Q][S]
    const uint32_t *off;    // NFA: [Q*S + 1] CSR offsets
    const uint16_t *tgt;    // NFA: targets
    const uint32_t *pool;   // NFA: prefix records
    const uint16_t *l2tab;  // NFA: second-level tables (see L2_SYMS), or null
    const uint32_t *pool2;  // NFA: second-level records
    const uint16_t *memox;  // NFA: second-level set index per k-gram (with l2tab)
    const uint32_t *band;   // NFA: band image (rows, then final bitmap) or null
    uint32_t pool_n;        // NFA: words of pool
    int32_t pool_smem;      // NFA: pool staged to smem
    int32_t band_smem;      // NFA: band rows staged to smem
    const uint32_t *surv;   // survival bitmap over m-grams, or null
    int32_t surv_m;         // m (0: no bitmap)
    uint32_t surv_words;
    const uint32_t *surv2;  // deep survival bitmap (global memory), or null
    int32_t surv2_m;
    int32_t Wq;             // NFA: 32-bit words of a state bitset
    int32_t surv_bytes;     // the shallow bitmap is staged as one byte per m-gram
                            // (2-grams of bytes: the gram index is the byte offset)
    int32_t tab_smem;       // DFA table staged to smem
    uint32_t *coop_g;       // NFA: global scratch for warp-wide state bitsets
    // output
    uint32_t *out;          // pfsm_match[cap] as words, or pfsm_bmatch
    uint64_t cap;
    unsigned long long *status;
    // chained-partitioning carry queue: DFA entries {job, start, pos, state},
    // NFA entries of 8 words (see NFA_CARRY_WORDS) with larger sets in cpool
    uint32_t *carry;
    uint32_t *carry_n;      // counters (DFA: [0] entries; NFA: see NFA_CARRY_WORDS)
    uint32_t carry_cap;     // entries; 0 = lazy partitioning
    uint16_t *cpool;
    uint32_t cpool_cap;
    // shared-memory layout (byte offsets into dynamic smem)
    uint32_t sm_memo, sm_tab, sm_text, sm_queue, sm_stage, sm_slots, sm_coop, sm_misc;
    int32_t coop_smem;      // NFA: warp-wide bitsets at sm_coop (else in coop_g)
    uint32_t sm_pack;       // the staged tiles as 2-bit symbols (alphabets of <= 4 symbols)
    uint32_t pk_words;      // words of one packed tile
    uint32_t nbuf;          // staged tile buffers, 2 or 3 (layout_smem turns 0 into 2)
    uint32_t hold_tiles;    // test of the timeout path: the producer warp hands no
                            // tile over, so the filtering warps' waits run out
    uint32_t sm_band, sm_pool, sm_surv, sm_list;
    uint32_t stage_n;       // staged matches per warp before a flush
    int32_t memo_smem;      // prefix table staged to smem (else read from global)
    int32_t settle_steps;   // NFA: settling step cap (0 = no settling)
    int32_t spt;            // starts per thread per filter round: 8 or 32 (0 = 32)
};

// Dynamic shared memory of the NFA carry kernel with `nw` warps: band rows
// (when the scan stages them), then per warp the lane slots, the match
// staging buffer and (when the scan keeps them in shared memory) the two
// warp-wide bitsets. Fills the four region offsets, returns the bytes.
inline __host__ __device__ uint32_t carry_nfa_layout(const ScanArgs &a, int nw, uint32_t off[4]) {
    auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    uint32_t o = 0;
    off[0] = o;
    if (a.band_smem && a.band) o += a16(static_cast<uint32_t>(a.Q + (a.Q + 31) / 32) * 4);
    off[1] = o;
    o += a16(static_cast<uint32_t>(nw) * 2 * NFA_SLOT * 32 * 2);
    off[2] = o;
    o += a16(static_cast<uint32_t>(nw) * a.stage_n * 16);
    off[3] = o;
    if (a.coop_smem) o += a16(static_cast<uint32_t>(nw) * 2 * a.Wq * 4);
    return o;
}

// ---- batch executor ------------------------------------------------------
// Machines of a batch fall into classes, one specialised persistent kernel
// each: (kind, prefix-symbol width SB in {0, 2, 8}, DFA table in shared
// memory). Class index: DFA 3 * tab + sb_index, NFA 6 + sb_index.
constexpr int kBatchClasses = 9;
constexpr uint32_t kNotStaged = 0xFFFFFFFFu;   // arena offset of a table left in global memory

// One text of a batch in the device job table (grouped by class, then
// sorted by machine). Its tiles are cut into work units of up to
// BatchArgs::unit_tiles consecutive tiles.
struct BatchJob {
    const uint8_t *text;
    uint32_t n;
    uint32_t mach;        // index into the batch's machine table
    uint32_t orig;        // caller's job index, reported with each match
    uint32_t unit_begin;  // first work unit of this text within its class
    uint32_t ntiles;      // tiles of this text
    uint32_t pad;
};
static_assert(sizeof(BatchJob) == 32, "BatchJob layout");

struct DevMachine {
    int32_t kind;     // 0 DFA, 1 NFA
    int32_t Q, S, q0, k, sbits;
    uint32_t memo_n;
    int32_t Wq;
    const uint16_t *memo;
    const uint16_t *tail;   // NFA: short-gram table (see tail_base), or null
    const uint32_t *ecl_off;// NFA with epsilon edges: closure lists, or null
    const uint16_t *ecl_tgt;
    const uint16_t *dtab;
    const uint32_t *off;
    const uint16_t *tgt;
    const uint32_t *pool;
    const uint16_t *l2tab;  // NFA: second-level tables, or null
    const uint32_t *pool2;
    const uint16_t *memox;  // NFA: second-level set index per k-gram (with l2tab)
    const uint32_t *band;
    uint32_t pool_n;
    int32_t surv_m;
    const uint32_t *surv;
    uint32_t surv_words;
    int32_t surv2_m;
    const uint32_t *surv2;
    // batch: byte offsets of the tables copied into the CTA's shared-memory
    // table arena when this machine's tiles run (kNotStaged: read from
    // global memory; for the survival bitmap: not used)
    uint32_t a_memo, a_tab, a_band, a_pool, a_surv;
    uint32_t a_coop;  // batch: NFA warp-wide bitsets, 2 * Wq words per warp
    int32_t settle;   // batch: NFA settling step cap (0 = no settling)
    int32_t lazy;     // batch: instances past their tile continue in place
};
static_assert(sizeof(DevMachine) % 8 == 0, "DevMachine layout");

// Arguments of one class's persistent batch kernel, read from device memory
// so that one captured graph serves every batch with the same classes.
struct BatchArgs {
    ScanArgs sa;              // class layout, output, status, carry, warp bitsets
    uint32_t nunits;          // work units of this class
    uint32_t job_lo, job_hi;  // this class's slice of the job table
    uint32_t unit_tiles;      // tiles per work unit
    uint32_t sm_arena;        // shared-memory offset of the table arena
    uint32_t pad;
    uint32_t *unit_counter;
    const BatchJob *jobs;     // the whole job table (carry entries use its indices)
    const DevMachine *machs;
    unsigned long long *job_counts;
};

// ---- launch helpers (scan_kernels.cu) ------------------------------------
// Fill the smem offsets of `a` (kind_mask: 1 = DFA present, 2 = NFA present)
// for `threads` threads and the table copies in `need`; returns total bytes.
struct SmemNeed {
    uint32_t memo_bytes;   // prefix table copy (0 = read from global)
    uint32_t tab_bytes;    // DFA table copy (0 = read from global)
    uint32_t band_bytes;   // NFA band image copy (0 = read from global)
    uint32_t pool_bytes;   // NFA prefix records copy (0 = read from global)
    uint32_t surv_bytes;   // survival bitmap (always in shared memory when used)
    uint32_t coop_bytes;   // NFA warp-wide bitsets, all warps (0 = global scratch)
};
uint32_t layout_smem(ScanArgs &a, int kind_mask, int threads, const SmemNeed &need);
cudaError_t launch_scan(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                        cudaStream_t s);
cudaError_t launch_carry(const ScanArgs &a, int grid, cudaStream_t s);
cudaError_t launch_carry_nfa(const ScanArgs &a, int grid, int threads, cudaStream_t s);
int max_ctas_per_sm(int kind, int sbits, int threads, uint32_t smem, bool tab_smem, int spt = 32);
// the kernel instantiated for 8 starts per thread (scan_kernels_spt8.cu)
cudaError_t launch_scan_spt8(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                             cudaStream_t s);
int max_ctas_per_sm_spt8(int kind, int sbits, int threads, uint32_t smem, bool tab_smem);

// ---- batch launch helpers (batch_kernels.cu) -----------------------------
int batch_class(int kind, int sbits, int k, bool tab_smem);
cudaError_t launch_units(int cls, const BatchArgs *dev_args, int threads, int grid,
                         uint32_t smem, cudaStream_t s);
cudaError_t launch_carry_batch(const BatchArgs *dev_args, int grid, cudaStream_t s);
int max_units_ctas_per_sm(int cls, int threads, uint32_t smem);

// Release the batch executor state of a context (batch.cu).
void batch_free(pfsm_ctx *ctx);

}  // namespace pfsm
