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
//            NFA: a record number (record = matches within the k steps and
//            the state set after them, see pool layout below)
constexpr uint16_t PT_SKIP = 0xFFFF;
constexpr uint16_t PT_WALK = 0xFFFE;
// NFA record r at word rec_off[r] of pool:
//   pool[o] = n_match | n_surv << 16
//   pool[o+1 .. o+n_match]       = step << 16 | final state   (step in 0..k-1)
//   pool[o+1+n_match .. +n_surv] = surviving states after k steps

// Work-queue entry of the filter phase (uint32): start offset inside the
// tile in bits 0..15, info in bits 16..31 (a prefix-table entry, or PT_WALK
// when the instance has to step from q0).

// ---- per-scan device state ---------------------------------------------
// status[0] = match count, status[1] = error bits (ERR_*).
constexpr unsigned long long ERR_SYMBOL = 1ull;
constexpr unsigned long long ERR_TIMEOUT = 2ull;

constexpr int NFA_SLOT = 8;       // states one lane holds for a small NFA set
constexpr int STAGE = 128;        // staged matches per warp before a flush

struct ScanArgs {
    // text
    const uint8_t *text;
    uint32_t n;
    uint32_t ntiles;
    uint32_t tile;          // starts per tile
    uint32_t halo;          // bytes staged past the tile
    uint32_t text_buf;      // bytes per staging buffer (tile + halo + 16)
    uint32_t aligned;       // text pointer is 16-byte aligned
    // machine
    int32_t Q, S, q0, k, sbits;
    uint32_t memo_n;        // entries of the prefix table (0 when k == 0)
    const uint16_t *memo;   // prefix table (global copy, staged to smem)
    const uint16_t *dtab;   // DFA: [Q][S]
    const uint32_t *off;    // NFA: [Q*S + 1] CSR offsets
    const uint16_t *tgt;    // NFA: targets
    const uint32_t *rec_off;// NFA: record offsets
    const uint32_t *pool;   // NFA: record words
    int32_t Wq;             // NFA: 32-bit words of a state bitset
    int32_t tab_smem;       // DFA table staged to smem
    // output
    uint32_t *out;          // pfsm_match[cap] as words, or pfsm_bmatch
    uint64_t cap;
    unsigned long long *status;
    // chained-partitioning carry queue (DFA): entries {start, pos, state}
    uint32_t *carry;
    uint32_t *carry_n;
    uint32_t carry_cap;
    // shared-memory layout (byte offsets into dynamic smem)
    uint32_t sm_memo, sm_tab, sm_text, sm_queue, sm_stage, sm_slots, sm_coop, sm_misc;
    uint32_t qcap;
};

// Per-item description for the batch kernel.
struct BatchItem {
    uint32_t job;     // index into the job table
    uint32_t tile;    // tile index inside the job's text
};

struct BatchJob {
    const uint8_t *text;
    uint32_t n;
    uint32_t aut;     // index into the machine table
};

struct DevMachine {
    int32_t kind;     // 0 DFA, 1 NFA
    int32_t Q, S, q0, k, sbits;
    uint32_t memo_n;
    int32_t Wq;
    const uint16_t *memo;
    const uint16_t *dtab;
    const uint32_t *off;
    const uint16_t *tgt;
    const uint32_t *rec_off;
    const uint32_t *pool;
};

// ---- launch helpers (scan_kernels.cu) ------------------------------------
struct LaunchCfg {
    int threads;
    int ctas_per_sm;
    uint32_t smem_bytes;
    int spt;
};

// Fill the smem offsets of `a` for `threads` threads; returns total bytes.
uint32_t layout_smem(ScanArgs &a, int kind, int threads, int spt);
cudaError_t launch_scan(const ScanArgs &a, int kind, int threads, int grid, cudaStream_t s);
cudaError_t launch_carry(const ScanArgs &a, int grid, cudaStream_t s);
int max_ctas_per_sm(int kind, int sbits, int threads, uint32_t smem, bool tab_smem);

// Release the batch executor state of a context (batch.cu).
void batch_free(pfsm_ctx *ctx);

}  // namespace pfsm
