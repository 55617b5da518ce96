// Device building blocks of the PFSM scan for sm_103a, shared by the
// single-text kernels (scan_kernels.cu) and the batch kernels (batch_kernels.cu).
//
//
// One persistent CTA loops over text tiles. A tile owns the instances that
// start in [b, b + tile) and stages t[b, b + tile + halo) into shared memory
// with a 1-D bulk TMA copy (double buffered, evict-first in L2). Instances
// that are still alive past the staged halo either go to a carry queue that a
// second kernel continues over the global text (chained data partitioning,
// Sec. III.D.2: a DFA instance as its start, position and state, an NFA
// instance as its start, position and state set) or continue in place
// (lazy data partitioning, same section).
//
// Every start i is an instance {(i, q0)} (reinitialisation, Sec. III.B step 1).
// Its first k steps depend only on t[i..i+k), so their outcome is read from a
// start-prefix table built at load time (one entry per k-gram: dies, a single
// surviving DFA state, or an NFA record of matches and survivors). The filter
// phase streams the tile, looks each start up and queues only the instances
// that still have work. The continuation phase drains the queue: every lane
// holds one instance, advances it one symbol per iteration through delta
// (Sec. III.B steps 3-4), reports final targets (start = tag, end = current
// position), and refills from the queue when its instance dies. A lane that
// holds an NFA set too large for its slot hands it to the whole warp, which
// advances it as a bitset over Q.
//
// Matches are staged per warp in shared memory with ballot/popc appends and
// flushed with one global atomic per flush.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pfsm_internal.h"

namespace pfsm {

#define FULLMASK 0xffffffffu

// PFSM_CHECKED builds (libpfsm_checked.so) test the data-dependent indices of
// the device code before they are used: a failing test sets ERR_CHECK in the
// scan's status (reported as PFSM_E_CHECK) and the access is skipped or made
// with a safe index instead. Nothing traps. Other builds compile the tests
// away (PFSM_OK_IDX is then always true).
#ifdef PFSM_CHECKED
#define PFSM_OK_IDX(cond, status) ((cond) ? true : (atomicOr(&(status)[1], ERR_CHECK), false))
#else
#define PFSM_OK_IDX(cond, status) true
#endif

// The dynamic shared memory of the scan kernels (the same array as the
// kernels' own extern declaration). A 2-gram byte table sits at offset 0 of
// it, so a gram indexes this array directly.
extern __shared__ __align__(128) uint8_t pfsm_dyn_smem[];

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint16_t ldg_u16_keep(const uint16_t *p, uint64_t pol) {
    uint16_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u32_keep(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Non-blocking test of a phase (for a thread that polls several barriers).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a bulk-copy barrier: gives up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return true;
}

// Wait on a barrier that other warps of the CTA complete: gives up after
// ~2 s during which no warp of the CTA was inside a drain (*busy == 0
// throughout). A drain ends by itself (every instance reaches the end of
// its text or dies), so the wait stays bounded.
__device__ __forceinline__ bool mbar_wait_live(uint64_t *bar, uint32_t parity,
                                               const uint32_t *busy) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        const uint64_t now = global_ns();
        if (*reinterpret_cast<const volatile uint32_t *>(busy) != 0) t0 = now;
        else if (now - t0 > 2000000000ull) return false;
    }
    return true;
}

// Shared-memory control words of a CTA.
constexpr int kTileBufs = 3;   // most staged tiles a CTA holds
struct Misc {
    uint64_t bar[2];              // batch kernel: bar[0] = the filtering warps' meetings
    uint64_t full[kTileBufs];     // the buffer's copy landed
    uint64_t ready[kTileBufs];    //   realigned and packed by the producer warp
    uint64_t empty[kTileBufs];    //   every filtering warp is done with it
    uint32_t q_count;
    uint32_t q_head;
    uint32_t abort;
    uint32_t busy;                // warps inside a drain (continuation work that
                                  // can run long but always ends): waits do not
                                  // time out while it is nonzero
};

// ------------------------------------------------------------ symbol checks
// Byte-wise "x >= S" over a 64-bit word, high bit of each byte set on hit.
__device__ __forceinline__ uint64_t bytes_ge(uint64_t x, uint32_t S) {
    const uint64_t ones = 0x0101010101010101ull, m7 = 0x7F7F7F7F7F7F7F7Full,
                   h = 0x8080808080808080ull;
    if (S <= 128) return (((x & m7) + (uint64_t)(0x80 - S) * ones) | x) & h;
    return (((x & m7) + (uint64_t)(0x80 - (S - 128)) * ones) & x) & h;
}

// 2-bit packing of 8 bytes (each 0..3) into 16 bits, byte m at bits 2m.
__device__ __forceinline__ uint32_t pack2(uint64_t x) {
    x &= 0x0303030303030303ull;
    x = (x | (x >> 6)) & 0x000F000F000F000Full;
    x = (x | (x >> 12)) & 0x000000FF000000FFull;
    x = (x | (x >> 24)) & 0xFFFFull;
    return static_cast<uint32_t>(x);
}

// Prefix-table index of the start at window byte r (k symbols from byte r).
template <int SB>
__device__ __forceinline__ uint32_t memo_index(uint64_t lo, uint64_t hi, uint32_t p2, int r,
                                               int k, int sbits, uint32_t mask) {
    if (SB == 2) {
        return (p2 >> (2 * r)) & mask;
    } else if (SB == 8) {
        const uint64_t w = r == 0 ? lo : ((lo >> (8 * r)) | (hi << (64 - 8 * r)));
        return static_cast<uint32_t>(w) & mask;
    } else {
        uint32_t idx = 0;
        const uint32_t sm = (1u << sbits) - 1;
        for (int m = 0; m < k; ++m) {
            const int j = r + m;
            const uint32_t byte =
                static_cast<uint32_t>((j < 8 ? (lo >> (8 * j)) : (hi >> (8 * (j - 8)))) & 0xFF);
            idx |= (byte & sm) << (sbits * m);
        }
        return idx;
    }
}

// m-gram index (m <= 12) of the start at offset `off` of the staged tile,
// read from four aligned words.
template <int SB>
__device__ __forceinline__ uint32_t gram_at16(const uint8_t *tsm, uint32_t off, int m, int sbits,
                                              uint32_t mask) {
    const uint32_t a4 = off & ~3u, r = off & 3u;
    const uint4 w = *reinterpret_cast<const uint4 *>(tsm + (a4 & ~15u));
    // realign to a4 (a4 may sit 4, 8 or 12 bytes into the 16-byte block)
    const uint32_t sh = (a4 & 15u) >> 2;
    const uint32_t x0 = sh == 0 ? w.x : sh == 1 ? w.y : sh == 2 ? w.z : w.w;
    const uint32_t x1 = sh == 0 ? w.y : sh == 1 ? w.z : sh == 2 ? w.w : 0u;
    const uint32_t x2 = sh == 0 ? w.z : sh == 1 ? w.w : 0u;
    const uint32_t x3 = sh == 0 ? w.w : 0u;
    uint32_t y1 = x1, y2 = x2, y3 = x3;
    if (sh) {   // the missing words come from the next 16-byte block
        const uint4 v = *reinterpret_cast<const uint4 *>(tsm + (a4 & ~15u) + 16);
        if (sh == 1) y3 = v.x;
        if (sh == 2) { y2 = v.x; y3 = v.y; }
        if (sh == 3) { y1 = v.x; y2 = v.y; y3 = v.z; }
    }
    const uint64_t lo = x0 | (static_cast<uint64_t>(y1) << 32);
    const uint64_t hi = y2 | (static_cast<uint64_t>(y3) << 32);
    const uint32_t p2 = SB == 2 ? (pack2(lo) | (pack2(hi) << 16)) : 0u;
    return memo_index<SB>(lo, hi, p2, static_cast<int>(r), m, sbits, mask);
}

// Symbols p .. p + 15 of the packed tile (2 bits each, symbol p lowest):
// the index of any gram of up to 16 symbols starting at p, after a mask.
__device__ __forceinline__ uint32_t pk_gram(const uint32_t *pk, uint32_t p) {
    return __funnelshift_r(pk[p >> 4], pk[(p >> 4) + 1], (p & 15u) * 2u);
}

// Byte-wise "x >= S" over a 32-bit word (S <= 128), high bit of each byte set
// on a hit: (x & 0x7F) + 0x80 - S carries into bit 7 exactly when the low
// seven bits reach S, and the OR with x catches bytes of 128 and above.
__device__ __forceinline__ uint32_t bytes_ge32(uint32_t x, uint32_t S) {
    return (((x & 0x7F7F7F7Fu) + (0x80u - S) * 0x01010101u) | x) & 0x80808080u;
}

// 2-bit packing of 16 bytes (each 0..3, in w0..w3) into 32 bits, byte m at
// bits 2m. Multiplying a word of four 2-bit values b0..b3 (one per byte) by
// 2^24 + 2^18 + 2^12 + 2^6 puts b0 + 4 b1 + 16 b2 + 64 b3 in its top byte:
// the product of byte i with the term 2^(24 - 6i) lands at bit 24 + 2i, every
// other partial product lands at bit 32 or above (dropped) or below bit 24,
// and those lower ones sum to less than 2^24, so nothing carries into the
// top byte. Three byte permutations gather the four top bytes.
__device__ __forceinline__ uint32_t pack16(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
    constexpr uint32_t M = 0x01041040u;
    constexpr uint32_t K = 0x03030303u;
    const uint32_t lo = __byte_perm((w0 & K) * M, (w1 & K) * M, 0x0073);
    const uint32_t hi = __byte_perm((w2 & K) * M, (w3 & K) * M, 0x0073);
    return __byte_perm(lo, hi, 0x5410);
}

// Packs the staged tile (len bytes at tsm) to 2-bit symbols, 16 per word,
// and checks the bytes of the tile's own starts [0, own) against the
// alphabet (S <= 4 here). The threads tid = 0, nt, 2 nt, ... of the caller
// share the work; the caller synchronises before the packed words are read.
__device__ __forceinline__ void pack_tile(const uint8_t *tsm, uint32_t *pk, uint32_t len,
                                          uint32_t own, uint32_t S, bool &bad_symbol, int tid,
                                          int nt) {
    const uint32_t nwords = (len + 15) / 16 + 1;
    const uint32_t full = own / 16;   // blocks whose 16 bytes are all own starts
    const uint4 *t4 = reinterpret_cast<const uint4 *>(tsm);
    uint32_t bad = 0;
#pragma unroll 4
    for (uint32_t w = tid; w < nwords; w += nt) {
        const uint4 v = t4[w];
        pk[w] = pack16(v.x, v.y, v.z, v.w);
        if (w < full) {
            bad |= bytes_ge32(v.x, S) | bytes_ge32(v.y, S) | bytes_ge32(v.z, S) |
                   bytes_ge32(v.w, S);
        } else if (16 * w < own) {
            // the block holding the last own start: bytes [16 w, own) only
            const uint32_t nb = own - 16 * w;   // 1 .. 15
            const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int valid = static_cast<int>(nb) - 4 * k;
                if (valid > 0) {
                    const uint32_t m = valid >= 4 ? 0xFFFFFFFFu : ((1u << (8 * valid)) - 1);
                    bad |= bytes_ge32(x[k], S) & m;
                }
            }
        }
    }
    if (bad) bad_symbol = true;
}

// Prefix-table index of the start at offset `off` of the staged tile (k
// symbols read from three aligned words; k <= 8).
template <int SB>
__device__ __forceinline__ uint32_t kgram_at(const uint8_t *tsm, uint32_t off, int k, int sbits,
                                             uint32_t mask) {
    const uint32_t a4 = off & ~3u, r = off & 3u;
    const uint32_t w0 = *reinterpret_cast<const uint32_t *>(tsm + a4);
    const uint32_t w1 = *reinterpret_cast<const uint32_t *>(tsm + a4 + 4);
    const uint32_t w2 = *reinterpret_cast<const uint32_t *>(tsm + a4 + 8);
    const uint64_t lo = w0 | (static_cast<uint64_t>(w1) << 32);
    const uint64_t hi = w2;
    const uint32_t p2 = SB == 2 ? (pack2(lo) | (pack2(hi) << 16)) : 0u;
    return memo_index<SB>(lo, hi, p2, static_cast<int>(r), k, sbits, mask);
}

// ------------------------------------------------------------ views
// The machine one tile runs (registers).
struct MView {
    int32_t Q, S, q0, k, sbits, Wq, surv_m, surv2_m;
    const uint32_t *surv2;
    const uint16_t *dtab;
    const uint32_t *off;
    const uint16_t *tgt;
    const uint16_t *tail;   // NFA short-gram table, or null
    const uint32_t *ecl_off;// NFA with epsilon edges: epsilon closure lists, or null
    const uint16_t *ecl_tgt;
    const uint16_t *l2tab;  // NFA second-level tables (see L2_SYMS), or null
    const uint32_t *pool2;  // NFA second-level records
    const uint16_t *memox;  // NFA second-level set index per k-gram (with l2tab)
    unsigned long long *chk;   // status words of the scan (bounds-check failures)
    uint32_t pool_n, memo_n;   // words of the record pool, entries of the prefix table
};

// Where matches and carried instances go.
struct OView {
    uint32_t *out;
    uint64_t cap;
    unsigned long long *status;       // [0] match count, [1] error bits
    unsigned long long *job_counts;   // per-text counts (batch) or null
    uint32_t *carry;                  // DFA: {job, start, pos, state} entries;
                                      // NFA: NFA_CARRY_WORDS-word entries
    uint32_t *carry_n;                // DFA: [0] entries. NFA: see NFA_CARRY_WORDS
    uint32_t carry_cap;               // entries (0: lazy partitioning)
    uint32_t stage_n;                 // per-warp staging capacity (entries)
    // (members below are zero when an initialiser list stops before them)
    uint16_t *cpool;                  // NFA: states of carried sets of more than
    uint32_t cpool_cap;               //   NFA_CARRY_INLINE states
    // NFA, single text: an instance started at i is carried from the end of
    // its own tile's staged text, min(n, (i / seg_tile + 1) seg_tile +
    // seg_halo), or from i + NFA_CARRY_AFTER if that comes first; seg_tile
    // 0: from the end of the tile staged when it runs
    uint32_t seg_tile, seg_halo;
};

// NFA carry queue: entries of 8 words {job, start, pos, n, ...}. The first
// half of the queue holds the sets a lane held (n <= NFA_CARRY_INLINE states
// packed two per word in words 4 .. 7; counter carry_n[0], claimed through
// carry_n[2]); the second half the sets the whole warp held, their states in
// cpool from the offset in word 4 (counter carry_n[3], claimed through
// carry_n[4]; carry_n[1] counts cpool states).
constexpr uint32_t NFA_CARRY_WORDS = 8;
constexpr uint32_t NFA_CARRY_INLINE = 8;
// An NFA instance is carried (chained partitioning) when it reaches the end
// of its tile's staged text or, earlier, NFA_CARRY_AFTER symbols past its
// start: a long-lived instance then runs in the carry kernel, which spreads
// such instances over every SM, instead of in the drain of the warp that
// queued it.
constexpr uint32_t NFA_CARRY_AFTER = 256;
// The same for DFA instances (chained scans): an instance still alive
// DFA_CARRY_AFTER symbols past its start goes to carry_dfa, one thread per
// instance over the whole grid. Instances that live that long are the
// paper's quadratic case (a machine without a dead state: every instance
// lives to the end of the text), where the early hand-over spreads them over
// every SM; a shorter bound would also hand over the few longest instances
// of ordinary scans, whose tail in the carry kernel then costs more than it
// saves in the drain.
constexpr uint32_t DFA_CARRY_AFTER = 256;

// One staged tile: bytes [b, b + len) of a text are in shared memory.
struct TileView {
    const uint8_t *sm;
    const uint8_t *text;
    uint32_t b, len, n;
    uint32_t job;    // index into the device job table (batch), 0 otherwise
    uint32_t orig;   // caller's text index reported with the matches
};

// Shared-memory regions of one CTA.
struct Smem {
    Misc *misc;
    const uint16_t *memo;
    const uint16_t *tab;
    const uint32_t *band;             // NFA band image (shared copy, global, or null)
    const uint32_t *pool;             // NFA prefix records (shared copy or global)
    const uint32_t *surv;             // survival bitmap (shared copy) or null
    const uint8_t *survb;             // the same as one byte per m-gram, or null
    uint16_t *list;                   // this warp's list of surviving starts
    uint32_t *pairs;                  // this warp's settling pool (SETTLE_PAIRS)
    uint32_t *pcount;                 // its fill count
    uint32_t *marks;                  // WARP_LIST bits: entries sent to the exact path
    uint32_t *wq_start;               // this warp's work queue: absolute starts
    uint16_t *wq_info;                //   and prefix-table entries (WARP_QUEUE)
    uint32_t *wq_flag;                //   NFA: bit i set = entry i is a second-level
                                      //   record (continue L2_SYMS symbols later)
    uint32_t *stage;   // this warp's staging buffer
    uint16_t *slots;   // this warp's NFA slots
    uint32_t *coop;    // this warp's two bitsets of Wq words
    uint32_t *pk;      // the staged tile as 2-bit symbols (2-bit kernels)
};

__device__ __forceinline__ uint32_t text_at(const TileView &tv, uint32_t pos) {
    const uint32_t rel = pos - tv.b;
    return rel < tv.len ? tv.sm[rel] : __ldg(tv.text + pos);
}

// ------------------------------------------------------------ match output
// Per-warp staging of matches (OUTW words each: [text,] start, end, state);
// `sn` is warp-uniform. A flush reserves room with one global atomic.
template <int OUTW>
__device__ __forceinline__ void stage_flush(uint32_t *buf, uint32_t &sn, const OView &ov,
                                            uint32_t orig, int lane) {
    __syncwarp();
    if (sn == 0) return;
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(&ov.status[0], (unsigned long long)sn);
        if (ov.job_counts) atomicAdd(&ov.job_counts[orig], (unsigned long long)sn);
    }
    base = __shfl_sync(FULLMASK, base, 0);
    const uint32_t words = OUTW * sn;
    for (uint32_t w = lane; w < words; w += 32) {
        const unsigned long long idx = base + w / OUTW;
        if (idx < ov.cap) ov.out[base * OUTW + w] = buf[w];
    }
    __syncwarp();
    sn = 0;
}

template <int OUTW>
__device__ __forceinline__ void warp_emit(bool has, uint32_t s, uint32_t e, uint32_t st,
                                          uint32_t *buf, uint32_t &sn, const OView &ov,
                                          const TileView &tv, int lane) {
    const uint32_t m = __ballot_sync(FULLMASK, has);
    if (m == 0) return;
    const uint32_t c = __popc(m);
    if (sn + c > ov.stage_n) stage_flush<OUTW>(buf, sn, ov, tv.orig, lane);
    if (!PFSM_OK_IDX(sn + c <= ov.stage_n, ov.status)) return;
    if (has) {
        uint32_t *p = buf + OUTW * (sn + __popc(m & lanemask_lt()));
        if (OUTW == 4) *p++ = tv.orig;
        p[0] = s;
        p[1] = e;
        p[2] = st;
    }
    sn += c;
}

// Direct append for divergent callers (warp-cooperative sets, carried runs).
template <int OUTW>
__device__ __forceinline__ void emit_direct(const OView &ov, uint32_t orig, uint32_t s,
                                            uint32_t e, uint32_t st) {
    const unsigned long long idx = atomicAdd(&ov.status[0], 1ull);
    if (ov.job_counts) atomicAdd(&ov.job_counts[orig], 1ull);
    if (idx < ov.cap) {
        uint32_t *p = ov.out + idx * OUTW;
        if (OUTW == 4) *p++ = orig;
        p[0] = s;
        p[1] = e;
        p[2] = st;
    }
}

// The matches of prefix records: lane l reports its n_l record entries
// (step << 16 | final, from rec[ptr]) for start `start`. One warp prefix sum
// over n_l places every lane's matches in the staging buffer (flushed when
// full), instead of one ballot per match.
template <int OUTW>
__device__ __forceinline__ void emit_record_matches(uint32_t n_l, const uint32_t *rec, uint32_t ptr,
                                                    uint32_t start, uint32_t *buf, uint32_t &sn,
                                                    const OView &ov, const TileView &tv, int lane) {
    uint32_t incl = n_l;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULLMASK, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULLMASK, incl, 31);
    const uint32_t excl = incl - n_l;
    uint32_t done = 0;   // ranks below this are staged (warp-uniform)
    while (done < total) {
        if (sn >= ov.stage_n) stage_flush<OUTW>(buf, sn, ov, tv.orig, lane);
        const uint32_t hi = min(total, done + (ov.stage_n - sn));
        const uint32_t a = max(excl, done), z = min(excl + n_l, hi);
        for (uint32_t r = a; r < z; ++r) {
            const uint32_t w = rec[ptr + (r - excl)];
            uint32_t *p = buf + OUTW * (sn + (r - done));
            if (OUTW == 4) *p++ = tv.orig;
            p[0] = start;
            p[1] = start + (w >> 16);
            p[2] = w & 0xFFFFu;
        }
        sn += hi - done;
        done = hi;
    }
    __syncwarp();
}

// ------------------------------------------------------------ continuation: DFA
// Drains the work queue with lane refill: one symbol per lane per iteration.
template <bool TAB_SMEM, int OUTW>
__device__ void drain_dfa(const OView &ov, const MView &mv, const TileView &tv, const Smem &sm,
                          uint32_t qn, uint32_t &sn, int lane, uint64_t pol_keep) {
    uint32_t head = 0;
    const uint32_t S = mv.S, n = tv.n;
    // no staged tile (the final drain): nothing to hand to the carry queue
    const uint32_t tile_end = tv.len ? tv.b + tv.len : 0xFFFFFFFFu;
    bool act = false;
    bool gmode = false;   // past the staged text and the carry queue is full
    uint32_t start = 0, pos = 0, s = 0;
    uint32_t pm_left = 0, pm_ptr = 0;   // matches of a prefix record still to report
    while (true) {
        const bool need = !act;
        const uint32_t m = __ballot_sync(FULLMASK, need);
        if (m && head < qn) {
            const uint32_t base = head;
            head += __popc(m);
            if (need) {
                const uint32_t qi = base + __popc(m & lanemask_lt());
                if (qi < qn) {
                    start = sm.wq_start[qi];
                    const uint32_t info = sm.wq_info[qi];
                    act = true;
                    gmode = false;
                    if (info == PT_WALK) {
                        s = mv.q0;
                        pos = start;
                    } else if (info & PT_REC) {
                        // the matches of the first k steps, then the survivor
                        const uint32_t ro = info & 0x7FFFu;
                        const uint32_t w0 = sm.pool[ro];
                        pm_left = w0 & 0xFFFFu;
                        pm_ptr = ro + 1;
                        if (w0 >> 16) {
                            s = sm.pool[ro + 1 + pm_left];
                            pos = start + mv.k;
                        } else {
                            act = false;
                        }
                    } else {
                        s = info;
                        pos = start + mv.k;
                    }
                }
            }
        }
        if (__any_sync(FULLMASK, pm_left > 0)) {
            emit_record_matches<OUTW>(pm_left, sm.pool, pm_ptr, start, sm.stage, sn, ov, tv, lane);
            pm_left = 0;
        }
        if (!__any_sync(FULLMASK, act)) {
            if (head >= qn) break;
            continue;   // every refilled entry was a finished record
        }
        bool hit = false;
        uint32_t hend = 0;
        if (act) {
            if (pos >= n) {
                act = false;
            } else if ((pos >= tile_end || pos - start >= DFA_CARRY_AFTER) && ov.carry_cap && !gmode) {
                // chained: hand the instance to the carry queue past the
                // staged text, or DFA_CARRY_AFTER symbols past its start;
                // lazy (no queue) or a full queue: continue in place
                const uint32_t ci = ov.carry_cap ? atomicAdd(ov.carry_n, 1u) : 0u;
                if (ci < ov.carry_cap) {
                    uint32_t *c = ov.carry + 4 * ci;
                    c[0] = tv.job;
                    c[1] = start;
                    c[2] = pos;
                    c[3] = s;
                    act = false;
                } else {
                    gmode = true;
                }
            }
            if (act) {
                const uint32_t c = text_at(tv, pos);
                uint16_t e = DEAD16;
                if (c < S) {
                    const uint32_t ix = s * S + c;
                    if (PFSM_OK_IDX(s < static_cast<uint32_t>(mv.Q), ov.status))
                        e = TAB_SMEM ? sm.tab[ix] : ldg_u16_keep(mv.dtab + ix, pol_keep);
                }
                if (e == DEAD16) {
                    act = false;
                } else {
                    s = e & 0x7FFFu;
                    hit = (e & FINAL_BIT) != 0;
                    hend = pos;
                    ++pos;
                }
            }
        }
        warp_emit<OUTW>(hit, start, hend, s, sm.stage, sn, ov, tv, lane);
    }
}

// ------------------------------------------------------------ NFA rows
// Visits delta(q, c) as (state | FINAL_BIT) values: from the band row of q
// when it has one, otherwise from the CSR arrays.
template <class F>
__device__ __forceinline__ void nfa_targets(const MView &mv, const uint32_t *band, uint32_t q,
                                            uint32_t c, uint64_t pol_keep, F &&f) {
    if (!PFSM_OK_IDX(q < static_cast<uint32_t>(mv.Q), mv.chk)) return;
    if (band) {
        const uint32_t row = band[q];
        if (row != BAND_CSR) {
            const uint32_t *fin = band + mv.Q;
            uint32_t m = (row >> (8 * c)) & 0xFFu;
            while (m) {
                const uint32_t t = q + __ffs(m);
                m &= m - 1;
                if (!PFSM_OK_IDX(t < static_cast<uint32_t>(mv.Q), mv.chk)) break;
                f(t | (((fin[t >> 5] >> (t & 31)) & 1u) << 15));
            }
            return;
        }
    }
    const uint32_t lo = ldg_u32_keep(mv.off + q * mv.S + c, pol_keep);
    const uint32_t hi = ldg_u32_keep(mv.off + q * mv.S + c + 1, pol_keep);
    for (uint32_t e = lo; e < hi; ++e) {
        const uint32_t t = ldg_u16_keep(mv.tgt + e, pol_keep);
        f(t);
        if (mv.ecl_off) {
            // step 2 of Sec. III.B: the states t reaches through epsilon edges
            const uint32_t ts = t & 0x7FFFu;
            const uint32_t a = ldg_u32_keep(mv.ecl_off + ts, pol_keep);
            const uint32_t z = ldg_u32_keep(mv.ecl_off + ts + 1, pol_keep);
            for (uint32_t x = a; x < z; ++x) f(static_cast<uint32_t>(ldg_u16_keep(mv.ecl_tgt + x, pol_keep)));
        }
    }
}

// Settling of surviving NFA starts, one warp at a time. The instances of a
// chunk of <= 32 list entries are split into (start, state) pairs, one per
// state of their prefix record; lanes advance one pair per iteration through
// the band rows (the first target stays in the lane, further targets go back
// to a per-warp pool) and refill from the pool. A pair dies when its state
// has no target on the next symbol. Since the futures of the states of a set
// are independent, an instance whose pairs all die before meeting a final
// state reports nothing and is settled. Any other outcome (a final target,
// a row outside the band, the staged text or the step limit running out, a
// full pool, matches inside the prefix) marks the instance, and marked
// instances are queued for the exact path, which redoes them from their
// record, so nothing is reported twice.
__device__ __forceinline__ void mark_entry(uint32_t *marks, uint32_t j) {
    atomicOr(&marks[j >> 5], 1u << (j & 31));
}
__device__ __forceinline__ bool marked(const uint32_t *marks, uint32_t j) {
    return (marks[j >> 5] >> (j & 31)) & 1u;
}

static __device__ void nfa_settle_chunk(const MView &mv, const Smem &sm, const TileView &tv,
                                 uint32_t j0, uint32_t total, uint32_t e, uint32_t r2, int lane,
                                 uint32_t max_steps) {
    uint32_t *pairs = sm.pairs;
    uint32_t *pcount = sm.pcount;
    uint32_t *marks = sm.marks;
    const uint32_t b = tv.b, n = tv.n, tile_end = tv.b + tv.len;
    const uint32_t *fin = sm.band + mv.Q;
    // 1. pairs from the prefix records of entries j0 + lane: the first-level
    //    record (its survivors at step 0, k symbols past the start) or, where
    //    the lane has one (r2 != L2_NO_REC), the second-level record (its
    //    survivors at step L2_SYMS)
    {
        const uint32_t j = j0 + lane;
        uint32_t ns = 0, rec = 0;
        uint32_t pre0 = 0, pre1 = 0, pre2 = 0;   // a second-level record's first survivors
        const bool lvl2 = r2 != L2_NO_REC;
        if (j < total) {
            if (e == PT_WALK) {
                mark_entry(marks, j);
            } else if (e != PT_SKIP) {
                uint32_t hdr;
                if (lvl2) {
                    // the header and the first three words after it in one
                    // round trip (the records are followed by 16 bytes of slack)
                    const uint32_t *p = mv.pool2 + r2;
                    hdr = __ldg(p);
                    pre0 = __ldg(p + 1);
                    pre1 = __ldg(p + 2);
                    pre2 = __ldg(p + 3);
                } else {
                    hdr = sm.pool[e];
                }
                if (hdr & 0xFFFFu) mark_entry(marks, j);   // matches inside the prefix
                else ns = hdr >> 16, rec = lvl2 ? r2 : e;
            }
        }
        uint32_t incl = ns;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(FULLMASK, incl, d);
            if (lane >= d) incl += v;
        }
        const uint32_t base = *pcount + incl - ns;
        const bool fits = base + ns <= static_cast<uint32_t>(SETTLE_PAIRS);
        if (ns && !fits) mark_entry(marks, j);
        if (ns && fits) {
            if (lvl2) {
                for (uint32_t x = 0; x < ns; ++x) {
                    const uint32_t q = x == 0 ? pre0 : x == 1 ? pre1 : x == 2 ? pre2
                                     : __ldg(mv.pool2 + rec + 1 + x);
                    pairs[base + x] = (j << 21) | (static_cast<uint32_t>(L2_SYMS) << 15) | q;
                }
            } else {
                for (uint32_t x = 0; x < ns; ++x)
                    pairs[base + x] = (j << 21) | sm.pool[rec + 1 + x];   // step 0
            }
        }
        const uint32_t end = __reduce_max_sync(FULLMASK, (ns && fits) ? base + ns : 0u);
        __syncwarp();
        if (lane == 0 && end > *pcount) *pcount = end;
        __syncwarp();
    }
    // 2. advance pairs with lane refill until the pool is empty
    bool has = false;
    uint32_t li = 0, step = 0, q = 0, start_pos = 0;
    while (true) {
        const uint32_t need = __ballot_sync(FULLMASK, !has);
        uint32_t avail = 0, take = 0;
        if (lane == 0) {
            avail = *pcount;
            take = min(avail, static_cast<uint32_t>(__popc(need)));
            *pcount = avail - take;
        }
        avail = __shfl_sync(FULLMASK, avail, 0);
        take = __shfl_sync(FULLMASK, take, 0);
        if (!has) {
            const uint32_t r = __popc(need & lanemask_lt());
            if (r < take) {
                const uint32_t e = pairs[avail - take + r];
                li = e >> 21;
                step = (e >> 15) & 0x3Fu;
                q = e & 0x7FFFu;
                start_pos = b + sm.list[li] + mv.k;
                has = true;
            }
        }
        __syncwarp();
        if (!__any_sync(FULLMASK, has)) break;
        if (has && marked(marks, li)) has = false;
        // each lane advances its pair up to SETTLE_BURST symbols between warp
        // synchronisations (pairs forked on the way go to the pool with
        // shared-memory atomics; a pair whose start another lane marked in
        // the meantime only does some useless steps)
        for (int burst = 0; burst < SETTLE_BURST && has; ++burst) {
            const uint32_t pos = start_pos + step;
            if (pos >= n) {
                has = false;
                break;
            }
            if (pos >= tile_end || step >= max_steps) {
                mark_entry(marks, li);
                has = false;
                break;
            }
            const uint32_t c = tv.sm[pos - b];
            const uint32_t row = c < static_cast<uint32_t>(mv.S) ? sm.band[q] : 0u;
            if (row == BAND_CSR) {
                mark_entry(marks, li);
                has = false;
                break;
            }
            uint32_t m = (row >> (8 * c)) & 0xFFu;
            bool first = true;
            uint32_t nq = 0;
            while (m) {
                const uint32_t t = q + __ffs(m);
                m &= m - 1;
                if ((fin[t >> 5] >> (t & 31)) & 1u) {
                    mark_entry(marks, li);
                    first = true;
                    nq = 0xFFFFFFFFu;
                    break;
                }
                if (first) {
                    nq = t;
                    first = false;
                } else {
                    const uint32_t slot = atomicAdd(pcount, 1u);
                    if (slot < static_cast<uint32_t>(SETTLE_PAIRS))
                        pairs[slot] = (li << 21) | ((step + 1) << 15) | t;
                    else
                        mark_entry(marks, li);
                }
            }
            if (first || nq == 0xFFFFFFFFu) {
                has = false;
                break;
            }
            q = nq;
            ++step;
        }
        __syncwarp();
        if (lane == 0 && *pcount > static_cast<uint32_t>(SETTLE_PAIRS)) *pcount = SETTLE_PAIRS;
        __syncwarp();
    }
}

// Sets or clears the flag of queue entry p (NFA queues: the entry's record is
// a second-level one). Called by the lane that writes the entry.
__device__ __forceinline__ void queue_flag(uint32_t *flag, uint32_t p, bool on) {
    if (on) atomicOr(&flag[p >> 5], 1u << (p & 31));
    else atomicAnd(&flag[p >> 5], ~(1u << (p & 31)));
}

// ------------------------------------------------------------ continuation: NFA
// Chained partitioning: one lane hands its instance (n <= NFA_CARRY_INLINE
// states, FINAL_BIT ignored) to the carry queue. False when the queue is full.
__device__ __forceinline__ bool carry_nfa_lane(const OView &ov, uint32_t job, uint32_t start,
                                               uint32_t pos, const uint16_t *st, uint32_t stride,
                                               uint32_t cnt) {
    const uint32_t ci = atomicAdd(&ov.carry_n[0], 1u);
    if (ci >= ov.carry_cap / 2) return false;
    uint32_t *c = ov.carry + NFA_CARRY_WORDS * ci;
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
#pragma unroll
    for (uint32_t i = 0; i < NFA_CARRY_INLINE; ++i) {
        const uint32_t v = i < cnt ? (static_cast<uint32_t>(st[i * stride]) & 0x7FFFu) << (16 * (i & 1))
                                   : 0u;
        if (i < 2) w0 |= v;
        else if (i < 4) w1 |= v;
        else if (i < 6) w2 |= v;
        else w3 |= v;
    }
    reinterpret_cast<uint4 *>(c)[0] = make_uint4(job, start, pos, cnt);
    reinterpret_cast<uint4 *>(c)[1] = make_uint4(w0, w1, w2, w3);
    return true;
}

// The whole warp hands the set in `bits` (a bitset over Q) to the carry
// queue, its states in cpool. False, with nothing queued, when there is no
// room (an entry claimed without pool room is written empty).
__device__ __forceinline__ bool carry_nfa_warp(const OView &ov, const MView &mv, uint32_t job,
                                                   uint32_t start, uint32_t pos, const uint32_t *bits,
                                                   int lane) {
    const uint32_t Wq = mv.Wq;
    uint32_t mine = 0;
    for (uint32_t w = lane; w < Wq; w += 32) mine += __popc(bits[w]);
    uint32_t incl = mine;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULLMASK, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(FULLMASK, incl, 31);
    uint32_t ci = 0, po = 0, ok = 0;
    if (lane == 0) {
        ci = atomicAdd(&ov.carry_n[3], 1u);
        if (ci < ov.carry_cap - ov.carry_cap / 2) {
            po = atomicAdd(&ov.carry_n[1], total);
            ok = po + total <= ov.cpool_cap && po + total >= po ? 1u : 2u;
        }
    }
    ok = __shfl_sync(FULLMASK, ok, 0);
    ci = __shfl_sync(FULLMASK, ci, 0);
    po = __shfl_sync(FULLMASK, po, 0);
    if (ok == 0) return false;
    uint32_t *c = ov.carry + NFA_CARRY_WORDS * (ov.carry_cap / 2 + ci);
    if (ok == 2) {   // an entry without pool room: written empty
        if (lane == 0) reinterpret_cast<uint4 *>(c)[0] = make_uint4(job, start, pos, 0u);
        __syncwarp();
        return false;
    }
    uint32_t j = po + incl - mine;
    for (uint32_t w = lane; w < Wq; w += 32) {
        uint32_t x = bits[w];
        while (x) {
            ov.cpool[j++] = static_cast<uint16_t>(w * 32 + __ffs(x) - 1);
            x &= x - 1;
        }
    }
    if (lane == 0) {
        reinterpret_cast<uint4 *>(c)[0] = make_uint4(job, start, pos, total);
        reinterpret_cast<uint4 *>(c)[1] = make_uint4(po, 0u, 0u, 0u);
    }
    __syncwarp();
    return true;
}

// Position of the k-th (from 0) set bit of x; k < popc(x).
__device__ __forceinline__ uint32_t select_bit(uint32_t x, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t low = __popc(x & ((1u << w) - 1u));
        if (k >= low) {
            k -= low;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Warp-cooperative advance of one instance as a bitset over Q. The states of
// each 32-word chunk of the set are ranked (a warp scan of the words' bit
// counts) and lane j steps the states of rank j, j + 32, ..., so a set packed
// into a few words spreads over the whole warp. At `seg_end` (the end of the
// instance's own segment) it goes to the carry queue when the scan has one
// (chained partitioning) and room is left, otherwise it reads the global
// text on (lazy).
template <int OUTW>
__device__ __forceinline__ void coop_run_body(const OView &ov, const MView &mv,
                                              const uint32_t *band, const TileView &tv,
                                              uint32_t *bits0, uint32_t *bits1, uint32_t start,
                                              uint32_t pos, uint32_t seg_end, int lane,
                                              uint64_t pol_keep) {
    const uint32_t Wq = mv.Wq, S = mv.S, n = tv.n;
    // single-text scans only: a batch's NFA machines are always lazy
    bool chain = OUTW == 3 && ov.carry_cap > 0;
    uint32_t *cur = bits0, *nxt = bits1;
    while (pos < n) {
        if (OUTW == 3 && chain && pos >= seg_end) {
            if (carry_nfa_warp(ov, mv, tv.job, start, pos, cur, lane)) break;
            chain = false;
        }
        const uint32_t c = text_at(tv, pos);
        if (c >= S) break;
        for (uint32_t w0 = 0; w0 < Wq; w0 += 32) {
            const uint32_t x = w0 + lane < Wq ? cur[w0 + lane] : 0u;
            const uint32_t cx = __popc(x);
            uint32_t incl = cx;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(FULLMASK, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t excl = incl - cx;
            const uint32_t total = __shfl_sync(FULLMASK, incl, 31);
            for (uint32_t r = 0; r < total; r += 32) {
                const uint32_t j = r + lane;
                // the lane holding rank j: the last with excl <= j
                uint32_t own = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const uint32_t e = __shfl_sync(FULLMASK, excl, own + step);
                    if (e <= j) own += step;
                }
                const uint32_t xo = __shfl_sync(FULLMASK, x, own);
                const uint32_t eo = __shfl_sync(FULLMASK, excl, own);
                if (j < total) {
                    const uint32_t q = (w0 + own) * 32 + select_bit(xo, j - eo);
                    nfa_targets(mv, band, q, c, pol_keep, [&](uint32_t t) {
                        const uint32_t ts = t & 0x7FFFu;
                        const uint32_t mb = 1u << (ts & 31);
                        const uint32_t old = atomicOr(&nxt[ts >> 5], mb);
                        if ((t & FINAL_BIT) && !(old & mb)) emit_direct<OUTW>(ov, tv.orig, start, pos, ts);
                    });
                }
            }
        }
        __syncwarp();
        uint32_t any = 0;
        for (uint32_t w = lane; w < Wq; w += 32) {
            cur[w] = 0;
            any |= nxt[w];
        }
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
        ++pos;
        if (!__any_sync(FULLMASK, any != 0)) break;
        __syncwarp();
    }
    __syncwarp();
}

// The batch kernels call the warp-wide run out of line (inlined, it costs
// their NFA classes hundreds of bytes of spills at 128 registers); the
// single-text kernels inline it, so that the views it reads need no stack
// copy at every drain.
template <int OUTW>
__device__ __noinline__ void coop_run_call(const OView &ov, const MView &mv, const uint32_t *band,
                                           const TileView &tv, uint32_t *bits0, uint32_t *bits1,
                                           uint32_t start, uint32_t pos, uint32_t seg_end, int lane,
                                           uint64_t pol_keep) {
    coop_run_body<OUTW>(ov, mv, band, tv, bits0, bits1, start, pos, seg_end, lane, pol_keep);
}
template <int OUTW>
__device__ __forceinline__ void coop_run(const OView &ov, const MView &mv, const uint32_t *band,
                                         const TileView &tv, uint32_t *bits0, uint32_t *bits1,
                                         uint32_t start, uint32_t pos, uint32_t seg_end, int lane,
                                         uint64_t pol_keep) {
    if constexpr (OUTW == 3)
        coop_run_body<OUTW>(ov, mv, band, tv, bits0, bits1, start, pos, seg_end, lane, pol_keep);
    else
        coop_run_call<OUTW>(ov, mv, band, tv, bits0, bits1, start, pos, seg_end, lane, pol_keep);
}

enum : uint32_t { MODE_LANE = 0, MODE_COOP_SLOT = 1, MODE_COOP_POOL = 2 };

// Drains the work queue for an NFA: each lane holds one instance's state set
// (up to NFA_SLOT states) and advances it one symbol per iteration. With
// CARRY the work is the first half of the carry queue instead (qn entries
// of lane-held sets, claimed through ov.carry_n[2] by every warp of the carry
// kernel, at most `claim` at a time, so that a short queue still spreads
// over every warp).
enum : uint32_t { REC_POOL = 0, REC_POOL2 = 1 };

template <int OUTW, bool CARRY = false>
__device__ void drain_nfa(const OView &ov, const MView &mv, const TileView &tv, const Smem &sm,
                          uint32_t qn, uint32_t &sn, int lane, uint64_t pol_keep,
                          uint32_t claim = 32) {
    uint32_t head = 0;
    const uint32_t S = mv.S, n = tv.n;
    // no staged tile (the final drain, the carry kernel): nothing to carry
    const uint32_t tile_end = tv.len ? tv.b + tv.len : 0xFFFFFFFFu;
    constexpr int C = NFA_SLOT;
    static_assert(C <= static_cast<int>(NFA_CARRY_INLINE), "a lane's set fits a carry entry");
    uint16_t *slots = sm.slots;
#define SLOT(sel, i) slots[((sel) * C + (i)) * 32 + lane]
    bool act = false;
    bool gmode = false;                // past the staged text with the carry queue full
    bool done = false;                 // CARRY: every entry is claimed
    uint32_t start = 0, pos = 0, cnt = 0, cb = 0, mode = MODE_LANE;
    uint32_t pm_left = 0, pm_ptr = 0, cptr = 0;
    uint32_t send = 0xFFFFFFFFu;       // end of the instance's own segment
    bool l2e = false;                  // this lane's record is a second-level one
    uint32_t rsel = REC_POOL;          // where its record (or carried set) is
    const uint32_t *rec = sm.pool;
    while (true) {
        const bool need = !act;
        const uint32_t m = __ballot_sync(FULLMASK, need);
        uint32_t base = 0;
        bool got = false;
        uint32_t take = __popc(m);
        if (CARRY) {
            take = min(take, claim);
            if (m && !done) {
                uint32_t b0 = 0;
                if (lane == 0) b0 = atomicAdd(&ov.carry_n[2], take);
                base = __shfl_sync(FULLMASK, b0, 0);
                done = base >= qn;
                got = !done;
            }
        } else if (m && head < qn) {
            base = head;
            head += __popc(m);
            got = true;
        }
        const uint32_t rank = __popc(m & lanemask_lt());
        if (got && need && (!CARRY || rank < take)) {
            const uint32_t qi = base + rank;
            if (CARRY && qi < qn) {
                const uint32_t *c = ov.carry + NFA_CARRY_WORDS * qi;
                const uint4 h = reinterpret_cast<const uint4 *>(c)[0];
                start = h.y;
                pos = h.z;
                cnt = h.w & 0xFFFFu;
                send = 0xFFFFFFFFu;
                act = true;
                gmode = false;
                mode = MODE_LANE;
                pm_left = 0;
                l2e = false;
                rsel = REC_POOL;
                const uint4 sw = reinterpret_cast<const uint4 *>(c)[1];
                if (cnt > static_cast<uint32_t>(C)) cnt = C;
#pragma unroll
                for (uint32_t i = 0; i < static_cast<uint32_t>(C); ++i) {
                    const uint32_t w = i < 2 ? sw.x : i < 4 ? sw.y : i < 6 ? sw.z : sw.w;
                    if (i < cnt) SLOT(cb, i) = static_cast<uint16_t>(w >> (16 * (i & 1)));
                }
            } else if (!CARRY && qi < qn) {
                {
                    start = sm.wq_start[qi];
                    const uint32_t info = sm.wq_info[qi];
                    act = true;
                    gmode = false;
                    // chained: the instance leaves at the end of its own
                    // tile's staged text, also when a later tile (or the
                    // final drain) runs it
                    if (OUTW == 3)
                        send = ov.seg_tile
                                   ? min(min(n, (start / ov.seg_tile + 1) * ov.seg_tile + ov.seg_halo),
                                         start + NFA_CARRY_AFTER)
                                   : tile_end;
                    mode = MODE_LANE;
                    pm_left = 0;
                    // a second-level record continues L2_SYMS symbols later
                    l2e = (sm.wq_flag[qi >> 5] >> (qi & 31)) & 1u;
                    rsel = l2e ? REC_POOL2 : REC_POOL;
                    rec = l2e ? mv.pool2 : sm.pool;
                    if (info == PT_WALK) {
                        SLOT(cb, 0) = static_cast<uint16_t>(mv.q0);
                        cnt = 1;
                        pos = start;
                    } else {
                        const uint32_t ro = info;
                        const uint32_t w0 = PFSM_OK_IDX(l2e || ro < mv.pool_n, ov.status) ? rec[ro] : 0u;
                        const uint32_t nm = w0 & 0xFFFFu, ns = w0 >> 16;
                        pm_left = nm;
                        pm_ptr = ro + 1;
                        pos = start + mv.k + (l2e ? static_cast<uint32_t>(L2_SYMS) : 0u);
                        cnt = ns;
                        if (ns > static_cast<uint32_t>(C)) {
                            mode = MODE_COOP_POOL;
                            cptr = ro + 1 + nm;
                        } else {
                            for (uint32_t i = 0; i < ns; ++i)
                                SLOT(cb, i) = static_cast<uint16_t>(rec[ro + 1 + nm + i]);
                        }
                    }
                }
            }
        }
        if (!__any_sync(FULLMASK, act)) break;

        // matches inside the first k steps, from the prefix record
        if (__any_sync(FULLMASK, pm_left > 0)) {
            emit_record_matches<OUTW>(pm_left, rec, pm_ptr, start, sm.stage, sn, ov, tv, lane);
            pm_left = 0;
        }
        if (act && mode == MODE_LANE && cnt == 0) act = false;

        // past the staged text: to the carry queue (chained partitioning)
        // unless the scan is lazy or the queue is full (single-text scans
        // only: a batch's NFA machines are always lazy)
        if (OUTW == 3 && act && pos < n && pos >= send && ov.carry_cap && !gmode) {
            if (mode == MODE_LANE) {
                if (carry_nfa_lane(ov, tv.job, start, pos, &SLOT(cb, 0), 32, cnt)) act = false;
                else gmode = true;
            }
        }

        // one symbol for every lane-held instance
        bool anyfin = false;
        if (act && mode == MODE_LANE) {
            if (pos >= n) {
                act = false;
            } else {
                const uint32_t c = text_at(tv, pos);
                if (c >= S) {
                    act = false;
                } else {
                    uint32_t ncnt = 0;
                    bool ovf = false;
                    for (uint32_t i = 0; i < cnt && !ovf; ++i) {
                        const uint32_t q = SLOT(cb, i) & 0x7FFFu;
                        nfa_targets(mv, sm.band, q, c, pol_keep, [&](uint32_t t) {
                            if (ovf) return;
                            const uint32_t ts = t & 0x7FFFu;
                            for (uint32_t j = 0; j < ncnt; ++j)
                                if ((SLOT(cb ^ 1, j) & 0x7FFFu) == ts) return;
                            if (ncnt == static_cast<uint32_t>(C)) {
                                ovf = true;
                                return;
                            }
                            SLOT(cb ^ 1, ncnt) = static_cast<uint16_t>(t);
                            ++ncnt;
                            anyfin |= (t & FINAL_BIT) != 0;
                        });
                    }
                    if (ovf) {
                        mode = MODE_COOP_SLOT;   // redo this symbol on the warp
                        anyfin = false;
                    } else {
                        cb ^= 1;
                        cnt = ncnt;
                    }
                }
            }
        }
        const uint32_t fin_n = __reduce_max_sync(FULLMASK, anyfin ? cnt : 0u);
        if (fin_n) {
            for (uint32_t j = 0; j < fin_n; ++j) {
                const bool has = anyfin && j < cnt && (SLOT(cb, j) & FINAL_BIT);
                warp_emit<OUTW>(has, start, pos, has ? (SLOT(cb, j) & 0x7FFFu) : 0u, sm.stage,
                                sn, ov, tv, lane);
            }
        }
        if (act && mode == MODE_LANE) {
            ++pos;
            if (cnt == 0) act = false;
        }

        // instances whose set outgrew the lane slot run on the whole warp
        uint32_t cm = __ballot_sync(FULLMASK, act && mode != MODE_LANE);
        while (cm) {
            const int src = __ffs(cm) - 1;
            cm &= cm - 1;
            const uint32_t cs = __shfl_sync(FULLMASK, start, src);
            const uint32_t cp = __shfl_sync(FULLMASK, pos, src);
            const uint32_t cmode = __shfl_sync(FULLMASK, mode, src);
            const uint32_t ccnt = __shfl_sync(FULLMASK, cnt, src);
            const uint32_t ccb = __shfl_sync(FULLMASK, cb, src);
            const uint32_t cpt = __shfl_sync(FULLMASK, cptr, src);
            const uint32_t cse = OUTW == 3 ? __shfl_sync(FULLMASK, gmode ? 0xFFFFFFFFu : send, src)
                                           : 0xFFFFFFFFu;
            const uint32_t csel = __shfl_sync(FULLMASK, rsel, src);
            const uint32_t *crec = csel == REC_POOL2 ? mv.pool2 : sm.pool;
            uint32_t *b0 = sm.coop, *b1 = sm.coop + mv.Wq;
            for (uint32_t w = lane; w < static_cast<uint32_t>(mv.Wq); w += 32) {
                b0[w] = 0;
                b1[w] = 0;
            }
            __syncwarp();
            if (cmode == MODE_COOP_SLOT) {
                if (static_cast<uint32_t>(lane) < ccnt) {
                    const uint32_t q = slots[(ccb * C + lane) * 32 + src] & 0x7FFFu;
                    atomicOr(&b0[q >> 5], 1u << (q & 31));
                }
            } else {
                for (uint32_t i = lane; i < ccnt; i += 32) {
                    const uint32_t q = crec[cpt + i];
                    if (!PFSM_OK_IDX(q < static_cast<uint32_t>(mv.Q), ov.status)) continue;
                    atomicOr(&b0[q >> 5], 1u << (q & 31));
                }
            }
            __syncwarp();
            coop_run<OUTW>(ov, mv, sm.band, tv, b0, b1, cs, cp, cse, lane, pol_keep);
            if (lane == src) {
                act = false;
                mode = MODE_LANE;
            }
        }
    }
#undef SLOT
}

template <int KIND, bool TAB_SMEM, int OUTW>
__device__ __forceinline__ void drain(const OView &ov, const MView &mv, const TileView &tv,
                                      const Smem &sm, uint32_t &wq_n, uint32_t &sn, int lane,
                                      uint64_t pol_keep) {
    if (wq_n == 0) return;
    // the CTA's waits do not time out while this drain runs
    if (lane == 0) atomicAdd(&sm.misc->busy, 1u);
    if (KIND == 0)
        drain_dfa<TAB_SMEM, OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
    else
        drain_nfa<OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
    __syncwarp();
    if (lane == 0) atomicSub(&sm.misc->busy, 1u);
    wq_n = 0;
}

// ------------------------------------------------------------ lane-local settling
// Single-text NFA scans with second-level records: a start that passes the
// deep filter is held by one lane (its start and the 32 symbols from it,
// packed), until every lane of the warp holds one. Then each lane, on its
// own, looks its start up (prefix entry and second-level set index side by
// side, the second-level entry, the first words of the second-level record)
// and advances the record's state set (at most SETTLE_LANE_STATES states,
// Sec. III.B step 3 on one instance) through the band rows from L2_SYMS
// steps past the prefix up to the settling cap. An instance whose set
// empties reports nothing and is done. Any other outcome (a final state,
// a match inside the records, a row outside the band, a larger set, the
// cap) sends the start to the exact path (the warp queue), which redoes it
// from its first-level record. No warp synchronisation inside the pass.
constexpr int SETTLE_LANE_STATES = 4;

// The same register slot serves DFA scans with a deep bitmap (see
// dfa_consume): there g0 is the start's prefix entry and g1 its deep-bitmap
// word as loaded a round earlier, sh the bit of g1 to test.
struct Pend {
    uint32_t start;   // absolute start
    uint32_t g0, g1;  // symbols start .. start + 15 and start + 16 .. start + 31
    uint32_t sh;
    bool on;
};

// DFA scans with a deep survival bitmap: the loads of a round's candidates
// (the starts that pass the shallow bitmap) are issued into the lanes'
// registers and consumed one round later, when the next round's filter has
// hidden their latency. A candidate whose deep bit is set and whose prefix
// entry is not PT_SKIP goes to the warp queue with that entry.
template <bool TAB_SMEM, int OUTW>
__device__ __forceinline__ void dfa_consume(const OView &ov, const MView &mv, const TileView &tv,
                                            const Smem &sm, Pend &p, uint32_t &wq_n, uint32_t &sn,
                                            int lane, uint64_t pol_keep) {
    const bool push = p.on && ((p.g1 >> p.sh) & 1u) && p.g0 != PT_SKIP;
    p.on = false;
    const uint32_t pm = __ballot_sync(FULLMASK, push);
    if (pm) {
        if (wq_n + 32 > static_cast<uint32_t>(WARP_QUEUE))
            drain<0, TAB_SMEM, OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
        if (push) {
            const uint32_t at = wq_n + __popc(pm & lanemask_lt());
            if (PFSM_OK_IDX(at < static_cast<uint32_t>(WARP_QUEUE), ov.status)) {
                sm.wq_start[at] = p.start;
                sm.wq_info[at] = static_cast<uint16_t>(p.g0);
            }
        }
        wq_n += __popc(pm);
        __syncwarp();
    }
}

template <int KIND, bool TAB_SMEM, int OUTW>
__device__ void settle_lanes(const OView &ov, const MView &mv, const TileView &tv, const Smem &sm,
                             Pend &p, uint32_t &wq_n, uint32_t &sn, int lane, uint64_t pol_keep,
                             uint32_t max_steps) {
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    const uint32_t kk = static_cast<uint32_t>(mv.k), n = tv.n;
    const uint32_t mask = (1u << (2 * kk)) - 1;
    const uint32_t *fin = sm.band + mv.Q;
    bool exact = false;
    bool from_l2 = false;   // the exact path continues from the second-level record
    uint32_t e = PT_SKIP;
    if (p.on) {
        const uint32_t gi = p.g0 & mask;
        const uint32_t x = ldg_u16_keep(mv.memox + gi, pol_keep);
        e = PFSM_OK_IDX(gi < mv.memo_n, ov.status) ? sm.memo[gi] : PT_SKIP;
        if (x == L2_NONE) {
            exact = e != PT_SKIP;
        } else {
            const uint32_t o2 = ldg_u16_keep(
                mv.l2tab + x * L2_GRAMS + ((p.g0 >> (2 * kk)) & (L2_GRAMS - 1)), pol_keep);
            if (o2 != L2_EMPTY) {
                // the first-level record has no matches: the exact path can
                // resume from this one (its matches and its set L2_SYMS later)
                e = o2;
                from_l2 = true;
                const uint32_t *q = mv.pool2 + o2;   // 16 bytes of slack follow the records
                const uint32_t hdr = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2),
                               w3 = __ldg(q + 3);
                const uint32_t ns = hdr >> 16;
                if ((hdr & 0xFFFFu) || ns == 0 || ns > 3) {
                    exact = true;
                } else {
                    uint32_t s0 = w1, s1 = ns > 1 ? w2 : NONE, s2 = ns > 2 ? w3 : NONE, s3 = NONE;
                    uint32_t cnt = ns;
                    for (uint32_t st = L2_SYMS; st < max_steps && cnt; ++st) {
                        const uint32_t pos = p.start + kk + st;
                        if (pos >= n) {   // the text ends: nothing more to report
                            cnt = 0;
                            break;
                        }
                        const uint32_t ix = kk + st;   // < 32
                        const uint32_t c = (ix < 16 ? p.g0 >> (2 * ix) : p.g1 >> (2 * (ix - 16))) & 3u;
                        uint32_t n0 = NONE, n1 = NONE, n2 = NONE, n3 = NONE, nc = 0;
                        bool bad = false;
#pragma unroll
                        for (int i = 0; i < SETTLE_LANE_STATES; ++i) {
                            const uint32_t qs = i == 0 ? s0 : i == 1 ? s1 : i == 2 ? s2 : s3;
                            if (static_cast<uint32_t>(i) < cnt && !bad) {
                                const uint32_t row = PFSM_OK_IDX(qs < static_cast<uint32_t>(mv.Q), ov.status)
                                                         ? sm.band[qs] : BAND_CSR;
                                if (row == BAND_CSR) {
                                    bad = true;
                                } else {
                                    uint32_t m = (row >> (8 * c)) & 0xFFu;
                                    while (m && !bad) {
                                        const uint32_t t = qs + __ffs(m);
                                        m &= m - 1;
                                        if ((fin[t >> 5] >> (t & 31)) & 1u) {
                                            bad = true;   // a match: the exact path reports it
                                        } else if (t != n0 && t != n1 && t != n2 && t != n3) {
                                            if (nc == SETTLE_LANE_STATES) {
                                                bad = true;
                                            } else {
                                                n0 = nc == 0 ? t : n0;
                                                n1 = nc == 1 ? t : n1;
                                                n2 = nc == 2 ? t : n2;
                                                n3 = nc == 3 ? t : n3;
                                                ++nc;
                                            }
                                        }
                                    }
                                }
                            }
                        }
                        if (bad) {
                            exact = true;
                            cnt = 0;
                            break;
                        }
                        s0 = n0;
                        s1 = n1;
                        s2 = n2;
                        s3 = n3;
                        cnt = nc;
                    }
                    if (cnt) exact = true;   // alive at the cap
                }
            }
        }
    }
    p.on = false;
    const uint32_t pm = __ballot_sync(FULLMASK, exact);
    if (pm) {
        if (wq_n + 32 > static_cast<uint32_t>(WARP_QUEUE))
            drain<KIND, TAB_SMEM, OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
        if (exact) {
            const uint32_t at = wq_n + __popc(pm & lanemask_lt());
            if (PFSM_OK_IDX(at < static_cast<uint32_t>(WARP_QUEUE), ov.status)) {
                sm.wq_start[at] = p.start;
                sm.wq_info[at] = static_cast<uint16_t>(e);
                queue_flag(sm.wq_flag, at, from_l2);
            }
        }
        wq_n += __popc(pm);
        __syncwarp();
    }
}

// ------------------------------------------------------------ one tile
// Filter phase over the tile's own starts [b, own_end), then the
// continuation of every queued instance. All threads of the CTA call this.
// SPT: starts per thread per filter round (SPT / 8 windows of 8; 8 or 32).
// NT consumer threads (ids 0 .. NT - 1) call it together.
// DEFER: NFA starts past the deep filter are settled lane by lane
// (settle_lanes) once every lane holds one, and a DFA round's deep-bitmap
// loads are consumed a round later (dfa_consume); `pend` persists across
// tiles of one text and the caller finishes what is left (settle_lanes /
// dfa_consume) before it changes text or machine and after its last tile.
template <int KIND, int SB, bool TAB_SMEM, int OUTW, int SPT = 32, bool DEFER = false>
__device__ void process_tile(const OView &ov, const MView &mv, const TileView &tv,
                             const Smem &sm, uint32_t own_end, uint32_t &wq_n, uint32_t &sn,
                             bool &bad_symbol, uint64_t pol_keep, uint32_t settle_steps, int NT,
                             Pend &pend) {
    static_assert(SPT == 8 || SPT == 32, "SPT");
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t n = tv.n, b = tv.b;
    const uint32_t kk = static_cast<uint32_t>(mv.k);
    const uint32_t kbits = static_cast<uint32_t>(mv.k * mv.sbits);
    const uint32_t mask = kbits >= 32 ? 0xFFFFFFFFu : ((1u << kbits) - 1);
    const uint32_t round = SPT * NT;
    const uint32_t mm = static_cast<uint32_t>(mv.surv_m);
    const uint32_t mbits = mm * static_cast<uint32_t>(mv.sbits);
    const uint32_t mmask = mbits >= 32 ? 0xFFFFFFFFu : ((1u << mbits) - 1);
    const uint32_t m2 = static_cast<uint32_t>(mv.surv2_m);
    const uint32_t m2bits = m2 * static_cast<uint32_t>(mv.sbits);
    const uint32_t m2mask = m2bits >= 32 ? 0xFFFFFFFFu : ((1u << m2bits) - 1);
    for (uint32_t r0 = b; r0 < own_end; r0 += round) {
        // 1. this thread's SPT starts, in SPT / 8 windows of 8 consecutive
        //    starts: window g of lane l of warp w begins at
        //    r0 + 32 SPT w + 256 g + 8 l, so the lanes of a warp read
        //    consecutive bytes of the tile (no shared-memory bank
        //    conflicts). Symbol check and the shared-memory survival bitmap,
        //    one 16-byte window per 8 starts; bit 8 g + r of `live` is start
        //    r of window g.
        const uint32_t wbase = r0 + static_cast<uint32_t>(tid >> 5) * (32u * SPT) + 8u * lane;
        uint32_t live = 0;
        // byte alphabets of 256 symbols with a 2-gram byte table, every window
        // of the round owned and clear of the end of the text: no checks
        const uint32_t wlast = wbase + 256u * (SPT / 8 - 1);
        const bool fast = SB == 8 && sm.survb != nullptr && mv.S == 256 && wlast + 8 <= own_end &&
                          wlast + 8 + mm <= n;
        // 2-bit symbols with a shallow bitmap (single-text kernels: at
        // offset 0), every window of the round owned and clear of the end
        const bool fast2 = SB == 2 && sm.surv == reinterpret_cast<const uint32_t *>(pfsm_dyn_smem) &&
                           wlast + 8 <= own_end && wlast + 8 + mm <= n;
        if (__all_sync(FULLMASK, fast2)) {
            const uint32_t *bm = reinterpret_cast<const uint32_t *>(pfsm_dyn_smem);
#pragma unroll
            for (int g = 0; g < SPT / 8; ++g) {
                const uint32_t p2 = pk_gram(sm.pk, wbase - b + 256u * g);
                uint32_t v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const uint32_t t = p2 >> (2 * r);
                    const uint32_t w = bm[(t & mmask) >> 5];
                    v[r] = __funnelshift_r(w, w, t) & 1u;   // rotate bit t mod 32 to bit 0
                }
                const uint32_t k01 = v[0] | (v[1] << 1), k23 = v[2] | (v[3] << 1);
                const uint32_t k45 = v[4] | (v[5] << 1), k67 = v[6] | (v[7] << 1);
                live |= ((k01 | (k23 << 2)) | ((k45 | (k67 << 2)) << 4)) << (8 * g);
            }
        } else if (__all_sync(FULLMASK, fast)) {
            const uint8_t *tp = tv.sm + (wbase - b);
#pragma unroll
            for (int g = 0; g < SPT / 8; ++g) {
                const uint2 l = *reinterpret_cast<const uint2 *>(tp + 256 * g);
                const uint32_t x0 = l.x, x1 = l.y;
                const uint32_t x2 = *reinterpret_cast<const uint32_t *>(tp + 256 * g + 8);
                uint32_t v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const uint32_t idx = r < 3 ? __byte_perm(x0, 0u, 0x4400 | ((r + 1) << 4) | r)
                                       : r == 3 ? __byte_perm(x0, x1, 0x0043) & 0xFFFFu
                                       : r < 7 ? __byte_perm(x1, 0u, 0x4400 | ((r - 3) << 4) | (r - 4))
                                               : __byte_perm(x1, x2, 0x0043) & 0xFFFFu;
                    v[r] = pfsm_dyn_smem[idx];
                }
                const uint32_t k01 = v[0] | (v[1] << 1), k23 = v[2] | (v[3] << 1);
                const uint32_t k45 = v[4] | (v[5] << 1), k67 = v[6] | (v[7] << 1);
                live |= ((k01 | (k23 << 2)) | ((k45 | (k67 << 2)) << 4)) << (8 * g);
            }
        } else
#pragma unroll
        for (int g = 0; g < SPT / 8; ++g) {
            const uint32_t iw = wbase + 256u * g;   // the window's first start
            if (iw < own_end) {
                const uint32_t gown = min(8u, own_end - iw);
                uint32_t keep = gown >= 8 ? 0xFFu : ((1u << gown) - 1);
                // 2-bit kernels read the packed tile (symbols checked when it
                // was packed); others the bytes of the window
                uint64_t lo = 0, hi = 0;
                if (SB != 2) {
                    const uint8_t *tp = tv.sm + (iw - b);
                    const uint2 l2 = *reinterpret_cast<const uint2 *>(tp);
                    const uint2 h2 = *reinterpret_cast<const uint2 *>(tp + 8);
                    lo = l2.x | (static_cast<uint64_t>(l2.y) << 32);
                    hi = h2.x | (static_cast<uint64_t>(h2.y) << 32);
                }
                if (SB != 2 && mv.S < 256) {
                    uint64_t badm = bytes_ge(lo, mv.S);
                    if (gown < 8) badm &= (1ull << (8 * gown)) - 1;
                    if (badm) bad_symbol = true;
                }
                if (sm.surv) {
                    const uint32_t p2 = SB == 2 ? pk_gram(sm.pk, iw - b) : 0u;
                    if ((SB == 2 || SB == 8) && gown == 8 && iw + 7 + mm <= n) {
                        // all eight starts have their m-gram: branch-free
                        // lookups, one bit per start, combined in a tree
                        const uint32_t x0 = static_cast<uint32_t>(lo);
                        const uint32_t x1 = static_cast<uint32_t>(lo >> 32);
                        const uint32_t x2 = static_cast<uint32_t>(hi);
                        uint32_t bit[8];
                        if (SB == 8 && sm.survb) {
                            // bytes r, r + 1 of the window are the 2-gram
                            // index, and the offset into the byte table
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                const uint32_t idx = r < 3 ? __byte_perm(x0, 0u, 0x4400 | ((r + 1) << 4) | r)
                                                   : r == 3 ? __byte_perm(x0, x1, 0x0043) & 0xFFFFu
                                                   : r < 7 ? __byte_perm(x1, 0u, 0x4400 | ((r - 3) << 4) | (r - 4))
                                                           : __byte_perm(x1, x2, 0x0043) & 0xFFFFu;
                                bit[r] = pfsm_dyn_smem[idx];   // the table is at offset 0
                            }
                        } else {
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                const uint32_t t = SB == 2 ? p2 >> (2 * r)
                                                           : __funnelshift_r(r < 4 ? x0 : x1, r < 4 ? x1 : x2, 8 * (r & 3));
                                const uint32_t w = sm.surv[(t & mmask) >> 5];
                                // rotating w right by t (mod 32) brings the bit to bit 0
                                bit[r] = __funnelshift_r(w, w, t) & 1u;
                            }
                        }
                        const uint32_t k01 = bit[0] | (bit[1] << 1), k23 = bit[2] | (bit[3] << 1);
                        const uint32_t k45 = bit[4] | (bit[5] << 1), k67 = bit[6] | (bit[7] << 1);
                        keep = (k01 | (k23 << 2)) | ((k45 | (k67 << 2)) << 4);
                    } else {
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            const uint32_t i = iw + r;
                            if (static_cast<uint32_t>(r) < gown && i + mm <= n) {
                                const uint32_t idx = memo_index<SB>(lo, hi, p2, r, mm, mv.sbits, mmask);
                                if (!((sm.surv[idx >> 5] >> (idx & 31)) & 1u)) keep &= ~(1u << r);
                            }
                        }
                    }
                }
                live |= keep << (8 * g);
            }
        }
        // 1b. (lane-local settling kernels) the deep survival bitmap straight
        //     from each window's keep bits: the eight loads of a window are
        //     issued together (predicated on the start's bit), their 13-gram
        //     indices cut from the 32 symbols after the window start, and
        //     only the starts that pass both bitmaps are compacted below
        const bool deep_here = DEFER && KIND == 1 && SB == 2 && mv.surv2 != nullptr;
        if (deep_here && __any_sync(FULLMASK, live != 0)) {
#pragma unroll
            for (int g = 0; g < SPT / 8; ++g) {
                const uint32_t k8 = (live >> (8 * g)) & 0xFFu;
                if (!__any_sync(FULLMASK, k8 != 0)) continue;
                const uint32_t iw = wbase + 256u * g;
                const uint32_t q0 = k8 ? pk_gram(sm.pk, iw - b) : 0u;
                const uint32_t q1 = k8 ? pk_gram(sm.pk, iw - b + 16) : 0u;
                // starts whose m2-gram would pass the end of the text are
                // kept without a lookup (only near the end of the text)
                const uint32_t look = iw + 7 + m2 <= n ? k8
                                    : k8 & (iw + m2 > n ? 0u : (2u << (n - iw - m2)) - 1u);
                uint32_t word[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    word[r] = 0xFFFFFFFFu;   // no lookup: kept
                    if ((look >> r) & 1u) {
                        const uint32_t i2 = __funnelshift_r(q0, q1, 2 * r) & m2mask;
                        word[r] = ldg_u32_keep(mv.surv2 + (i2 >> 5), pol_keep) >> (i2 & 31);
                    }
                }
                uint32_t d8 = 0;
#pragma unroll
                for (int r = 0; r < 8; ++r) d8 |= (word[r] & 1u) << r;
                live &= ~((k8 & ~d8) << (8 * g));
            }
        }
        // 2. compact the surviving starts into this warp's list: a ballot
        //    per survivor rank when no lane holds more than two, else a
        //    prefix sum over the lanes' counts. A DFA without survival
        //    bitmaps keeps every start: its list is implicit, entry j being
        //    start j of the warp's range.
        uint32_t total = 0;
        const bool implicit = KIND == 0 && !sm.surv && !mv.surv2;
        const uint32_t wfirst = r0 + static_cast<uint32_t>(tid >> 5) * (32u * SPT);   // the warp's range
        if (implicit) {
            total = wfirst < own_end ? min(32u * SPT, own_end - wfirst) : 0u;
        } else if (__any_sync(FULLMASK, live != 0)) {
            if (!__any_sync(FULLMASK, __popc(live) > 2)) {
                uint32_t x = live;
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const uint32_t m = __ballot_sync(FULLMASK, x != 0);
                    if (x) {
                        const uint32_t r = __ffs(x) - 1;
                        x &= x - 1;
                        sm.list[total + __popc(m & lanemask_lt())] =
                            static_cast<uint16_t>(wbase + 256u * (r >> 3) + (r & 7u) - b);
                    }
                    total += __popc(m);
                }
            } else {
                const uint32_t c = __popc(live);
                uint32_t incl = c;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t v = __shfl_up_sync(FULLMASK, incl, d);
                    if (lane >= d) incl += v;
                }
                total = __shfl_sync(FULLMASK, incl, 31);
                uint32_t p = incl - c;
                uint32_t x = live;
                while (x) {
                    const uint32_t r = __ffs(x) - 1;
                    x &= x - 1;
                    if (PFSM_OK_IDX(p < static_cast<uint32_t>(WARP_LIST), ov.status))
                        sm.list[p] = static_cast<uint16_t>(wbase + 256u * (r >> 3) + (r & 7u) - b);
                    ++p;
                }
            }
            __syncwarp();
        }
        // 2b. (DFA, deferred deep filter) the previous round's candidates,
        //     then this round's loads, left in flight; a round with more
        //     than 32 candidates takes the steps below instead
        if (DEFER && KIND == 0 && mv.surv2) {
            dfa_consume<TAB_SMEM, OUTW>(ov, mv, tv, sm, pend, wq_n, sn, lane, pol_keep);
            if (total <= 32) {
                if (static_cast<uint32_t>(lane) < total) {
                    const uint32_t off = sm.list[lane];
                    pend.start = b + off;
                    pend.g0 = PT_WALK;
                    if (kk != 0 && b + off + kk <= n)
                        pend.g0 = sm.memo[SB == 2 ? pk_gram(sm.pk, off) & mask
                                                  : kgram_at<SB>(tv.sm, off, mv.k, mv.sbits, mask)];
                    pend.g1 = 1u;
                    pend.sh = 0u;
                    if (b + off + m2 <= n) {
                        uint32_t i2;
                        if (SB == 2) {
                            i2 = pk_gram(sm.pk, off) & m2mask;
                        } else if (SB == 8 && m2 <= 4) {
                            const uint8_t *q = tv.sm + off;
                            i2 = (q[0] | (q[1] << 8) | (q[2] << 16) | (static_cast<uint32_t>(q[3]) << 24)) & m2mask;
                        } else {
                            i2 = gram_at16<SB>(tv.sm, off, m2, mv.sbits, m2mask);
                        }
                        pend.g1 = ldg_u32_keep(mv.surv2 + (i2 >> 5), pol_keep);
                        pend.sh = i2 & 31u;
                    }
                    pend.on = true;
                }
                __syncwarp();
                continue;
            }
        }
        // 3a. deep survival bitmap (global memory, L2 resident). The list is
        //     taken DEEP_GROUP chunks of 32 at a time: every lane first issues
        //     the loads of all its chunks, then the chunks are consumed in
        //     order and the list compacted in place (an entry is written at
        //     or below its own position, so chunks not yet consumed are
        //     intact), so a warp waits for one L2 round trip per group
        //     instead of one per chunk.
        if (mv.surv2 && total && !deep_here) {
            uint32_t w = 0;
            for (uint32_t g0 = 0; g0 < total; g0 += 32 * DEEP_GROUP) {
                uint32_t word[DEEP_GROUP], bit[DEEP_GROUP];
#pragma unroll
                for (int c = 0; c < DEEP_GROUP; ++c) {
                    const uint32_t j = g0 + 32 * c + lane;
                    word[c] = 1u;
                    bit[c] = 0u;
                    if (j < total) {
                        const uint32_t off = sm.list[j];
                        if (b + off + m2 <= n) {
                            uint32_t i2;
                            if (SB == 2) {
                                i2 = pk_gram(sm.pk, off) & m2mask;
                            } else if (SB == 8 && m2 <= 4) {
                                // bytes off .. off + 3 (the staged tile has slack past its end)
                                const uint8_t *q = tv.sm + off;
                                i2 = (q[0] | (q[1] << 8) | (q[2] << 16) | (static_cast<uint32_t>(q[3]) << 24)) & m2mask;
                            } else {
                                i2 = gram_at16<SB>(tv.sm, off, m2, mv.sbits, m2mask);
                            }
                            word[c] = ldg_u32_keep(mv.surv2 + (i2 >> 5), pol_keep);
                            bit[c] = i2 & 31u;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < DEEP_GROUP; ++c) {
                    const uint32_t j = g0 + 32 * c + lane;
                    if (g0 + 32 * c >= total) break;   // warp-uniform
                    const bool keep = j < total && ((word[c] >> bit[c]) & 1u);
                    const uint32_t off = j < total ? sm.list[j] : 0u;
                    const uint32_t km = __ballot_sync(FULLMASK, keep);
                    __syncwarp();
                    if (keep) sm.list[w + __popc(km & lanemask_lt())] = static_cast<uint16_t>(off);
                    w += __popc(km);
                    __syncwarp();
                }
            }
            total = w;
        }
        // 3b'. lane-local settling: the entries are handed to lanes without
        //      a start; a warp whose lanes all hold one settles them. Starts
        //      too close to the end of the text for the second level go to
        //      the exact path at once.
        if (DEFER && KIND == 1 && SB == 2 && sm.band && settle_steps > 0 && mv.memox && total) {
            for (uint32_t j0 = 0; j0 < total;) {
                const uint32_t freem = __ballot_sync(FULLMASK, !pend.on);
                if (freem == 0) {
                    settle_lanes<KIND, TAB_SMEM, OUTW>(ov, mv, tv, sm, pend, wq_n, sn, lane, pol_keep,
                                                       settle_steps);
                    continue;
                }
                const uint32_t take = min(static_cast<uint32_t>(__popc(freem)), total - j0);
                bool near_end = false;
                uint32_t e = PT_SKIP, off = 0;
                if (!pend.on) {
                    const uint32_t r = __popc(freem & lanemask_lt());
                    if (r < take) {
                        off = sm.list[j0 + r];
                        if (b + off + kk + L2_SYMS < n) {
                            pend.start = b + off;
                            pend.g0 = pk_gram(sm.pk, off);
                            pend.g1 = pk_gram(sm.pk, off + 16);
                            pend.on = true;
                        } else {
                            near_end = true;
                            const uint32_t gram = pk_gram(sm.pk, off);
                            if (b + off + kk <= n) {
                                e = sm.memo[gram & mask];
                            } else if (mv.tail) {
                                const int jl = static_cast<int>(n - (b + off));
                                e = __ldg(mv.tail + tail_base(jl, mv.sbits) + (gram & ((1u << (jl * 2)) - 1)));
                            }
                            near_end = e != PT_SKIP;
                        }
                    }
                }
                j0 += take;
                const uint32_t nm = __ballot_sync(FULLMASK, near_end);
                if (nm) {
                    if (wq_n + 32 > static_cast<uint32_t>(WARP_QUEUE))
                        drain<KIND, TAB_SMEM, OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
                    if (near_end && PFSM_OK_IDX(wq_n + __popc(nm & lanemask_lt()) <
                                                    static_cast<uint32_t>(WARP_QUEUE), ov.status)) {
                        const uint32_t at = wq_n + __popc(nm & lanemask_lt());
                        sm.wq_start[at] = b + off;
                        sm.wq_info[at] = static_cast<uint16_t>(e);
                        queue_flag(sm.wq_flag, at, false);
                    }
                    wq_n += __popc(nm);
                    __syncwarp();
                }
            }
            __syncwarp();
            continue;
        }
        // 3b. every lane takes list entries: prefix table, settling, queue
        const bool settle = KIND == 1 && sm.band && settle_steps > 0 && total;
        if (settle) {
            sm.marks[lane] = 0;
            if (lane == 0) *sm.pcount = 0;
            __syncwarp();
        }
        for (uint32_t j0 = 0; j0 < total; j0 += 32) {
            const uint32_t j = j0 + lane;
            uint32_t e = PT_SKIP, off = 0;
            uint32_t r2 = L2_NO_REC;   // second-level record of this lane's start
            if (j < total) {
                off = implicit ? wfirst - b + j : sm.list[j];
                e = PT_WALK;
                if (kk != 0 && b + off + kk <= n) {
                    const uint32_t gram = SB == 2 ? pk_gram(sm.pk, off) : 0u;
                    const uint32_t gi = SB == 2 ? gram & mask : kgram_at<SB>(tv.sm, off, mv.k, mv.sbits, mask);
                    // an NFA record with survivors and no matches carries the
                    // start L2_SYMS symbols further through the second level:
                    // its set index is read beside the prefix entry
                    const bool l2 = KIND == 1 && SB == 2 && mv.memox && b + off + kk + L2_SYMS <= n;
                    const uint32_t x = l2 ? ldg_u16_keep(mv.memox + gi, pol_keep) : L2_NONE;
                    e = PFSM_OK_IDX(gi < mv.memo_n, ov.status) ? sm.memo[gi] : PT_SKIP;
                    if (l2 && x != L2_NONE) {
                        const uint32_t o2 = ldg_u16_keep(
                            mv.l2tab + x * L2_GRAMS + ((gram >> (2 * kk)) & (L2_GRAMS - 1)), pol_keep);
                        if (o2 == L2_EMPTY) e = PT_SKIP;   // nothing left: no match
                        else r2 = o2;
                    }
                } else if (kk != 0 && mv.tail) {
                    // fewer than k symbols left: their matches are the whole result
                    const int jl = static_cast<int>(n - (b + off));
                    const uint32_t jm = (1u << (jl * mv.sbits)) - 1;
                    e = __ldg(mv.tail + tail_base(jl, mv.sbits) +
                              ((SB == 2 ? pk_gram(sm.pk, off) : kgram_at<SB>(tv.sm, off, mv.k, mv.sbits, mask)) & jm));
                }
            }
            // a record without survivors (its matches end the instance) is
            // reported here instead of going through the queue
            {
                uint32_t pm_left = 0, pm_ptr = 0;
                // (a start with a second-level record has survivors)
                if (j < total && r2 == L2_NO_REC && e != PT_SKIP && e != PT_WALK &&
                    (KIND == 1 || (e & PT_REC))) {
                    const uint32_t ro = KIND == 1 ? e : (e & 0x7FFFu);
                    const uint32_t hdr = sm.pool[ro];
                    if ((hdr >> 16) == 0) {
                        pm_left = hdr & 0xFFFFu;
                        pm_ptr = ro + 1;
                        e = PT_SKIP;
                    }
                }
                if (__any_sync(FULLMASK, pm_left > 0))
                    emit_record_matches<OUTW>(pm_left, sm.pool, pm_ptr, b + off, sm.stage, sn, ov, tv, lane);
            }
            bool push = e != PT_SKIP;
            if (settle) {
                nfa_settle_chunk(mv, sm, tv, j0, total, e, r2, lane, settle_steps);
                push = j < total && marked(sm.marks, j);
            }
            const uint32_t pmask = __ballot_sync(FULLMASK, push);
            if (pmask) {
                // this warp's queue: drain it first when these would not fit
                if (wq_n + 32 > static_cast<uint32_t>(WARP_QUEUE))
                    drain<KIND, TAB_SMEM, OUTW>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
                if (push && PFSM_OK_IDX(wq_n + __popc(pmask & lanemask_lt()) < static_cast<uint32_t>(WARP_QUEUE),
                                        ov.status)) {
                    const uint32_t p = wq_n + __popc(pmask & lanemask_lt());
                    sm.wq_start[p] = b + off;
                    sm.wq_info[p] = static_cast<uint16_t>(e);
                    if (KIND == 1) queue_flag(sm.wq_flag, p, false);
                }
                wq_n += __popc(pmask);
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// `nw` = the warps that own per-warp regions (the layout's thread count / 32).
__device__ __forceinline__ Smem smem_regions(uint8_t *base, const ScanArgs &a, int wid, int nw) {
    Smem s;
    s.misc = reinterpret_cast<Misc *>(base + a.sm_misc);
    s.memo = a.memo_smem ? reinterpret_cast<const uint16_t *>(base + a.sm_memo) : a.memo;
    s.tab = reinterpret_cast<const uint16_t *>(base + a.sm_tab);
    s.wq_start = reinterpret_cast<uint32_t *>(base + a.sm_queue) + wid * WARP_QUEUE;
    s.wq_info = reinterpret_cast<uint16_t *>(base + a.sm_queue + nw * WARP_QUEUE * 4) +
                wid * WARP_QUEUE;
    s.wq_flag = reinterpret_cast<uint32_t *>(base + a.sm_queue + nw * WARP_QUEUE * 6) +
                wid * (WARP_QUEUE / 32);
    s.stage = reinterpret_cast<uint32_t *>(base + a.sm_stage) + wid * (4 * a.stage_n);
    s.slots = reinterpret_cast<uint16_t *>(base + a.sm_slots) + wid * (2 * NFA_SLOT * 32);
    s.coop = a.coop_smem ? reinterpret_cast<uint32_t *>(base + a.sm_coop) + wid * 2 * a.Wq
           : a.coop_g ? a.coop_g + (static_cast<size_t>(blockIdx.x) * nw + wid) * 2 * a.Wq
                      : nullptr;
    s.band = a.band_smem ? reinterpret_cast<const uint32_t *>(base + a.sm_band) : a.band;
    s.pk = reinterpret_cast<uint32_t *>(base + a.sm_pack);
    s.surv = a.surv ? reinterpret_cast<const uint32_t *>(base + a.sm_surv) : nullptr;
    s.survb = a.surv && a.surv_bytes ? base + a.sm_surv : nullptr;
    uint8_t *wl = base + a.sm_list + wid * WARP_LIST_BYTES;
    s.list = reinterpret_cast<uint16_t *>(wl);
    s.pairs = reinterpret_cast<uint32_t *>(wl + 2 * WARP_LIST);
    s.marks = reinterpret_cast<uint32_t *>(wl + 2 * WARP_LIST + 4 * SETTLE_PAIRS);
    s.pcount = s.marks + WARP_LIST / 32;
    s.pool = a.pool_smem ? reinterpret_cast<const uint32_t *>(base + a.sm_pool) : a.pool;
    return s;
}

__device__ __forceinline__ void stage_u16(uint16_t *dst, const uint16_t *src, uint32_t count,
                                          int tid, int nt) {
    const uint32_t words = (count + 1) / 2;
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = tid; i < words; i += nt) d[i] = __ldg(s + i);
}

// Moves the staged bytes buf[sh, sh + len) down to buf[0, len) (0 < sh < 16;
// buf is 16-byte aligned with room for len + 32 bytes). A tile of a text
// that does not start on a 16-byte boundary is copied by TMA from the
// boundary below it and realigned here. Every thread of the CTA calls it;
// it ends with a barrier.
__device__ __forceinline__ void realign_tile(uint8_t *buf, uint32_t sh, uint32_t len, int tid,
                                             int nt) {
    constexpr int PER = 4;   // output blocks per thread per chunk
    uint4 *b4 = reinterpret_cast<uint4 *>(buf);
    const uint32_t q = (len + 15) >> 4;
    const uint32_t ws = sh >> 2, bs = (sh & 3u) * 8u;
    for (uint32_t c0 = 0; c0 < q; c0 += PER * nt) {
        uint4 o[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t i = c0 + j * nt + tid;
            if (i < q) {
                const uint4 x = b4[i], y = b4[i + 1];
                // words ws .. ws + 4 of the eight words of x and y
                const uint32_t w0 = ws == 0 ? x.x : ws == 1 ? x.y : ws == 2 ? x.z : x.w;
                const uint32_t w1 = ws == 0 ? x.y : ws == 1 ? x.z : ws == 2 ? x.w : y.x;
                const uint32_t w2 = ws == 0 ? x.z : ws == 1 ? x.w : ws == 2 ? y.x : y.y;
                const uint32_t w3 = ws == 0 ? x.w : ws == 1 ? y.x : ws == 2 ? y.y : y.z;
                const uint32_t w4 = ws == 0 ? y.x : ws == 1 ? y.y : ws == 2 ? y.z : y.w;
                o[j].x = __funnelshift_r(w0, w1, bs);
                o[j].y = __funnelshift_r(w1, w2, bs);
                o[j].z = __funnelshift_r(w2, w3, bs);
                o[j].w = __funnelshift_r(w3, w4, bs);
            }
        }
        __syncthreads();   // this chunk's reads precede its writes; later
                           // chunks read only blocks this one does not write
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t i = c0 + j * nt + tid;
            if (i < q) b4[i] = o[j];
        }
    }
    __syncthreads();
}

// realign_tile for one warp that owns the buffer (the producer warp of the
// single-text kernel): the same chunked shift with warp synchronisation.
__device__ __forceinline__ void realign_tile_warp(uint8_t *buf, uint32_t sh, uint32_t len,
                                                  int lane) {
    constexpr int PER = 8;
    uint4 *b4 = reinterpret_cast<uint4 *>(buf);
    const uint32_t q = (len + 15) >> 4;
    const uint32_t ws = sh >> 2, bs = (sh & 3u) * 8u;
    for (uint32_t c0 = 0; c0 < q; c0 += PER * 32) {
        uint4 o[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t i = c0 + j * 32 + lane;
            if (i < q) {
                const uint4 x = b4[i], y = b4[i + 1];
                const uint32_t w0 = ws == 0 ? x.x : ws == 1 ? x.y : ws == 2 ? x.z : x.w;
                const uint32_t w1 = ws == 0 ? x.y : ws == 1 ? x.z : ws == 2 ? x.w : y.x;
                const uint32_t w2 = ws == 0 ? x.z : ws == 1 ? x.w : ws == 2 ? y.x : y.y;
                const uint32_t w3 = ws == 0 ? x.w : ws == 1 ? y.x : ws == 2 ? y.y : y.z;
                const uint32_t w4 = ws == 0 ? y.x : ws == 1 ? y.y : ws == 2 ? y.z : y.w;
                o[j].x = __funnelshift_r(w0, w1, bs);
                o[j].y = __funnelshift_r(w1, w2, bs);
                o[j].z = __funnelshift_r(w2, w3, bs);
                o[j].w = __funnelshift_r(w3, w4, bs);
            }
        }
        __syncwarp();   // this chunk's reads precede its writes
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint32_t i = c0 + j * 32 + lane;
            if (i < q) b4[i] = o[j];
        }
        __syncwarp();
    }
}

// Copies an NFA's band rows and prefix records into shared memory (either
// source may be null: that table is then read from global memory).
__device__ __forceinline__ void stage_nfa(uint8_t *base, uint32_t sm_band, uint32_t sm_pool,
                                          const uint32_t *band, int32_t Q,
                                          const uint32_t *pool, uint32_t pool_n, int tid,
                                          int nt) {
    if (band) {
        uint32_t *d = reinterpret_cast<uint32_t *>(base + sm_band);
        const int32_t words = Q + (Q + 31) / 32;
        for (int32_t i = tid; i < words; i += nt) d[i] = __ldg(band + i);
    }
    if (pool) {
        uint32_t *d = reinterpret_cast<uint32_t *>(base + sm_pool);
        for (uint32_t i = tid; i < pool_n; i += nt) d[i] = __ldg(pool + i);
    }
}

}  // namespace pfsm
