// PFSM scan kernels for sm_103a.
//
// One persistent CTA loops over text tiles. A tile owns the instances that
// start in [b, b + tile) and stages t[b, b + tile + halo) into shared memory
// with a 1-D bulk TMA copy (double buffered, evict-first in L2). Instances
// that are still alive past the staged halo continue on the global text:
// DFA instances are pushed to a carry queue drained by a second kernel
// (chained data partitioning, Sec. III.D.2), NFA instances continue in place
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
#include <cuda_runtime.h>
#include <stdint.h>

#include "pfsm_internal.h"

namespace pfsm {

#define FULLMASK 0xffffffffu

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
// Bounded wait on a bulk-copy barrier: gives up after ~2 s of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return true;
}

// Shared-memory control words of a CTA.
struct Misc {
    uint64_t bar[2];
    uint32_t q_count;
    uint32_t q_head;
    uint32_t abort;
    uint32_t pad;
};

// ------------------------------------------------------------ match output
// Per-warp staging of (start, end, state) triples; `sn` is warp-uniform.
__device__ __forceinline__ void stage_flush(uint32_t *buf, uint32_t &sn, const ScanArgs &a,
                                            int lane) {
    __syncwarp();
    if (sn == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.status[0], (unsigned long long)sn);
    base = __shfl_sync(FULLMASK, base, 0);
    const uint32_t words = 3 * sn;
    for (uint32_t w = lane; w < words; w += 32) {
        const unsigned long long idx = base + w / 3;
        if (idx < a.cap) a.out[base * 3 + w] = buf[w];
    }
    __syncwarp();
    sn = 0;
}

__device__ __forceinline__ void warp_emit(bool has, uint32_t s, uint32_t e, uint32_t st,
                                          uint32_t *buf, uint32_t &sn, const ScanArgs &a,
                                          int lane) {
    const uint32_t m = __ballot_sync(FULLMASK, has);
    if (m == 0) return;
    const uint32_t c = __popc(m);
    if (sn + c > STAGE) stage_flush(buf, sn, a, lane);
    if (has) {
        const uint32_t i = sn + __popc(m & lanemask_lt());
        buf[3 * i] = s;
        buf[3 * i + 1] = e;
        buf[3 * i + 2] = st;
    }
    sn += c;
}

// Direct append for the rare warp-cooperative path (divergent callers).
__device__ __forceinline__ void emit_direct(const ScanArgs &a, uint32_t s, uint32_t e,
                                            uint32_t st) {
    const unsigned long long idx = atomicAdd(&a.status[0], 1ull);
    if (idx < a.cap) {
        a.out[3 * idx] = s;
        a.out[3 * idx + 1] = e;
        a.out[3 * idx + 2] = st;
    }
}

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

// ------------------------------------------------------------ text access
struct TileView {
    const uint8_t *sm;   // staged bytes of [b, b + len)
    uint32_t b, len;
};

__device__ __forceinline__ uint32_t text_at(const ScanArgs &a, const TileView &tv,
                                            uint32_t pos) {
    const uint32_t rel = pos - tv.b;
    return rel < tv.len ? tv.sm[rel] : __ldg(a.text + pos);
}

// ------------------------------------------------------------ continuation: DFA
// Drains the work queue: lane-refill loop, one symbol per lane per iteration.
template <bool TAB_SMEM>
__device__ void drain_dfa(const ScanArgs &a, const TileView &tv, Misc *misc,
                          const uint32_t *queue, const uint16_t *tab_sm, uint32_t *stage,
                          uint32_t &sn, int lane, uint64_t pol_keep) {
    const uint32_t qn = misc->q_count;
    const uint32_t S = a.S;
    const uint32_t n = a.n;
    const uint32_t tile_end = tv.b + tv.len;
    bool act = false;
    bool gmode = false;   // past the staged text and the carry queue is full
    uint32_t start = 0, pos = 0, s = 0;
    while (true) {
        const bool need = !act;
        const uint32_t m = __ballot_sync(FULLMASK, need);
        if (m) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&misc->q_head, __popc(m));
            base = __shfl_sync(FULLMASK, base, 0);
            if (need) {
                const uint32_t qi = base + __popc(m & lanemask_lt());
                if (qi < qn) {
                    const uint32_t e = queue[qi];
                    start = tv.b + (e & 0xFFFFu);
                    const uint32_t info = e >> 16;
                    if (info == PT_WALK) {
                        s = a.q0;
                        pos = start;
                    } else {
                        s = info;
                        pos = start + a.k;
                    }
                    act = true;
                    gmode = false;
                }
            }
        }
        if (!__any_sync(FULLMASK, act)) break;
        bool hit = false;
        uint32_t hend = 0;
        if (act) {
            if (pos >= n) {
                act = false;
            } else if (pos >= tile_end && !gmode) {
                const uint32_t ci = atomicAdd(a.carry_n, 1u);
                if (ci < a.carry_cap) {
                    a.carry[3 * ci] = start;
                    a.carry[3 * ci + 1] = pos;
                    a.carry[3 * ci + 2] = s;
                    act = false;
                } else {
                    gmode = true;
                }
            }
            if (act) {
                const uint32_t c = text_at(a, tv, pos);
                uint16_t e = DEAD16;
                if (c < S) {
                    const uint32_t ix = s * S + c;
                    e = TAB_SMEM ? tab_sm[ix] : ldg_u16_keep(a.dtab + ix, pol_keep);
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
        warp_emit(hit, start, hend, s, stage, sn, a, lane);
    }
}

// ------------------------------------------------------------ continuation: NFA
// Warp-cooperative advance of one instance as a bitset over Q (lazy data
// partitioning: reads the global text once past the staged bytes).
__device__ void coop_run(const ScanArgs &a, const TileView &tv, uint32_t *bits0,
                         uint32_t *bits1, uint32_t start, uint32_t pos, int lane,
                         uint64_t pol_keep) {
    const uint32_t Wq = a.Wq, S = a.S, n = a.n;
    uint32_t *cur = bits0, *nxt = bits1;
    while (pos < n) {
        const uint32_t c = text_at(a, tv, pos);
        if (c >= S) break;
        for (uint32_t w = lane; w < Wq; w += 32) {
            uint32_t x = cur[w];
            while (x) {
                const uint32_t bit = __ffs(x) - 1;
                x &= x - 1;
                const uint32_t q = w * 32 + bit;
                const uint32_t lo = ldg_u32_keep(a.off + q * S + c, pol_keep);
                const uint32_t hi = ldg_u32_keep(a.off + q * S + c + 1, pol_keep);
                for (uint32_t e = lo; e < hi; ++e) {
                    const uint32_t t = ldg_u16_keep(a.tgt + e, pol_keep);
                    const uint32_t ts = t & 0x7FFFu;
                    const uint32_t mb = 1u << (ts & 31);
                    const uint32_t old = atomicOr(&nxt[ts >> 5], mb);
                    if ((t & FINAL_BIT) && !(old & mb)) emit_direct(a, start, pos, ts);
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

enum : uint32_t { MODE_LANE = 0, MODE_COOP_SLOT = 1, MODE_COOP_POOL = 2 };

__device__ void drain_nfa(const ScanArgs &a, const TileView &tv, Misc *misc,
                          const uint32_t *queue, uint16_t *slots, uint32_t *coop,
                          uint32_t *stage, uint32_t &sn, int lane, uint64_t pol_keep) {
    const uint32_t qn = misc->q_count;
    const uint32_t S = a.S, n = a.n;
    constexpr int C = NFA_SLOT;
#define SLOT(sel, i) slots[((sel) * C + (i)) * 32 + lane]
    bool act = false;
    uint32_t start = 0, pos = 0, cnt = 0, cb = 0, mode = MODE_LANE;
    uint32_t pm_left = 0, pm_ptr = 0, cptr = 0;
    while (true) {
        const bool need = !act;
        const uint32_t m = __ballot_sync(FULLMASK, need);
        if (m) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&misc->q_head, __popc(m));
            base = __shfl_sync(FULLMASK, base, 0);
            if (need) {
                const uint32_t qi = base + __popc(m & lanemask_lt());
                if (qi < qn) {
                    const uint32_t e = queue[qi];
                    start = tv.b + (e & 0xFFFFu);
                    const uint32_t info = e >> 16;
                    act = true;
                    mode = MODE_LANE;
                    pm_left = 0;
                    if (info == PT_WALK) {
                        SLOT(cb, 0) = static_cast<uint16_t>(a.q0);
                        cnt = 1;
                        pos = start;
                    } else {
                        const uint32_t ro = ldg_u32_keep(a.rec_off + info, pol_keep);
                        const uint32_t w0 = ldg_u32_keep(a.pool + ro, pol_keep);
                        const uint32_t nm = w0 & 0xFFFFu, ns = w0 >> 16;
                        pm_left = nm;
                        pm_ptr = ro + 1;
                        pos = start + a.k;
                        if (ns > static_cast<uint32_t>(C)) {
                            mode = MODE_COOP_POOL;
                            cptr = ro + 1 + nm;
                            cnt = ns;
                        } else {
                            for (uint32_t i = 0; i < ns; ++i)
                                SLOT(cb, i) = static_cast<uint16_t>(
                                    ldg_u32_keep(a.pool + ro + 1 + nm + i, pol_keep));
                            cnt = ns;
                        }
                    }
                }
            }
        }
        if (!__any_sync(FULLMASK, act)) break;

        // matches inside the first k steps, from the prefix record
        while (__any_sync(FULLMASK, pm_left > 0)) {
            const bool has = pm_left > 0;
            uint32_t o = 0, f = 0;
            if (has) {
                const uint32_t w = ldg_u32_keep(a.pool + pm_ptr, pol_keep);
                o = w >> 16;
                f = w & 0xFFFFu;
                ++pm_ptr;
                --pm_left;
            }
            warp_emit(has, start, start + o, f, stage, sn, a, lane);
        }
        if (act && mode == MODE_LANE && cnt == 0) act = false;

        // one symbol for every lane-held instance
        bool anyfin = false;
        if (act && mode == MODE_LANE) {
            if (pos >= n) {
                act = false;
            } else {
                const uint32_t c = text_at(a, tv, pos);
                if (c >= S) {
                    act = false;
                } else {
                    uint32_t ncnt = 0;
                    bool ovf = false;
                    for (uint32_t i = 0; i < cnt && !ovf; ++i) {
                        const uint32_t q = SLOT(cb, i) & 0x7FFFu;
                        const uint32_t lo = ldg_u32_keep(a.off + q * S + c, pol_keep);
                        const uint32_t hi = ldg_u32_keep(a.off + q * S + c + 1, pol_keep);
                        for (uint32_t e = lo; e < hi; ++e) {
                            const uint16_t t = ldg_u16_keep(a.tgt + e, pol_keep);
                            const uint32_t ts = t & 0x7FFFu;
                            bool dup = false;
                            for (uint32_t j = 0; j < ncnt; ++j)
                                if ((SLOT(cb ^ 1, j) & 0x7FFFu) == ts) {
                                    dup = true;
                                    break;
                                }
                            if (dup) continue;
                            if (ncnt == static_cast<uint32_t>(C)) {
                                ovf = true;
                                break;
                            }
                            SLOT(cb ^ 1, ncnt) = t;
                            ++ncnt;
                            anyfin |= (t & FINAL_BIT) != 0;
                        }
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
        if (__any_sync(FULLMASK, anyfin)) {
            for (uint32_t j = 0; j < static_cast<uint32_t>(C); ++j) {
                const bool has = anyfin && j < cnt && (SLOT(cb, j) & FINAL_BIT);
                warp_emit(has, start, pos, has ? (SLOT(cb, j) & 0x7FFFu) : 0u, stage, sn, a,
                          lane);
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
            uint32_t *b0 = coop, *b1 = coop + a.Wq;
            for (uint32_t w = lane; w < static_cast<uint32_t>(a.Wq); w += 32) {
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
                    const uint32_t q = ldg_u32_keep(a.pool + cpt + i, pol_keep);
                    atomicOr(&b0[q >> 5], 1u << (q & 31));
                }
            }
            __syncwarp();
            coop_run(a, tv, b0, b1, cs, cp, lane, pol_keep);
            if (lane == src) {
                act = false;
                mode = MODE_LANE;
            }
        }
    }
#undef SLOT
}

// ------------------------------------------------------------ the tile kernel
template <int KIND, int SB, bool TAB_SMEM>
__global__ void __launch_bounds__(512) scan_tiles(const ScanArgs a) {
    extern __shared__ __align__(128) uint8_t sm[];
    constexpr int SPT = 8;   // starts per thread per filter round
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int NT = blockDim.x;
    Misc *misc = reinterpret_cast<Misc *>(sm + a.sm_misc);
    uint16_t *memo_sm = reinterpret_cast<uint16_t *>(sm + a.sm_memo);
    uint16_t *tab_sm = reinterpret_cast<uint16_t *>(sm + a.sm_tab);
    uint8_t *text_sm = sm + a.sm_text;
    uint32_t *queue = reinterpret_cast<uint32_t *>(sm + a.sm_queue);
    uint32_t *stage = reinterpret_cast<uint32_t *>(sm + a.sm_stage) + wid * (3 * STAGE);
    uint16_t *slots = reinterpret_cast<uint16_t *>(sm + a.sm_slots) + wid * (2 * NFA_SLOT * 32);
    uint32_t *coop = reinterpret_cast<uint32_t *>(sm + a.sm_coop) + wid * (2 * a.Wq);
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    // tables into shared memory
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(a.memo);
        uint32_t *dst = reinterpret_cast<uint32_t *>(memo_sm);
        const uint32_t words = (a.memo_n + 1) / 2;
        for (uint32_t i = tid; i < words; i += NT) dst[i] = __ldg(src + i);
        if (TAB_SMEM) {
            const uint32_t tw = (static_cast<uint32_t>(a.Q) * a.S + 1) / 2;
            const uint32_t *ts = reinterpret_cast<const uint32_t *>(a.dtab);
            uint32_t *td = reinterpret_cast<uint32_t *>(tab_sm);
            for (uint32_t i = tid; i < tw; i += NT) td[i] = __ldg(ts + i);
        }
    }
    if (tid == 0) {
        mbar_init(&misc->bar[0], 1);
        mbar_init(&misc->bar[1], 1);
        misc->q_count = 0;
        misc->q_head = 0;
        misc->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t sn = 0;   // staged matches of this warp
    bool bad_symbol = false;
    const uint32_t n = a.n;

    auto issue = [&](uint32_t tile, int buf) {
        const uint32_t b = tile * a.tile;
        const uint32_t len = min(a.tile + a.halo, n - b);
        const uint32_t len16 = len & ~15u;
        if (a.aligned && len16) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&misc->bar[buf], len16);
            tma_load_1d(text_sm + buf * a.text_buf, a.text + b, len16, &misc->bar[buf],
                        pol_stream);
        }
    };

    uint32_t it = 0;
    if (tid == 0 && blockIdx.x < a.ntiles) issue(blockIdx.x, 0);
    for (uint32_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        const uint32_t b = tile * a.tile;
        const uint32_t len = min(a.tile + a.halo, n - b);
        const uint32_t len16 = len & ~15u;
        uint8_t *tsm = text_sm + buf * a.text_buf;
        // prefetch the next tile into the other buffer (freed at the end of
        // the previous iteration)
        if (tid == 0 && tile + gridDim.x < a.ntiles) issue(tile + gridDim.x, buf ^ 1);
        if (a.aligned && len16) {
            if (!mbar_wait_bounded(&misc->bar[buf], parity)) misc->abort = 1;
            for (uint32_t i = len16 + tid; i < len; i += NT) tsm[i] = a.text[b + i];
        } else {
            for (uint32_t i = tid; i < len; i += NT) tsm[i] = a.text[b + i];
        }
        __syncthreads();
        if (misc->abort) break;
        const TileView tv{tsm, b, len};

        // ---------------- filter phase over the tile's own starts
        const uint32_t own_end = min(b + a.tile, n);
        const uint32_t kk = static_cast<uint32_t>(a.k);
        const uint32_t mask = (a.k * a.sbits >= 32) ? 0xFFFFFFFFu : ((1u << (a.k * a.sbits)) - 1);
        const uint32_t round = SPT * NT;
        for (uint32_t r0 = b; r0 < own_end; r0 += round) {
            if (misc->q_count + round > a.qcap) {
                if (KIND == 0)
                    drain_dfa<TAB_SMEM>(a, tv, misc, queue, tab_sm, stage, sn, lane, pol_keep);
                else
                    drain_nfa(a, tv, misc, queue, slots, coop, stage, sn, lane, pol_keep);
                __syncthreads();
                if (tid == 0) {
                    misc->q_count = 0;
                    misc->q_head = 0;
                }
                __syncthreads();
            }
            const uint32_t i0 = r0 + SPT * tid;
            uint32_t pm = 0;
            uint32_t ent[SPT];
#pragma unroll
            for (int r = 0; r < SPT; ++r) ent[r] = 0;
            if (i0 < own_end) {
                const uint8_t *tp = tsm + (i0 - b);
                const uint2 l2 = *reinterpret_cast<const uint2 *>(tp);
                const uint2 h2 = *reinterpret_cast<const uint2 *>(tp + 8);
                const uint64_t lo = l2.x | (static_cast<uint64_t>(l2.y) << 32);
                const uint64_t hi = h2.x | (static_cast<uint64_t>(h2.y) << 32);
                const uint32_t nown = min(static_cast<uint32_t>(SPT), own_end - i0);
                if (a.S < 256) {
                    uint64_t badm = bytes_ge(lo, a.S);
                    if (nown < 8) badm &= (1ull << (8 * nown)) - 1;
                    if (badm) bad_symbol = true;
                }
                const uint32_t p2 = SB == 2 ? (pack2(lo) | (pack2(hi) << 16)) : 0u;
#pragma unroll
                for (int r = 0; r < SPT; ++r) {
                    if (static_cast<uint32_t>(r) < nown) {
                        const uint32_t i = i0 + r;
                        if (kk == 0 || i + kk > n) {
                            ent[r] = PT_WALK;
                            pm |= 1u << r;
                        } else {
                            const uint32_t idx = memo_index<SB>(lo, hi, p2, r, a.k, a.sbits, mask);
                            const uint16_t e = memo_sm[idx];
                            if (e != PT_SKIP) {
                                ent[r] = e;
                                pm |= 1u << r;
                            }
                        }
                    }
                }
            }
            // warp-aggregated append to the CTA work queue
            const uint32_t c = __popc(pm);
            if (__ballot_sync(FULLMASK, c != 0)) {
                uint32_t incl = c;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t v = __shfl_up_sync(FULLMASK, incl, d);
                    if (lane >= d) incl += v;
                }
                const uint32_t wtot = __shfl_sync(FULLMASK, incl, 31);
                uint32_t wbase = 0;
                if (lane == 31) wbase = atomicAdd(&misc->q_count, wtot);
                wbase = __shfl_sync(FULLMASK, wbase, 31);
                uint32_t p = wbase + incl - c;
#pragma unroll
                for (int r = 0; r < SPT; ++r)
                    if (pm >> r & 1u) queue[p++] = (i0 + r - b) | (ent[r] << 16);
            }
            __syncthreads();
        }
        // ---------------- continuation phase
        if (KIND == 0)
            drain_dfa<TAB_SMEM>(a, tv, misc, queue, tab_sm, stage, sn, lane, pol_keep);
        else
            drain_nfa(a, tv, misc, queue, slots, coop, stage, sn, lane, pol_keep);
        __syncthreads();
        if (tid == 0) {
            misc->q_count = 0;
            misc->q_head = 0;
        }
        __syncthreads();
    }
    stage_flush(stage, sn, a, lane);
    if (bad_symbol) atomicOr(&a.status[1], ERR_SYMBOL);
    if (tid == 0 && misc->abort) atomicOr(&a.status[1], ERR_TIMEOUT);
    // a tile whose copy timed out may still have one in flight: wait for it
    // (bounded) before the CTA's shared memory is released
    if (tid == 0 && misc->abort) {
        mbar_wait_bounded(&misc->bar[0], 0);
        mbar_wait_bounded(&misc->bar[1], 0);
    }
}

// ------------------------------------------------------------ DFA carry queue
// Continues instances that outlived their tile's staged text, reading the
// text from global memory (chained data partitioning).
__global__ void __launch_bounds__(256) carry_dfa(const ScanArgs a) {
    const uint32_t nc = min(*a.carry_n, a.carry_cap);
    const uint64_t pol_keep = policy_evict_last();
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
         idx += gridDim.x * blockDim.x) {
        const uint32_t start = a.carry[3 * idx];
        uint32_t pos = a.carry[3 * idx + 1];
        uint32_t s = a.carry[3 * idx + 2];
        while (pos < a.n) {
            const uint32_t c = __ldg(a.text + pos);
            if (c >= static_cast<uint32_t>(a.S)) break;
            const uint16_t e = ldg_u16_keep(a.dtab + s * a.S + c, pol_keep);
            if (e == DEAD16) break;
            s = e & 0x7FFFu;
            if (e & FINAL_BIT) emit_direct(a, start, pos, s);
            ++pos;
        }
    }
}

// ------------------------------------------------------------ host helpers
uint32_t layout_smem(ScanArgs &a, int kind, int threads, int spt) {
    const int nw = threads / 32;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) & ~(align - 1);
        const uint32_t r = o;
        o += bytes;
        return r;
    };
    a.sm_misc = take(sizeof(Misc), 16);
    a.sm_memo = take(((a.memo_n + 1) / 2) * 4 + 4, 16);
    a.sm_tab = take(a.tab_smem ? ((static_cast<uint32_t>(a.Q) * a.S + 1) / 2) * 4 : 0, 16);
    a.sm_text = take(2 * a.text_buf, 128);
    a.sm_queue = take(a.qcap * 4, 16);
    a.sm_stage = take(nw * STAGE * 12, 16);
    a.sm_slots = take(kind == 1 ? nw * 2 * NFA_SLOT * 32 * 2 : 0, 16);
    a.sm_coop = take(kind == 1 ? nw * 2 * a.Wq * 4 : 0, 16);
    (void)spt;
    return (o + 127) & ~127u;
}

template <int KIND, int SB, bool TAB>
static cudaError_t launch_t(const ScanArgs &a, int threads, int grid, uint32_t smem,
                            cudaStream_t s) {
    auto k = scan_tiles<KIND, SB, TAB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KIND, bool TAB>
static cudaError_t launch_sb(const ScanArgs &a, int threads, int grid, uint32_t smem,
                             cudaStream_t s) {
    if (a.k > 0 && a.sbits == 2) return launch_t<KIND, 2, TAB>(a, threads, grid, smem, s);
    if (a.k > 0 && a.sbits == 8) return launch_t<KIND, 8, TAB>(a, threads, grid, smem, s);
    return launch_t<KIND, 0, TAB>(a, threads, grid, smem, s);
}

cudaError_t launch_scan(const ScanArgs &a, int kind, int threads, int grid, cudaStream_t s) {
    ScanArgs c = a;
    const uint32_t smem = layout_smem(c, kind, threads, 8);
    if (kind == 0) {
        if (c.tab_smem) return launch_sb<0, true>(c, threads, grid, smem, s);
        return launch_sb<0, false>(c, threads, grid, smem, s);
    }
    return launch_sb<1, false>(c, threads, grid, smem, s);
}

cudaError_t launch_carry(const ScanArgs &a, int grid, cudaStream_t s) {
    carry_dfa<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KIND, int SB, bool TAB>
static int occ_t(int threads, uint32_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(scan_tiles<KIND, SB, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_tiles<KIND, SB, TAB>, threads,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

int max_ctas_per_sm(int kind, int sbits, int threads, uint32_t smem, bool tab_smem) {
    const int sb = sbits == 2 ? 2 : (sbits == 8 ? 8 : 0);
    if (kind == 0) {
        if (tab_smem) {
            if (sb == 2) return occ_t<0, 2, true>(threads, smem);
            if (sb == 8) return occ_t<0, 8, true>(threads, smem);
            return occ_t<0, 0, true>(threads, smem);
        }
        if (sb == 2) return occ_t<0, 2, false>(threads, smem);
        if (sb == 8) return occ_t<0, 8, false>(threads, smem);
        return occ_t<0, 0, false>(threads, smem);
    }
    if (sb == 2) return occ_t<1, 2, false>(threads, smem);
    if (sb == 8) return occ_t<1, 8, false>(threads, smem);
    return occ_t<1, 0, false>(threads, smem);
}

}  // namespace pfsm
