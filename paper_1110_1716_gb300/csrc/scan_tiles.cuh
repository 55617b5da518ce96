// The single-text scan kernel and its launch helpers, as templates over the
// starts each thread takes per filter round (SPT). scan_kernels.cu
// instantiates SPT = 32 (long texts), scan_kernels_spt8.cu SPT = 8 (short
// texts: four times the warps for the same text).
#pragma once

#include "scan_device.cuh"

namespace pfsm {

// ------------------------------------------------------------ single-text kernel
// Long texts (SPT = 32, many tiles per CTA) run a producer/consumer pipeline.
// Warps 0 .. NC/32 - 1 are consumers (filter, settling, queues; NC =
// blockDim.x - 32), the last warp is the producer. The producer copies the
// CTA's tiles into a.nbuf (3) buffers by TMA, realigns and packs each one and
// releases it to the consumers (mbarrier `ready`); every consumer warp
// releases a buffer when it is done with it (`empty`, one arrival per warp),
// and the producer refills it a.nbuf tiles on. No CTA-wide barrier
// holds the warps between tiles: a warp that finished its part of a tile
// starts on the next one.
//
// Short texts (SPT = 8) give a CTA one or two tiles, where a pipeline has
// nothing to overlap and the producer warp's registers would cost a CTA per
// SM: every warp filters, two buffers alternate and the CTA synchronises once
// per tile. Every wait is bounded (2 s) in both forms.
template <int KIND, int SB, bool TAB_SMEM, int SPT>
__global__ void __launch_bounds__(SPT == 8 || KIND == 1 ? 512 : 544, 1) scan_tiles(const ScanArgs a) {
    constexpr bool PIPE = SPT != 8;
    // lane-held deferral (NFA settling, DFA deep-bitmap loads): every
    // single-text kernel but the DFA one for short texts, which keeps its
    // registers for a third CTA per SM
    constexpr bool DEFER = KIND == 1 || SPT != 8;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (PIPE ? (a.nbuf < 2 || a.nbuf > kTileBufs) : a.nbuf != 2) {   // the layout's buffers
        if (tid == 0) atomicOr(&a.status[1], ERR_SYMBOL);
        return;
    }
    const int NT = blockDim.x;
    const int NC = PIPE ? NT - 32 : NT;   // consumer threads
    const int ncw = NC >> 5;              // consumer warps
    const bool producer = PIPE && wid == ncw;
    const Smem sm = smem_regions(smem, a, producer ? 0 : wid, ncw);
    Misc *misc = sm.misc;
    uint8_t *text_sm = smem + a.sm_text;
    uint32_t *pk_sm = reinterpret_cast<uint32_t *>(smem + a.sm_pack);
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const OView ov{a.out, a.cap, a.status, nullptr, a.carry, a.carry_n, a.carry_cap, a.stage_n,
                   a.cpool, a.cpool_cap, KIND == 1 ? a.tile : 0u, a.halo};
    const MView mv{a.Q, a.S, a.q0, a.k, a.sbits, a.Wq, a.surv_m, a.surv2_m, a.surv2, a.dtab, a.off, a.tgt,
                   a.tail, a.ecl_off, a.ecl_tgt, a.l2tab, a.pool2, a.memox, a.status, a.pool_n,
                   a.memo_n};

    // Tables that go to shared memory as they are (prefix table, DFA table,
    // NFA band rows, records, survival bitmap) arrive by 1-D bulk copies
    // that one thread issues, completing on misc->bar[1]. Their device
    // sections start on 256-byte boundaries and are padded to them, so each
    // copy is rounded up to whole 16-byte blocks (the shared-memory regions
    // are rounded up the same way).
    auto r16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    const uint32_t b_memo = a.memo_smem ? r16(((a.memo_n + 1) / 2) * 4) : 0u;
    const uint32_t b_tab = TAB_SMEM ? r16(((static_cast<uint32_t>(a.Q) * a.S + 1) / 2) * 4) : 0u;
    const uint32_t b_band = KIND == 1 && a.band_smem
                                ? r16(static_cast<uint32_t>(a.Q + (a.Q + 31) / 32) * 4) : 0u;
    const uint32_t b_pool = a.pool_smem ? r16(a.pool_n * 4) : 0u;
    const uint32_t b_surv = a.surv && !a.surv_bytes ? r16(a.surv_words * 4) : 0u;
    const uint32_t b_all = b_memo + b_tab + b_band + b_pool + b_surv;
    if (tid == 0 && b_all) {
        mbar_init(&misc->bar[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&misc->bar[1], b_all);
        if (b_memo) tma_load_1d(smem + a.sm_memo, a.memo, b_memo, &misc->bar[1], pol_keep);
        if (b_tab) tma_load_1d(smem + a.sm_tab, a.dtab, b_tab, &misc->bar[1], pol_keep);
        if (b_band) tma_load_1d(smem + a.sm_band, a.band, b_band, &misc->bar[1], pol_keep);
        if (b_pool) tma_load_1d(smem + a.sm_pool, a.pool, b_pool, &misc->bar[1], pol_keep);
        if (b_surv) tma_load_1d(smem + a.sm_surv, a.surv, b_surv, &misc->bar[1], pol_keep);
    }
    if (a.surv && a.surv_bytes) {
        // one byte (0 or 1) per m-gram: word i of the bitmap gives bytes
        // 32 i .. 32 i + 31, written as eight words of four bytes
        uint32_t *d = reinterpret_cast<uint32_t *>(smem + a.sm_surv);
        for (uint32_t i = tid; i < 8 * a.surv_words; i += NT) {
            const uint32_t nib = (__ldg(a.surv + (i >> 3)) >> (4 * (i & 7))) & 0xFu;
            d[i] = (nib & 1u) | ((nib & 2u) << 7) | ((nib & 4u) << 14) | ((nib & 8u) << 21);
        }
    }

    if (tid == 0) {
        for (int i = 0; i < kTileBufs; ++i) {
            mbar_init(&misc->full[i], 1);
            mbar_init(&misc->ready[i], 1);
            mbar_init(&misc->empty[i], static_cast<uint32_t>(ncw));
        }
        misc->q_count = 0;
        misc->q_head = 0;
        misc->abort = 0;
        misc->busy = 0;
        fence_mbar_init();
    }
    __syncthreads();   // barriers initialised, the byte table expanded
    const uint32_t n = a.n;
    const uint32_t nb = a.nbuf;   // staged tile buffers, <= kTileBufs
    // this CTA's k-th tile is blockIdx.x + k * gridDim.x
    const uint32_t my_tiles = blockIdx.x < a.ntiles ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0u;
    bool bad_symbol = false;
    // tile k into buffer k % nb: one bulk copy from the 16-byte boundary at
    // or below its first byte (a 16-byte block never crosses a page, so the
    // bytes around the text that it covers are readable)
    auto issue = [&](uint32_t k) {
        const uint32_t tile = blockIdx.x + k * gridDim.x;
        const int buf = static_cast<int>(k % nb);
        const uint32_t b = tile * a.tile;
        const uint32_t len = min(a.tile + a.halo, n - b);
        const uint32_t bytes = (a.shift + len + 15) & ~15u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&misc->full[buf], bytes);
        tma_load_1d(text_sm + buf * a.text_buf,
                    reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(a.text) + b - a.shift),
                    bytes, &misc->full[buf], pol_stream);
    };
    // short texts: the first tile's copy goes out with the tables' copies
    // still in flight, so the two round trips overlap
    if constexpr (!PIPE) {
        if (tid == 0 && my_tiles > 0) issue(0);
    }
    if (b_all) {
        // the bulk copies of the tables (bounded wait; on a timeout the
        // CTA waits once more for them and for a tile copy it issued,
        // bounded, and leaves)
        if (tid == 0 && !mbar_wait_bounded(&misc->bar[1], 0)) misc->abort = 2;
        __syncthreads();
        if (misc->abort == 2) {
            if (tid == 0) {
                atomicOr(&a.status[1], ERR_TIMEOUT);
                mbar_wait_bounded(&misc->bar[1], 0);
                if (!PIPE && my_tiles > 0) mbar_wait_bounded(&misc->full[0], 0);
            }
            return;
        }
    }
    uint32_t sn = 0;
    uint32_t wq_n = 0;   // entries in this warp's queue
    Pend pend{0u, 0u, 0u, 0u, false};   // the start this lane holds (lane-local settling,
                                        // or a DFA candidate whose loads are in flight)
    uint32_t abort_at = ~0u;   // CTA-synchronous form: the tile whose copy failed

    if constexpr (PIPE) {
        if (producer) {
            // Two duties, polled without blocking so that neither waits on
            // the other: a tile whose copy landed is realigned, packed and
            // handed over at once; a buffer every consumer warp released is
            // refilled at once. A fast warp can thus run a whole tile ahead
            // of the slowest one.
            bool ok = true;
            uint32_t issued = 0, prepped = 0;   // copies issued / tiles handed over
            for (; issued < my_tiles && issued < nb; ++issued)
                if (lane == 0) issue(issued);
            uint64_t idle_since = global_ns();
            while (prepped < my_tiles) {
                bool progress = false;
                const int buf = static_cast<int>(prepped % nb);
                if (prepped < issued &&
                    __all_sync(0xffffffffu, mbar_test_wait(&misc->full[buf], (prepped / nb) & 1))) {
                    const uint32_t tile = blockIdx.x + prepped * gridDim.x;
                    const uint32_t b = tile * a.tile;
                    const uint32_t len = min(a.tile + a.halo, n - b);
                    uint8_t *tsm = text_sm + buf * a.text_buf;
                    if (a.shift) realign_tile_warp(tsm, a.shift, len, lane);
                    if (SB == 2)
                        pack_tile(tsm, pk_sm + buf * a.pk_words, len, min(b + a.tile, n) - b,
                                  static_cast<uint32_t>(a.S), bad_symbol, lane, 32);
                    // the realigned bytes are rewritten by a later bulk copy
                    if (a.shift) fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0 && !a.hold_tiles) mbar_arrive(&misc->ready[buf]);
                    ++prepped;
                    progress = true;
                }
                // tile `issued` goes to the buffer of tile issued - nb once
                // every consumer warp is done with that tile
                if (issued < my_tiles &&
                    __all_sync(0xffffffffu, mbar_test_wait(&misc->empty[issued % nb],
                                                           (issued / nb - 1) & 1))) {
                    if (lane == 0) issue(issued);
                    ++issued;
                    progress = true;
                }
                if (progress || *reinterpret_cast<volatile uint32_t *>(&misc->busy) != 0) {
                    idle_since = global_ns();
                } else {
                    // give up after 2 s without progress (one decision per warp)
                    if (__shfl_sync(0xffffffffu, global_ns() - idle_since > 2000000000ull ? 1 : 0, 0)) {
                        ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            if (!ok && lane == 0) {
                misc->abort = 1;
                atomicOr(&a.status[1], ERR_TIMEOUT);
                // copies still in flight: wait for them (bounded) before exit
                for (uint32_t t = prepped; t < issued; ++t)
                    mbar_wait_bounded(&misc->full[t % nb], (t / nb) & 1);
            }
            if (bad_symbol) atomicOr(&a.status[1], ERR_SYMBOL);
            return;
        }
        Smem smk = sm;
        for (uint32_t k = 0; k < my_tiles; ++k) {
            const int buf = static_cast<int>(k % nb);
            const uint32_t tile = blockIdx.x + k * gridDim.x;
            const uint32_t b = tile * a.tile;
            const uint32_t len = min(a.tile + a.halo, n - b);
            const bool go = mbar_wait_live(&misc->ready[buf], (k / nb) & 1, &misc->busy) &&
                            !*reinterpret_cast<volatile uint32_t *>(&misc->abort);
            if (!__all_sync(0xffffffffu, go)) {
                if (lane == 0) atomicOr(&a.status[1], ERR_TIMEOUT);
                break;
            }
            smk.pk = pk_sm + buf * a.pk_words;
            const TileView tv{text_sm + buf * a.text_buf, a.text, b, len, n, 0u, 0u};
            process_tile<KIND, SB, TAB_SMEM, 3, SPT, DEFER>(ov, mv, tv, smk, min(b + a.tile, n), wq_n,
                                                                 sn, bad_symbol, pol_keep,
                                                                 static_cast<uint32_t>(a.settle_steps), NC,
                                                                 pend);
            __syncwarp();
            if (lane == 0) mbar_arrive(&misc->empty[buf]);
        }
    } else {
        for (uint32_t k = 0; k < my_tiles; ++k) {
            const int buf = static_cast<int>(k & 1);
            const uint32_t tile = blockIdx.x + k * gridDim.x;
            const uint32_t b = tile * a.tile;
            const uint32_t len = min(a.tile + a.halo, n - b);
            uint8_t *tsm = text_sm + buf * a.text_buf;
            // the other buffer's tile was finished by every warp before the
            // barrier that ended the previous iteration
            if (tid == 0 && k + 1 < my_tiles) issue(k + 1);
            if (!mbar_wait_bounded(&misc->full[buf], (k >> 1) & 1)) misc->abort = 1;
            if (a.shift) realign_tile(tsm, a.shift, len, tid, NT);   // ends with a barrier
            else __syncthreads();
            if (misc->abort) { abort_at = k; break; }
            if (SB == 2) {   // 2-bit symbols: pack the tile once for every gram read
                pack_tile(tsm, pk_sm, len, min(b + a.tile, n) - b, static_cast<uint32_t>(a.S),
                          bad_symbol, tid, NT);
                __syncthreads();
            }
            const TileView tv{tsm, a.text, b, len, n, 0u, 0u};
            process_tile<KIND, SB, TAB_SMEM, 3, SPT, DEFER>(ov, mv, tv, sm, min(b + a.tile, n), wq_n,
                                                                 sn, bad_symbol, pol_keep,
                                                                 static_cast<uint32_t>(a.settle_steps), NT,
                                                                 pend);
            __syncthreads();   // the buffer is refilled next tile: every warp must be done
        }
    }
    // starts still held for lane-local settling, then the instances queued
    // across tiles, reading the text from global memory (the staged tiles
    // are gone)
    {
        const TileView tv{text_sm, a.text, 0u, 0u, n, 0u, 0u};
        if (KIND == 1 && __any_sync(0xffffffffu, pend.on))
            settle_lanes<KIND, TAB_SMEM, 3>(ov, mv, tv, sm, pend, wq_n, sn, lane, pol_keep,
                                            static_cast<uint32_t>(a.settle_steps));
        if (KIND == 0 && DEFER && __any_sync(0xffffffffu, pend.on))
            dfa_consume<TAB_SMEM, 3>(ov, mv, tv, sm, pend, wq_n, sn, lane, pol_keep);
        drain<KIND, TAB_SMEM, 3>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
    }
    stage_flush<3>(sm.stage, sn, ov, 0u, lane);
    if (bad_symbol) atomicOr(&a.status[1], ERR_SYMBOL);
    if (!PIPE && tid == 0 && abort_at != ~0u) {
        atomicOr(&a.status[1], ERR_TIMEOUT);
        // copies still in flight: wait for them (bounded) before exit
        for (uint32_t t = abort_at; t < my_tiles && t < abort_at + 2; ++t)
            mbar_wait_bounded(&misc->full[t & 1], (t >> 1) & 1);
    }
}

template <int KIND, int SB, bool TAB, int SPT>
static cudaError_t launch_t(const ScanArgs &a, int threads, int grid, uint32_t smem,
                            cudaStream_t s) {
    auto k = scan_tiles<KIND, SB, TAB, SPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads + (SPT == 8 ? 0 : 32), smem, s>>>(a);   // + the producer warp
    return cudaGetLastError();
}

template <int KIND, bool TAB, int SPT>
static cudaError_t launch_sb(const ScanArgs &a, int threads, int grid, uint32_t smem,
                             cudaStream_t s) {
    if (a.k > 0 && a.sbits == 2) return launch_t<KIND, 2, TAB, SPT>(a, threads, grid, smem, s);
    if (a.k > 0 && a.sbits == 8) return launch_t<KIND, 8, TAB, SPT>(a, threads, grid, smem, s);
    return launch_t<KIND, 0, TAB, SPT>(a, threads, grid, smem, s);
}

template <int KIND, int SB, bool TAB, int SPT>
static int occ_t(int threads, uint32_t smem) {
    int nb = 0;
    cudaFuncSetAttribute(scan_tiles<KIND, SB, TAB, SPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_tiles<KIND, SB, TAB, SPT>,
                                                      threads + (SPT == 8 ? 0 : 32), smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

// Launch and occupancy of the kernel instantiated for SPT starts per thread;
// `threads` counts the filtering threads (the pipelined form's producer warp
// is added here).
template <int SPT>
static cudaError_t launch_scan_spt(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                                   cudaStream_t s) {
    if (kind == 0) {
        if (a.tab_smem) return launch_sb<0, true, SPT>(a, threads, grid, smem, s);
        return launch_sb<0, false, SPT>(a, threads, grid, smem, s);
    }
    return launch_sb<1, false, SPT>(a, threads, grid, smem, s);
}

template <int SPT>
static int occupancy_spt(int kind, int sbits, int threads, uint32_t smem, bool tab_smem) {
    const int sb = sbits == 2 ? 2 : (sbits == 8 ? 8 : 0);
    if (kind == 0) {
        if (tab_smem) {
            if (sb == 2) return occ_t<0, 2, true, SPT>(threads, smem);
            if (sb == 8) return occ_t<0, 8, true, SPT>(threads, smem);
            return occ_t<0, 0, true, SPT>(threads, smem);
        }
        if (sb == 2) return occ_t<0, 2, false, SPT>(threads, smem);
        if (sb == 8) return occ_t<0, 8, false, SPT>(threads, smem);
        return occ_t<0, 0, false, SPT>(threads, smem);
    }
    if (sb == 2) return occ_t<1, 2, false, SPT>(threads, smem);
    if (sb == 8) return occ_t<1, 8, false, SPT>(threads, smem);
    return occ_t<1, 0, false, SPT>(threads, smem);
}

}  // namespace pfsm
