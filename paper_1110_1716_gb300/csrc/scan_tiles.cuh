// The single-text scan kernel and its launch helpers, as templates over the
// starts each thread takes per filter round (SPT). scan_kernels.cu
// instantiates SPT = 32 (long texts), scan_kernels_spt8.cu SPT = 8 (short
// texts: four times the warps for the same text).
#pragma once

#include "scan_device.cuh"

namespace pfsm {

// ------------------------------------------------------------ single-text kernel
template <int KIND, int SB, bool TAB_SMEM, int SPT>
__global__ void __launch_bounds__(512, 1) scan_tiles(const ScanArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int NT = blockDim.x;
    const Smem sm = smem_regions(smem, a, wid);
    Misc *misc = sm.misc;
    uint8_t *text_sm = smem + a.sm_text;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const OView ov{a.out, a.cap, a.status, nullptr, a.carry, a.carry_n, a.carry_cap, a.stage_n};
    const MView mv{a.Q, a.S, a.q0, a.k, a.sbits, a.Wq, a.surv_m, a.surv2_m, a.surv2, a.dtab, a.off, a.tgt,
                   a.tail, a.ecl_off, a.ecl_tgt};

    if (a.memo_smem) stage_u16(const_cast<uint16_t *>(sm.memo), a.memo, a.memo_n, tid, NT);
    if (TAB_SMEM) stage_u16(const_cast<uint16_t *>(sm.tab), a.dtab, a.Q * a.S, tid, NT);
    if (KIND == 1) stage_nfa(smem, a.sm_band, a.sm_pool, a.band_smem ? a.band : nullptr, a.Q,
                             a.pool_smem ? a.pool : nullptr, a.pool_n, tid, NT);
    if (a.surv) {
        uint32_t *d = reinterpret_cast<uint32_t *>(smem + a.sm_surv);
        for (uint32_t i = tid; i < a.surv_words; i += NT) d[i] = __ldg(a.surv + i);
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

    uint32_t sn = 0;
    uint32_t wq_n = 0;   // entries in this warp's queue
    bool bad_symbol = false;
    const uint32_t n = a.n;
    // tile `tile` into buffer `buf`: one bulk copy from the 16-byte boundary
    // at or below its first byte (a 16-byte block never crosses a page, so
    // the bytes around the text that it covers are readable)
    auto issue = [&](uint32_t tile, int buf) {
        const uint32_t b = tile * a.tile;
        const uint32_t len = min(a.tile + a.halo, n - b);
        const uint32_t bytes = (a.shift + len + 15) & ~15u;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&misc->bar[buf], bytes);
        tma_load_1d(text_sm + buf * a.text_buf,
                    reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(a.text) + b - a.shift),
                    bytes, &misc->bar[buf], pol_stream);
    };

    uint32_t it = 0;
    if (tid == 0 && blockIdx.x < a.ntiles) issue(blockIdx.x, 0);
    for (uint32_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        const uint32_t b = tile * a.tile;
        const uint32_t len = min(a.tile + a.halo, n - b);
        uint8_t *tsm = text_sm + buf * a.text_buf;
        if (tid == 0 && tile + gridDim.x < a.ntiles) issue(tile + gridDim.x, buf ^ 1);
        if (!mbar_wait_bounded(&misc->bar[buf], parity)) misc->abort = 1;
        if (a.shift) realign_tile(tsm, a.shift, len, tid, NT);   // ends with a barrier
        else __syncthreads();
        if (misc->abort) break;
        if (SB == 2) {   // 2-bit symbols: pack the tile once for every gram read
            pack_tile(tsm, sm.pk, len, min(b + a.tile, n) - b, static_cast<uint32_t>(a.S),
                      bad_symbol, tid, NT);
            __syncthreads();
        }
        const TileView tv{tsm, a.text, b, len, n, 0u, 0u};
        process_tile<KIND, SB, TAB_SMEM, 3, SPT>(ov, mv, tv, sm, min(b + a.tile, n), wq_n, sn,
                                            bad_symbol, pol_keep, static_cast<uint32_t>(a.settle_steps));
        // the staged buffer is refilled two tiles on: every warp must be done
        __syncthreads();
    }
    // instances queued across tiles run now, reading the text from global
    // memory (the staged tiles are gone)
    {
        const TileView tv{text_sm, a.text, 0u, 0u, n, 0u, 0u};
        drain<KIND, TAB_SMEM, 3>(ov, mv, tv, sm, wq_n, sn, lane, pol_keep);
    }
    stage_flush<3>(sm.stage, sn, ov, 0u, lane);
    if (bad_symbol) atomicOr(&a.status[1], ERR_SYMBOL);
    if (tid == 0 && misc->abort) {
        atomicOr(&a.status[1], ERR_TIMEOUT);
        // a copy may still be in flight: wait for it (bounded) before exit
        mbar_wait_bounded(&misc->bar[0], 0);
        mbar_wait_bounded(&misc->bar[1], 0);
    }
}

template <int KIND, int SB, bool TAB, int SPT>
static cudaError_t launch_t(const ScanArgs &a, int threads, int grid, uint32_t smem,
                            cudaStream_t s) {
    auto k = scan_tiles<KIND, SB, TAB, SPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, s>>>(a);
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_tiles<KIND, SB, TAB, SPT>, threads,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

// Launch and occupancy of the kernel instantiated for SPT starts per thread.
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
