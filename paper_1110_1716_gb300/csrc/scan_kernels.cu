// PFSM single-text scan kernels for sm_103a: one persistent CTA per SM loops
// over the tiles of one text (the device building blocks are in
// scan_device.cuh), plus the carry kernel that finishes DFA instances past
// their tile, and the shared-memory layout and launch helpers.
#include "scan_device.cuh"

namespace pfsm {

// ------------------------------------------------------------ single-text kernel
template <int KIND, int SB, bool TAB_SMEM>
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
        process_tile<KIND, SB, TAB_SMEM, 3>(ov, mv, tv, sm, min(b + a.tile, n), wq_n, sn,
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

// ------------------------------------------------------------ DFA carry queue
// Continues DFA instances that outlived their tile's staged text, reading the
// text from global memory (chained data partitioning, Sec. III.D.2). Entries
// are {job, start, pos, state}.
__global__ void __launch_bounds__(256) carry_dfa(const ScanArgs a) {
    const uint32_t nc = min(*a.carry_n, a.carry_cap);
    const uint64_t pol_keep = policy_evict_last();
    const OView ov{a.out, a.cap, a.status, nullptr, a.carry, a.carry_n, a.carry_cap, a.stage_n};
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
         idx += gridDim.x * blockDim.x) {
        const uint32_t *c = a.carry + 4 * idx;
        const uint32_t start = c[1];
        uint32_t pos = c[2], s = c[3];
        while (pos < a.n) {
            const uint32_t ch = __ldg(a.text + pos);
            if (ch >= static_cast<uint32_t>(a.S)) break;
            const uint16_t e = ldg_u16_keep(a.dtab + s * a.S + ch, pol_keep);
            if (e == DEAD16) break;
            s = e & 0x7FFFu;
            if (e & FINAL_BIT) emit_direct<3>(ov, 0u, start, pos, s);
            ++pos;
        }
    }
}

// ------------------------------------------------------------ host helpers
uint32_t layout_smem(ScanArgs &a, int kind_mask, int threads, const SmemNeed &need) {
    const int nw = threads / 32;
    const bool has_nfa = (kind_mask & 2) != 0;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) & ~(align - 1);
        const uint32_t r = o;
        o += bytes;
        return r;
    };
    if (a.stage_n == 0) a.stage_n = STAGE;
    a.sm_misc = take(sizeof(Misc), 16);
    a.sm_memo = take(need.memo_bytes, 16);
    a.memo_smem = need.memo_bytes > 0;
    a.sm_tab = take(need.tab_bytes, 16);
    a.sm_band = take(need.band_bytes, 16);
    a.sm_pool = take(need.pool_bytes, 16);
    a.sm_surv = take(need.surv_bytes, 16);
    a.band_smem = need.band_bytes > 0;
    a.pool_smem = need.pool_bytes > 0;
    a.sm_list = take(nw * WARP_LIST_BYTES, 16);
    a.sm_text = take(2 * a.text_buf, 128);
    // the current tile packed to 2-bit symbols, 16 per word (+1 word read past)
    a.sm_pack = take(((a.text_buf + 15) / 16 + 2) * 4, 16);
    a.sm_queue = take(nw * WARP_QUEUE * 6, 16);
    a.sm_stage = take(nw * a.stage_n * 16, 16);
    a.sm_slots = take(has_nfa ? nw * 2 * NFA_SLOT * 32 * 2 : 0, 16);
    // warp-wide NFA bitsets: shared memory when planned, else global scratch
    a.sm_coop = take(has_nfa ? need.coop_bytes : 0u, 16);
    a.coop_smem = has_nfa && need.coop_bytes > 0;
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

cudaError_t launch_scan(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                        cudaStream_t s) {
    if (kind == 0) {
        if (a.tab_smem) return launch_sb<0, true>(a, threads, grid, smem, s);
        return launch_sb<0, false>(a, threads, grid, smem, s);
    }
    return launch_sb<1, false>(a, threads, grid, smem, s);
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
