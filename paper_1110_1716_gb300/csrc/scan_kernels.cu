// PFSM single-text scan kernels for sm_103a: one persistent CTA per SM loops
// over the tiles of one text (the device building blocks are in
// scan_device.cuh), plus the carry kernels that finish DFA and NFA instances
// past their tile, and the shared-memory layout and launch helpers.
#include "scan_tiles.cuh"

namespace pfsm {

// ------------------------------------------------------------ DFA carry queue
// Continues DFA instances that outlived their tile's staged text (or ran
// DFA_CARRY_AFTER symbols), one thread per instance, reading the text from
// global memory (chained data partitioning, Sec. III.D.2). Entries are {job,
// start, pos, state}. A table of at most 48 KB is read from a shared copy
// (dynamic shared memory of the launch; none otherwise). The matches of the
// lanes that report together are appended with one atomic.
__global__ void __launch_bounds__(256) carry_dfa(const ScanArgs a) {
    // launched as a programmatic dependent of the tile kernel: its launch
    // overlaps the tile kernel's end, and this waits for that kernel to
    // complete (and its writes to be visible) before the queue is read
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t nc = min(*a.carry_n, a.carry_cap);
    if (blockIdx.x * blockDim.x >= nc) return;
    const uint64_t pol_keep = policy_evict_last();
    const uint32_t QS = static_cast<uint32_t>(a.Q) * a.S;
    const bool tab_sm = QS * 2 <= 48 * 1024;
    const uint16_t *tab = a.dtab;
    if (tab_sm) {
        uint32_t *d = reinterpret_cast<uint32_t *>(smem);
        const uint32_t *g = reinterpret_cast<const uint32_t *>(a.dtab);
        for (uint32_t i = threadIdx.x; i < (QS + 1) / 2; i += blockDim.x) d[i] = __ldg(g + i);
        __syncthreads();
        tab = reinterpret_cast<const uint16_t *>(smem);
    }
    const int lane = threadIdx.x & 31;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
         idx += gridDim.x * blockDim.x) {
        const uint4 c = *reinterpret_cast<const uint4 *>(a.carry + 4 * idx);
        const uint32_t start = c.y;
        uint32_t pos = c.z, s = c.w;
        while (pos < a.n) {
            const uint32_t ch = __ldg(a.text + pos);
            if (ch >= static_cast<uint32_t>(a.S)) break;
            if (!PFSM_OK_IDX(s < static_cast<uint32_t>(a.Q), a.status)) break;
            const uint32_t ix = s * a.S + ch;
            const uint16_t e = tab_sm ? tab[ix] : ldg_u16_keep(a.dtab + ix, pol_keep);
            if (e == DEAD16) break;
            s = e & 0x7FFFu;
            if (e & FINAL_BIT) {
                // the lanes that report at this point together: one atomic
                const uint32_t grp = __activemask();
                const int lead = __ffs(grp) - 1;
                unsigned long long base = 0;
                if (lane == lead) base = atomicAdd(&a.status[0], static_cast<unsigned long long>(__popc(grp)));
                base = __shfl_sync(grp, base, lead) + __popc(grp & lanemask_lt());
                if (base < a.cap) {
                    uint32_t *o = a.out + base * 3;
                    o[0] = start;
                    o[1] = pos;
                    o[2] = s;
                }
            }
            ++pos;
        }
    }
}

// ------------------------------------------------------------ NFA carry queue
// Continues NFA instances that outlived their segment (chained data
// partitioning, Sec. III.D.2: the live instance, its start as the tag and its
// state set, passes to the next stage), on the global text to its end. Sets
// that the whole warp held (the second half of the queue) are claimed one
// per warp and run as bitsets over Q; then the lane-held sets (the first
// half) by the exact path's lane refill, one instance per lane. Shared
// memory: band rows (when the scan staged them), then per warp the lane
// slots, the match staging buffer and, when the scan keeps them in shared
// memory, the two warp-wide bitsets.
__global__ void __launch_bounds__(256, 1) carry_nfa(const ScanArgs a) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    uint32_t off[4];
    carry_nfa_layout(a, nw, off);
    const uint32_t half = a.carry_cap / 2;
    const uint32_t n_lane = min(a.carry_n[0], half);
    const uint32_t n_warp = min(a.carry_n[3], a.carry_cap - half);
    if (n_lane == 0 && n_warp == 0) return;
    const uint64_t pol_keep = policy_evict_last();
    // nothing is carried again: the carried instances run to the end
    const OView ov{a.out, a.cap, a.status, nullptr, a.carry, a.carry_n, 0u, a.stage_n,
                   a.cpool, a.cpool_cap};
    const MView mv{a.Q, a.S, a.q0, a.k, a.sbits, a.Wq, a.surv_m, a.surv2_m, a.surv2, a.dtab, a.off, a.tgt,
                   a.tail, a.ecl_off, a.ecl_tgt, a.l2tab, a.pool2, a.memox, a.status, a.pool_n,
                   a.memo_n};
    Smem sm = {};
    if (a.band_smem && a.band) {
        uint32_t *b = reinterpret_cast<uint32_t *>(smem + off[0]);
        const uint32_t words = static_cast<uint32_t>(a.Q + (a.Q + 31) / 32);
        for (uint32_t i = tid; i < words; i += blockDim.x) b[i] = __ldg(a.band + i);
        sm.band = b;
    } else {
        sm.band = a.band;
    }
    __syncthreads();
    sm.pool = a.pool;
    sm.slots = reinterpret_cast<uint16_t *>(smem + off[1]) + wid * (2 * NFA_SLOT * 32);
    sm.stage = reinterpret_cast<uint32_t *>(smem + off[2]) + wid * (4 * a.stage_n);
    sm.coop = a.coop_smem ? reinterpret_cast<uint32_t *>(smem + off[3]) + wid * 2 * a.Wq
            : a.coop_g ? a.coop_g + (static_cast<size_t>(blockIdx.x) * nw + wid) * 2 * a.Wq
                       : nullptr;
    const TileView tv{nullptr, a.text, 0u, 0u, a.n, 0u, 0u};
    // 1. warp-held sets, one per warp
    if (sm.coop) {
        uint32_t *b0 = sm.coop, *b1 = sm.coop + a.Wq;
        while (true) {
            uint32_t idx = 0;
            if (lane == 0) idx = atomicAdd(&a.carry_n[4], 1u);
            idx = __shfl_sync(FULLMASK, idx, 0);
            if (idx >= n_warp) break;
            const uint4 h = *reinterpret_cast<const uint4 *>(a.carry + NFA_CARRY_WORDS * (half + idx));
            const uint32_t po = a.carry[NFA_CARRY_WORDS * (half + idx) + 4];
            for (uint32_t w = lane; w < static_cast<uint32_t>(a.Wq); w += 32) {
                b0[w] = 0;
                b1[w] = 0;
            }
            __syncwarp();
            for (uint32_t i = lane; i < h.w; i += 32) {
                const uint32_t q = a.cpool[po + i];
                if (!PFSM_OK_IDX(q < static_cast<uint32_t>(a.Q), a.status)) continue;
                atomicOr(&b0[q >> 5], 1u << (q & 31));
            }
            __syncwarp();
            coop_run<3>(ov, mv, sm.band, tv, b0, b1, h.y, h.z, 0xFFFFFFFFu, lane, pol_keep);
        }
    }
    // 2. lane-held sets
    uint32_t sn = 0;
    // entries per claim: the lane-held sets spread over every warp of the grid
    const uint32_t warps = gridDim.x * nw;
    const uint32_t claim = min(32u, max(1u, (n_lane + warps - 1) / warps));
    if (n_lane) drain_nfa<3, true>(ov, mv, tv, sm, n_lane, sn, lane, pol_keep, claim);
    stage_flush<3>(sm.stage, sn, ov, 0u, lane);
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
    // table regions are whole 16-byte blocks: they are filled by bulk copies
    auto r16 = [](uint32_t x) { return (x + 15u) & ~15u; };
    if (a.stage_n == 0) a.stage_n = STAGE;
    // the shallow survival bitmap (or 2-gram byte table) sits at offset 0:
    // the single-text kernel indexes the shared array with the gram itself
    if (need.surv_bytes) a.sm_surv = take(r16(need.surv_bytes), 16);
    a.sm_misc = take(sizeof(Misc), 16);
    a.sm_memo = take(r16(need.memo_bytes), 16);
    a.memo_smem = need.memo_bytes > 0;
    a.sm_tab = take(r16(need.tab_bytes), 16);
    a.sm_band = take(r16(need.band_bytes), 16);
    a.sm_pool = take(r16(need.pool_bytes), 16);
    if (!need.surv_bytes) a.sm_surv = 0;
    a.band_smem = need.band_bytes > 0;
    a.pool_smem = need.pool_bytes > 0;
    a.sm_list = take(nw * WARP_LIST_BYTES, 16);
    if (a.nbuf == 0) a.nbuf = 2;   // the kernels index the buffers by this count
    const uint32_t nbuf = a.nbuf;
    a.sm_text = take(nbuf * a.text_buf, 128);
    // each staged tile packed to 2-bit symbols, 16 per word (+1 word read past)
    a.pk_words = (a.text_buf + 15) / 16 + 2;
    a.sm_pack = take(nbuf * a.pk_words * 4, 16);
    // queue: starts (uint32), prefix entries (uint16), and one flag bit per
    // entry (NFA: the entry is a second-level record)
    a.sm_queue = take(nw * WARP_QUEUE * 6 + nw * (WARP_QUEUE / 8), 16);
    a.sm_stage = take(nw * a.stage_n * 16, 16);
    a.sm_slots = take(has_nfa ? nw * 2 * NFA_SLOT * 32 * 2 : 0, 16);
    // warp-wide NFA bitsets: shared memory when planned, else global scratch
    a.sm_coop = take(has_nfa ? need.coop_bytes : 0u, 16);
    a.coop_smem = has_nfa && need.coop_bytes > 0;
    return (o + 127) & ~127u;
}

cudaError_t launch_scan(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                        cudaStream_t s) {
    if (a.spt == 8) return launch_scan_spt8(a, kind, threads, grid, smem, s);
    return launch_scan_spt<32>(a, kind, threads, grid, smem, s);
}

cudaError_t launch_carry(const ScanArgs &a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(256);
    // the table's shared copy (carry_dfa takes it when it is at most 48 KB)
    const uint32_t tab_bytes = static_cast<uint32_t>(a.Q) * a.S * 2;
    cfg.dynamicSmemBytes = tab_bytes <= 48 * 1024 ? ((tab_bytes + 3) & ~3u) : 0u;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, carry_dfa, a);
}

cudaError_t launch_carry_nfa(const ScanArgs &a, int grid, int threads, cudaStream_t s) {
    uint32_t off[4];
    const uint32_t smem = carry_nfa_layout(a, threads / 32, off);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(carry_nfa, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return cudaGetLastError();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, carry_nfa, a);
}

int max_ctas_per_sm(int kind, int sbits, int threads, uint32_t smem, bool tab_smem, int spt) {
    if (spt == 8) return max_ctas_per_sm_spt8(kind, sbits, threads, smem, tab_smem);
    return occupancy_spt<32>(kind, sbits, threads, smem, tab_smem);
}

}  // namespace pfsm
