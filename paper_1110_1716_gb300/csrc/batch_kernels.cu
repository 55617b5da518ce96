// Batch scan kernels for sm_103a: many texts, each with its own machine.
//
// The machines of a batch are grouped into classes (kind, prefix-symbol
// width, DFA table in shared memory) and every class runs its own
// specialised persistent kernel, so each keeps the register budget of the
// matching single-text kernel. The class kernels of one batch run side by
// side on the device (parallel branches of one CUDA graph).
//
// Inside a class, the texts' tiles are cut into work units of a few
// consecutive tiles of one text; persistent CTAs pull units from the class's
// counter. While consecutive tiles belong to the same text, a CTA keeps its
// per-warp instance queues and staged matches across the tile boundary
// (queued instances read the earlier bytes from global memory), and drains
// them only when the text changes: this combines the regex partitioning of
// Sec. III.D (machines split across texts) with the data partitioning of the
// same section (texts cut into tiles).
//
// Each machine's tables (survival bitmap, prefix table, DFA table, NFA band
// rows and prefix records) are copied into a shared-memory table arena when
// a CTA moves to that machine, at offsets chosen on the host.
#include "scan_device.cuh"

namespace pfsm {

// One claimed tile of a unit.
struct UnitDesc {
    const uint8_t *text;
    uint32_t valid, job, orig, mach, b, len, n, sh;
};

// Last job of [lo, hi) whose unit_begin <= u.
__device__ __forceinline__ uint32_t find_unit_job(const BatchJob *jobs, uint32_t lo, uint32_t hi,
                                                  uint32_t u) {
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].unit_begin <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ MView mview_of(const DevMachine &m, unsigned long long *status) {
    return MView{m.Q, m.S, m.q0, m.k, m.sbits, m.Wq, m.surv_m, m.surv2_m, m.surv2, m.dtab, m.off, m.tgt,
                 m.tail, m.ecl_off, m.ecl_tgt, m.l2tab, m.pool2, m.memox, status, m.pool_n,
                 m.memo_n};
}

// Copies `words` 32-bit words (16-byte aligned source and destination).
__device__ __forceinline__ void stage_words(uint8_t *dst, const void *src, uint32_t words, int tid,
                                            int nt) {
    const uint32_t quads = words >> 2;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = tid; i < quads; i += nt) d4[i] = __ldg(s4 + i);
    const uint32_t *s1 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d1 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = 4 * quads + tid; i < words; i += nt) d1[i] = __ldg(s1 + i);
}

// Warps 0 .. NC/32 - 1 filter (NC = blockDim.x - 32; at most 15 warps for
// the NFA classes, which keeps their 128 registers per thread); the last
// warp is the producer. The producer claims work units through the class's atomic
// cursor, copies their tiles by TMA into A.sa.nbuf buffers, realigns and
// packs each one and hands it over with its descriptor (mbarrier `ready`);
// each filtering warp releases a buffer when it is done with it (`empty`,
// one arrival per warp). A descriptor that is not valid ends the work. The
// producer polls both duties, so a landed tile is handed over while older
// tiles are still in use. Filtering warps meet only when the machine
// changes (two meetings on a bounded mbarrier around the restaging of the
// table arena); a warp whose next tile belongs to another text first drains
// its queue and flushes its staged matches (per-text counts need every
// flush to belong to one text). Every wait is bounded (2 s).
template <int KIND, int SB, bool TAB>
__global__ void __launch_bounds__(KIND == 1 ? 512 : 544, 1) scan_units(const BatchArgs *__restrict__ gargs) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ BatchArgs A;
    __shared__ UnitDesc desc[kTileBufs];
    // The views of the current machine and of the output live in shared
    // memory: read from the machine table in global memory they would
    // otherwise stay in registers across a whole tile (the NFA classes run
    // at 128 registers per thread). ovs[1] is the lazy form (no carry).
    __shared__ MView mv_sh;
    __shared__ OView ovs[2];
    __shared__ UnitDesc prev_sh[16];   // per filtering warp: its previous tile
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int NT = blockDim.x;
    const int NC = NT - 32;   // filtering threads
    const int ncw = NC >> 5;
    const bool producer = wid == ncw;
    if (tid == 0) A = *gargs;
    __syncthreads();
    const uint32_t nb = A.sa.nbuf;
    if (nb < 2 || nb > static_cast<uint32_t>(kTileBufs)) {   // the layout's buffers
        if (tid == 0) atomicOr(&A.sa.status[1], ERR_SYMBOL);
        return;
    }
    const Smem sm = smem_regions(smem, A.sa, producer ? 0 : wid, ncw);
    Misc *misc = sm.misc;
    uint8_t *text_sm = smem + A.sa.sm_text;
    uint32_t *pk_sm = reinterpret_cast<uint32_t *>(smem + A.sa.sm_pack);
    uint8_t *arena = smem + A.sm_arena;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    if (tid == 0) {
        ovs[0] = OView{A.sa.out, A.sa.cap, A.sa.status, A.job_counts, A.sa.carry, A.sa.carry_n,
                       A.sa.carry_cap, A.sa.stage_n};
        ovs[1] = ovs[0];
        ovs[1].carry_cap = 0;
    }
    const OView &ov = ovs[0];
    if (tid == 0) {
        for (int i = 0; i < kTileBufs; ++i) {
            mbar_init(&misc->full[i], 1);
            mbar_init(&misc->ready[i], 1);
            mbar_init(&misc->empty[i], static_cast<uint32_t>(ncw));
        }
        mbar_init(&misc->bar[0], static_cast<uint32_t>(ncw));   // filtering warps' meetings
        misc->q_count = 0;
        misc->q_head = 0;
        misc->abort = 0;
        misc->busy = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (producer) {
        // lane 0's cursor: the tiles [cur_tile, cur_end) of job cur_job remain
        // in its current unit
        uint32_t cur_job = 0, cur_tile = 0, cur_end = 0;
        // tile k into buffer k % nb (lane 0 claims it and starts its copy);
        // returns whether there was one
        auto claim = [&](uint32_t k) -> bool {
            uint32_t valid = 0;
            if (lane == 0) {
                UnitDesc &d = desc[k % nb];
                valid = 1;
                if (cur_tile >= cur_end) {
                    const uint32_t u = atomicAdd(A.unit_counter, 1u);
                    if (u >= A.nunits) {
                        valid = 0;
                    } else {
                        cur_job = find_unit_job(A.jobs, A.job_lo, A.job_hi, u);
                        const BatchJob &J = A.jobs[cur_job];
                        cur_tile = (u - J.unit_begin) * A.unit_tiles;
                        cur_end = min(cur_tile + A.unit_tiles, J.ntiles);
                    }
                }
                d.valid = valid;
                if (valid) {
                    const BatchJob &J = A.jobs[cur_job];
                    d.job = cur_job;
                    d.text = J.text;
                    d.n = J.n;
                    d.orig = J.orig;
                    d.mach = J.mach;
                    d.b = cur_tile * A.sa.tile;
                    ++cur_tile;
                    d.len = min(A.sa.tile + A.sa.halo, d.n - d.b);
                    // one bulk copy from the 16-byte boundary at or below the
                    // tile's first byte (the block it starts in lies in the
                    // text's page)
                    const uintptr_t src = reinterpret_cast<uintptr_t>(d.text) + d.b;
                    d.sh = static_cast<uint32_t>(src & 15u);
                    const uint32_t bytes = (d.sh + d.len + 15) & ~15u;
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&misc->full[k % nb], bytes);
                    tma_load_1d(text_sm + (k % nb) * A.sa.text_buf,
                                reinterpret_cast<const void *>(src - d.sh), bytes, &misc->full[k % nb],
                                pol_stream);
                }
            }
            return __shfl_sync(0xffffffffu, valid, 0) != 0;
        };
        bool ok = true;
        uint32_t issued = 0, prepped = 0;   // tiles claimed / handed over
        uint32_t total = 0xFFFFFFFFu;       // index of the closing (invalid) descriptor
        while (issued < nb && total == 0xFFFFFFFFu) {
            if (!claim(issued)) total = issued;
            ++issued;
        }
        uint64_t idle_since = global_ns();
        while (true) {
            bool progress = false;
            if (prepped < issued) {
                const int buf = static_cast<int>(prepped % nb);
                if (prepped == total) {   // the closing descriptor: no copy
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&misc->ready[buf]);
                    break;
                }
                if (__all_sync(0xffffffffu, mbar_test_wait(&misc->full[buf], (prepped / nb) & 1))) {
                    __syncwarp();   // lane 0's descriptor writes are visible
                    const UnitDesc d = desc[buf];
                    uint8_t *tsm = text_sm + buf * A.sa.text_buf;
                    if (d.sh) realign_tile_warp(tsm, d.sh, d.len, lane);
                    if (SB == 2) {
                        bool bad = false;
                        pack_tile(tsm, pk_sm + buf * A.sa.pk_words, d.len, min(d.b + A.sa.tile, d.n) - d.b,
                                  static_cast<uint32_t>(A.machs[d.mach].S), bad, lane, 32);
                        if (bad) atomicOr(&A.sa.status[1], ERR_SYMBOL);
                    }
                    // the realigned bytes are rewritten by a later bulk copy
                    if (d.sh) fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&misc->ready[buf]);
                    ++prepped;
                    progress = true;
                }
            }
            // tile `issued` goes to the buffer of tile issued - nb once every
            // filtering warp is done with that tile
            if (total == 0xFFFFFFFFu &&
                __all_sync(0xffffffffu, mbar_test_wait(&misc->empty[issued % nb], (issued / nb - 1) & 1))) {
                if (!claim(issued)) total = issued;
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
            atomicOr(&A.sa.status[1], ERR_TIMEOUT);
            // copies still in flight: wait for them (bounded) before exit
            for (uint32_t t = prepped; t < issued; ++t)
                if (t != total) mbar_wait_bounded(&misc->full[t % nb], (t / nb) & 1);
        }
        return;
    }

    uint32_t sn = 0;
    uint32_t wq_n = 0;
    Pend pend{0u, 0u, 0u, 0u, false};   // held start of the current text (see process_tile)
    bool bad_symbol = false;
    bool aborted = false;
    uint32_t cur_mach = 0xFFFFFFFFu;   // machine whose tables the arena holds
    uint32_t meet = 0;                 // meetings so far
    Smem smi = sm;
    // the previous tile's text: its queue is drained when the text changes
    bool have_prev = false;
    UnitDesc &prev = prev_sh[wid];
    const OView *prev_ov = &ovs[0];
    // every filtering warp arrives and waits (bounded)
    auto meet_all = [&]() -> bool {
        __syncwarp();
        if (lane == 0) mbar_arrive(&misc->bar[0]);
        const bool okm = __all_sync(0xffffffffu, mbar_wait_live(&misc->bar[0], meet & 1, &misc->busy));
        ++meet;
        return okm;
    };
    // drains this warp's queue of the previous text (reading it from global
    // memory: its staged tile may be gone) and flushes its staged matches
    auto drain_prev = [&]() {
        // the arena and mv_sh still hold the previous tile's machine: a
        // machine change restages them only after this drain
        const MView &pmv = mv_sh;
        const TileView ptv{text_sm, prev.text, 0u, 0u, prev.n, prev.job, prev.orig};
        // the starts this warp still holds for the previous text (lane-local
        // settling, deferred deep-bitmap loads) go first: the arena still
        // holds that machine's tables
        if (KIND == 1 && __any_sync(0xffffffffu, pend.on))
            settle_lanes<KIND, TAB, 4>(*prev_ov, pmv, ptv, smi, pend, wq_n, sn, lane, pol_keep,
                                       static_cast<uint32_t>(A.machs[prev.mach].settle));
        if (KIND == 0 && __any_sync(0xffffffffu, pend.on))
            dfa_consume<TAB, 4>(*prev_ov, pmv, ptv, smi, pend, wq_n, sn, lane, pol_keep);
        drain<KIND, TAB, 4>(*prev_ov, pmv, ptv, smi, wq_n, sn, lane, pol_keep);
        stage_flush<4>(sm.stage, sn, ov, prev.orig, lane);
    };
    for (uint32_t k = 0;; ++k) {
        const int buf = static_cast<int>(k % nb);
        const bool go = mbar_wait_live(&misc->ready[buf], (k / nb) & 1, &misc->busy) &&
                        !*reinterpret_cast<volatile uint32_t *>(&misc->abort);
        if (!__all_sync(0xffffffffu, go)) {
            if (lane == 0) atomicOr(&A.sa.status[1], ERR_TIMEOUT);
            aborted = true;
            break;
        }
        const UnitDesc d = desc[buf];
        if (!d.valid) break;
        if (have_prev && d.job != prev.job) drain_prev();
        const DevMachine &M = A.machs[d.mach];
        if (d.mach != cur_mach) {
            // a new machine: every warp is done with the old one's tables
            // (its queue drained above) before the arena is rewritten, and
            // the new tables are complete before any warp reads them
            if (!meet_all()) {
                if (lane == 0) atomicOr(&A.sa.status[1], ERR_TIMEOUT);
                aborted = true;
                break;
            }
            if (M.a_surv != kNotStaged) stage_words(arena + M.a_surv, M.surv, M.surv_words, tid, NC);
            if (M.a_memo != kNotStaged) stage_words(arena + M.a_memo, M.memo, (M.memo_n + 1) / 2, tid, NC);
            if (TAB) stage_words(arena + M.a_tab, M.dtab, (static_cast<uint32_t>(M.Q) * M.S + 1) / 2, tid, NC);
            if (KIND == 1) {
                if (M.a_band != kNotStaged)
                    stage_words(arena + M.a_band, M.band, static_cast<uint32_t>(M.Q + (M.Q + 31) / 32), tid, NC);
                if (M.a_pool != kNotStaged) stage_words(arena + M.a_pool, M.pool, M.pool_n, tid, NC);
            }
            smi.surv = M.a_surv != kNotStaged ? reinterpret_cast<const uint32_t *>(arena + M.a_surv) : nullptr;
            smi.memo = M.a_memo != kNotStaged ? reinterpret_cast<const uint16_t *>(arena + M.a_memo) : M.memo;
            smi.tab = TAB ? reinterpret_cast<const uint16_t *>(arena + M.a_tab) : nullptr;
            smi.band = M.a_band != kNotStaged ? reinterpret_cast<const uint32_t *>(arena + M.a_band) : M.band;
            smi.pool = M.a_pool != kNotStaged ? reinterpret_cast<const uint32_t *>(arena + M.a_pool) : M.pool;
            smi.coop = M.a_coop != kNotStaged
                           ? reinterpret_cast<uint32_t *>(arena + M.a_coop) + wid * 2 * M.Wq : sm.coop;
            if (tid == 0) mv_sh = mview_of(M, A.sa.status);
            cur_mach = d.mach;
            if (!meet_all()) {
                if (lane == 0) atomicOr(&A.sa.status[1], ERR_TIMEOUT);
                aborted = true;
                break;
            }
        }
        const MView &mv = mv_sh;
        const TileView tv{text_sm + buf * A.sa.text_buf, d.text, d.b, d.len, d.n, d.job, d.orig};
        // lazy partitioning for this machine; NFA machines of a batch are
        // always lazy (the batch carry queue holds DFA entries only)
        const OView &ovm = ovs[(M.lazy || KIND == 1) ? 1 : 0];
        smi.pk = pk_sm + buf * A.sa.pk_words;
        const uint32_t own_end = min(d.b + A.sa.tile, d.n);
        process_tile<KIND, SB, TAB, 4, 32, true>(ovm, mv, tv, smi, own_end, wq_n, sn, bad_symbol,
                                                 pol_keep, static_cast<uint32_t>(M.settle), NC, pend);
        __syncwarp();
        if (lane == 0) mbar_arrive(&misc->empty[buf]);
        have_prev = true;
        if (lane == 0) prev = d;
        __syncwarp();
        prev_ov = &ovm;
    }
    if (have_prev && !aborted) drain_prev();
    if (bad_symbol) atomicOr(&A.sa.status[1], ERR_SYMBOL);
}

// ------------------------------------------------------------ DFA carry queue
// Batch form of the carry continuation (chained data partitioning,
// Sec. III.D.2); entries are {job, start, pos, state} with global job indices.
__global__ void __launch_bounds__(256) carry_batch(const BatchArgs *__restrict__ g) {
    const uint32_t nc = min(*g->sa.carry_n, g->sa.carry_cap);
    const uint64_t pol_keep = policy_evict_last();
    const OView ov{g->sa.out, g->sa.cap, g->sa.status, g->job_counts, g->sa.carry,
                   g->sa.carry_n, g->sa.carry_cap, g->sa.stage_n};
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nc;
         idx += gridDim.x * blockDim.x) {
        const uint32_t *c = g->sa.carry + 4 * idx;
        const uint32_t start = c[1];
        uint32_t pos = c[2], s = c[3];
        const BatchJob &J = g->jobs[c[0]];
        const DevMachine &M = g->machs[J.mach];
        const uint32_t S = M.S;
        while (pos < J.n) {
            const uint32_t ch = __ldg(J.text + pos);
            if (ch >= S) break;
            const uint16_t e = ldg_u16_keep(M.dtab + s * S + ch, pol_keep);
            if (e == DEAD16) break;
            s = e & 0x7FFFu;
            if (e & FINAL_BIT) emit_direct<4>(ov, J.orig, start, pos, s);
            ++pos;
        }
    }
}

// ------------------------------------------------------------ host helpers
int batch_class(int kind, int sbits, int k, bool tab_smem) {
    const int sbi = (k > 0 && sbits == 2) ? 1 : ((k > 0 && sbits == 8) ? 2 : 0);
    if (kind == 1) return 6 + sbi;
    return 3 * (tab_smem ? 1 : 0) + sbi;
}

template <int KIND, int SB, bool TAB>
static cudaError_t launch_u(const BatchArgs *dev_args, int threads, int grid, uint32_t smem,
                            cudaStream_t s) {
    auto k = scan_units<KIND, SB, TAB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads + 32, smem, s>>>(dev_args);   // + the producer warp
    return cudaGetLastError();
}

template <int KIND, int SB, bool TAB>
static int occ_u(int threads, uint32_t smem) {
    int nb = 0;
    auto k = scan_units<KIND, SB, TAB>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads + 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_units(int cls, const BatchArgs *dev_args, int threads, int grid,
                         uint32_t smem, cudaStream_t s) {
    switch (cls) {
        case 0: return launch_u<0, 0, false>(dev_args, threads, grid, smem, s);
        case 1: return launch_u<0, 2, false>(dev_args, threads, grid, smem, s);
        case 2: return launch_u<0, 8, false>(dev_args, threads, grid, smem, s);
        case 3: return launch_u<0, 0, true>(dev_args, threads, grid, smem, s);
        case 4: return launch_u<0, 2, true>(dev_args, threads, grid, smem, s);
        case 5: return launch_u<0, 8, true>(dev_args, threads, grid, smem, s);
        case 6: return launch_u<1, 0, false>(dev_args, threads, grid, smem, s);
        case 7: return launch_u<1, 2, false>(dev_args, threads, grid, smem, s);
        case 8: return launch_u<1, 8, false>(dev_args, threads, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

int max_units_ctas_per_sm(int cls, int threads, uint32_t smem) {
    switch (cls) {
        case 0: return occ_u<0, 0, false>(threads, smem);
        case 1: return occ_u<0, 2, false>(threads, smem);
        case 2: return occ_u<0, 8, false>(threads, smem);
        case 3: return occ_u<0, 0, true>(threads, smem);
        case 4: return occ_u<0, 2, true>(threads, smem);
        case 5: return occ_u<0, 8, true>(threads, smem);
        case 6: return occ_u<1, 0, false>(threads, smem);
        case 7: return occ_u<1, 2, false>(threads, smem);
        case 8: return occ_u<1, 8, false>(threads, smem);
        default: return 0;
    }
}

cudaError_t launch_carry_batch(const BatchArgs *dev_args, int grid, cudaStream_t s) {
    carry_batch<<<grid, 256, 0, s>>>(dev_args);
    return cudaGetLastError();
}

}  // namespace pfsm
