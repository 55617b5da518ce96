// Batched scans: many texts, each with its own machine. This combines the
// two partitionings of Sec. III.D: the set of machines is split across texts
// (regex partitioning) and every text is cut into tiles (data partitioning).
//
// The machines of a batch are grouped into classes, one specialised
// persistent kernel each (batch_kernels.cu). Every class has a fixed launch
// shape per context (threads, CTAs, shared-memory layout with a table arena
// of fixed size), so one launch sequence serves every batch: counter and
// status resets, one branch per class (the class kernels run side by side;
// a class with no work in the batch claims nothing and exits), then the DFA
// carry kernel. That sequence is captured once per stream as a CUDA graph
// and replayed; the per-batch argument blocks, job table and machine table
// are copied to a fixed device block before each replay.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "pfsm_host.h"

namespace pfsm {

constexpr uint32_t kBatchTile = 16384;
constexpr uint32_t kBatchHalo = 2048;
constexpr uint32_t kMinArena = 8192;     // smallest table arena worth a class shape
constexpr int kUnitTilesMax = 8;        // tiles per work unit, at most
constexpr int kCarryCtr = 15;           // counter word holding the carry count
constexpr uint32_t kAllClasses = (1u << kBatchClasses) - 1;

struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t gen = 0;
};

struct BatchState {
    cudaStream_t capture = nullptr;   // private stream used to capture the graphs
    cudaStream_t aux[kBatchClasses] = {};   // one capture branch per class
    cudaEvent_t fork = nullptr, join[kBatchClasses] = {};
    size_t cap_jobs = 0, cap_machs = 0;
    size_t off_jobs = 0, off_machs = 0, block_bytes = 0;
    uint8_t *dev = nullptr;           // BatchArgs[kBatchClasses] | jobs | machines
    uint8_t *host = nullptr;          // pinned staging of the same layout
    uint32_t *ctr = nullptr;          // device: [c] unit counter of class c, [15] carry count
    unsigned long long *status = nullptr;       // device: total, errors, per-job counts
    unsigned long long *host_status = nullptr;  // pinned copy of status
    uint32_t *carry = nullptr;
    uint32_t *coop = nullptr;         // warp-wide NFA bitsets of every NFA class
    size_t coop_words = 0;
    cudaEvent_t staged = nullptr;     // previous staging copy has been consumed
    bool staged_pending = false;
    std::map<uint32_t, BatchGraph> graphs;   // by class mask
};

static void drop_graphs(BatchState *b) {
    for (auto &kv : b->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

static void state_free(BatchState *b) {
    if (!b) return;
    drop_graphs(b);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->fork) cudaEventDestroy(b->fork);
    for (int c = 0; c < kBatchClasses; ++c) {
        if (b->join[c]) cudaEventDestroy(b->join[c]);
        if (b->aux[c]) cudaStreamDestroy(b->aux[c]);
    }
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->dev);
    cudaFree(b->ctr);
    cudaFree(b->coop);
    cudaFreeHost(b->host);
    cudaFreeHost(b->host_status);
    delete b;
}

void batch_free(pfsm_ctx *ctx) {
    for (auto &kv : ctx->batch) state_free(kv.second);
    ctx->batch.clear();
}

static int state_reserve(pfsm_ctx *ctx, cudaStream_t s, size_t njobs, size_t nmachs,
                         BatchState **out) {
    BatchState *&b = ctx->batch[s];
    if (!b) {
        b = new BatchState();
        bool ok = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int c = 0; ok && c < kBatchClasses; ++c)
            ok = cudaStreamCreateWithFlags(&b->aux[c], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return PFSM_E_CUDA;
        }
    }
    if (njobs <= b->cap_jobs && nmachs <= b->cap_machs) {
        *out = b;
        return PFSM_OK;
    }
    // grow: everything captured so far refers to the old buffers
    if (b->staged_pending) cudaEventSynchronize(b->staged);
    b->staged_pending = false;
    cudaStreamSynchronize(s);
    drop_graphs(b);
    cudaFree(b->dev);
    cudaFree(b->ctr);
    cudaFreeHost(b->host);
    cudaFreeHost(b->host_status);
    b->dev = nullptr;
    b->ctr = nullptr;
    b->host = nullptr;
    b->host_status = nullptr;
    b->cap_jobs = std::max<size_t>(std::max<size_t>(njobs, 2 * b->cap_jobs), 256);
    b->cap_machs = std::max<size_t>(std::max<size_t>(nmachs, 2 * b->cap_machs), 16);
    b->off_jobs = align256(kBatchClasses * sizeof(BatchArgs));
    b->off_machs = align256(b->off_jobs + b->cap_jobs * sizeof(BatchJob));
    b->block_bytes = align256(b->off_machs + b->cap_machs * sizeof(DevMachine));
    const size_t ctr_bytes = 256 + align256((b->cap_jobs + 2) * 8) + static_cast<size_t>(kCarryCap) * 16;
    if (cudaMalloc(&b->dev, b->block_bytes) != cudaSuccess ||
        cudaMalloc(&b->ctr, ctr_bytes) != cudaSuccess ||
        cudaMallocHost(&b->host, b->block_bytes) != cudaSuccess ||
        cudaMallocHost(&b->host_status, (b->cap_jobs + 2) * 8) != cudaSuccess) {
        cudaGetLastError();
        b->cap_jobs = b->cap_machs = 0;
        return PFSM_E_NOMEM;
    }
    b->status = reinterpret_cast<unsigned long long *>(reinterpret_cast<uint8_t *>(b->ctr) + 256);
    b->carry = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(b->ctr) + 256 +
                                            align256((b->cap_jobs + 2) * 8));
    *out = b;
    return PFSM_OK;
}

// The launch shape of class `cls`: threads and CTAs per SM from the batch
// parameters (or the class default), everything but the table arena laid out
// by layout_smem, and the arena taking the rest of the CTA's share of the
// SM's shared memory. Shrinks the match staging, then the tile, then the
// thread count until an arena of kMinArena fits.
static int class_shape(pfsm_ctx *ctx, int cls) {
    BatchShape &sh = ctx->batch_shape[cls];
    if (sh.ready) return PFSM_OK;
    const int kind = cls >= 6 ? 1 : 0;
    // filtering threads per CTA (the kernel adds its producer warp): an NFA
    // class keeps 512 threads in all, so 15 filtering warps
    int threads = ctx->batch_threads ? ctx->batch_threads : (kind ? 512 : 256);
    if (kind && threads + 32 > 512) threads = 480;
    const int ctas = ctx->batch_ctas ? ctx->batch_ctas : (kind ? 1 : 2);
    uint32_t tile = ctx->batch_tile ? ctx->batch_tile : kBatchTile;
    // whole filter rounds (32 starts per filtering thread) per tile
    auto whole_rounds = [&](uint32_t t, int th) {
        const uint32_t round = 32u * static_cast<uint32_t>(th);
        return std::max(round, t / round * round);
    };
    tile = whole_rounds(tile, threads);
    ScanArgs a;
    memset(&a, 0, sizeof(a));
    a.stage_n = kind ? 32 : STAGE;
    // staged tiles: three for the NFA classes (one CTA per SM); two for the
    // DFA classes, whose two CTAs per SM share the shared memory with their
    // table arenas
    a.nbuf = kind ? 3 : 2;
    const uint32_t share = ctx->smem_sm / static_cast<uint32_t>(ctas);
    const uint32_t budget =
        std::min<uint32_t>(kSmemMax, share > ctx->smem_rsv ? share - ctx->smem_rsv : 0) - kBatchSmemStatic;
    uint32_t base = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        a.tile = tile;
        a.halo = kBatchHalo;
        a.text_buf = (tile + kBatchHalo + 32 + 127) & ~127u;
        base = layout_smem(a, kind ? 2 : 1, threads, SmemNeed{0u, 0u, 0u, 0u, 0u, 0u});
        if (base + kMinArena <= budget) break;
        if (a.stage_n > 32) a.stage_n = 32;
        else if (tile > 8192) tile = whole_rounds(8192, threads);
        else if (threads > 128) {
            threads /= 2;
            tile = whole_rounds(tile, threads);
        } else {
            return PFSM_E_INVAL;
        }
    }
    if (base + kMinArena > budget) return PFSM_E_INVAL;
    // the table arena comes first (offset 0: a machine's survival bitmap,
    // placed first in it, is where the kernels' check-free filter path
    // expects it); every other region moves up by its size
    const uint32_t arena = (budget - base) & ~127u;
    for (uint32_t *o : {&a.sm_misc, &a.sm_memo, &a.sm_tab, &a.sm_band, &a.sm_pool, &a.sm_surv,
                        &a.sm_list, &a.sm_text, &a.sm_pack, &a.sm_queue, &a.sm_stage, &a.sm_slots,
                        &a.sm_coop})
        *o += arena;
    const uint32_t smem = base + arena;
    const int occ = max_units_ctas_per_sm(cls, threads, smem);
    if (occ <= 0) return PFSM_E_INVAL;
    sh.threads = threads;
    sh.grid = ctx->nsm * std::min(occ, ctas);
    sh.smem = smem;
    sh.arena = arena;
    sh.layout = a;
    sh.ready = true;
    return PFSM_OK;
}

// Chooses which of a machine's tables go to the table arena (in order of
// use per start: survival bitmap, prefix table, DFA table, NFA band rows,
// NFA prefix records, the warp-wide NFA bitsets of `warps` warps) and
// returns the machine's class. With a deep bitmap in global memory few
// starts reach the prefix table, so it stays in global memory and leaves
// the arena to the rest.
static int place_tables(const Machine &m, uint32_t arena, int warps, DevMachine &d) {
    d.a_memo = d.a_tab = d.a_band = d.a_pool = d.a_surv = d.a_coop = kNotStaged;
    d.settle = m.params.settle > 0 ? m.params.settle : 0;
    d.lazy = m.params.partition == 1 || m.kind == 1 ? 1 : 0;
    uint32_t used = 0;
    auto take = [&](uint32_t bytes) {
        const uint32_t at = (used + 15) & ~15u;
        if (bytes == 0 || at + bytes > arena) return kNotStaged;
        used = at + bytes;
        return at;
    };
    const bool deep = !m.surv2.empty();
    if (!m.surv.empty()) d.a_surv = take(static_cast<uint32_t>(m.surv.size() * 4));
    if (!deep && d.memo_n > 0) d.a_memo = take(((d.memo_n + 1) / 2) * 4);
    if (m.kind == 0) {
        // table_smem 0: the DFA table stays in global memory (L2)
        if (m.params.table_smem != 0) d.a_tab = take(((static_cast<uint32_t>(m.Q) * m.S + 1) / 2) * 4);
    } else {
        if (!m.band.empty()) d.a_band = take(static_cast<uint32_t>(m.band.size() * 4));
        if (!m.pool.empty()) d.a_pool = take(static_cast<uint32_t>(m.pool.size() * 4));
        d.a_coop = take(static_cast<uint32_t>(warps * 2 * d.Wq * 4));
    }
    return batch_class(m.kind, m.sbits, m.k, m.kind == 0 && d.a_tab != kNotStaged);
}

struct BatchPlan {
    std::vector<BatchJob> jobs;
    std::vector<DevMachine> machs;
    std::vector<Machine *> used;            // the machines the batch reads
    uint32_t mask = 0;                      // classes with work
    uint32_t job_lo[kBatchClasses] = {}, job_hi[kBatchClasses] = {};
    uint32_t nunits[kBatchClasses] = {}, unit_tiles[kBatchClasses] = {};
    int32_t wq[kBatchClasses] = {};         // NFA: widest bitset kept in global scratch (words)
};

// Validate the jobs, make their machines resident, classify them and cut
// every class's texts into work units.
static int plan_batch(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, BatchPlan &pl,
                      cudaStream_t s) {
    NvtxRange nr("pfsm batch plan");
    ctx->epoch++;
    // machine slot of every job (slots numbered in order of first use)
    std::map<int, uint32_t> slot_of;
    std::vector<int> ids;
    std::vector<uint32_t> job_slot(static_cast<size_t>(k));
    int last_aut = 0;
    uint32_t last_slot = 0xFFFFFFFFu;
    for (int32_t i = 0; i < k; ++i) {
        const pfsm_job &j = jobs[i];
        if (j.reserved != 0 || j.n >= (1ull << 32) || (j.n > 0 && !j.text)) return PFSM_E_INVAL;
        if (last_slot == 0xFFFFFFFFu || j.aut != last_aut) {
            auto f = slot_of.find(j.aut);
            if (f == slot_of.end()) {
                auto it = ctx->machines.find(j.aut);
                if (it == ctx->machines.end()) return PFSM_E_NOENT;
                it->second.pin = ctx->epoch;
                f = slot_of.emplace(j.aut, static_cast<uint32_t>(ids.size())).first;
                ids.push_back(j.aut);
            }
            last_aut = j.aut;
            last_slot = f->second;
        }
        job_slot[i] = last_slot;
    }
    if (ids.size() >= (1u << 24)) return PFSM_E_INVAL;
    for (int id : ids) {
        int st = make_resident(ctx, id, ctx->machines[id], s);
        if (st) return st;
    }
    // the DFA classes share one shape (threads, arena), as do the NFA classes
    int st = class_shape(ctx, 0);
    if (!st) st = class_shape(ctx, 6);
    if (st) return st;
    for (int c = 1; c < kBatchClasses && !st; ++c)
        if (!ctx->batch_shape[c].ready) st = class_shape(ctx, c);
    if (st) return st;
    std::vector<int> cls_of(ids.size());
    for (size_t i = 0; i < ids.size(); ++i) {
        Machine &m = ctx->machines[ids[i]];
        DevMachine d = m.dm;
        const BatchShape &sh = ctx->batch_shape[m.kind == 1 ? 6 : 0];
        pl.used.push_back(&m);
        cls_of[i] = place_tables(m, sh.arena, sh.threads / 32, d);
        if (m.kind == 1 && d.a_coop == kNotStaged) pl.wq[cls_of[i]] = std::max(pl.wq[cls_of[i]], d.Wq);
        pl.machs.push_back(d);
    }
    // jobs grouped by class, then by machine, so that consecutive units share
    // tables, keeping the order of the caller's jobs within a machine: a
    // counting sort over the machine slots, taken in (class, slot) order
    std::vector<uint32_t> slot_order(ids.size());
    for (size_t i = 0; i < ids.size(); ++i) slot_order[i] = static_cast<uint32_t>(i);
    std::sort(slot_order.begin(), slot_order.end(), [&](uint32_t x, uint32_t y) {
        return cls_of[x] != cls_of[y] ? cls_of[x] < cls_of[y] : x < y;
    });
    std::vector<uint32_t> first(ids.size() + 1, 0);
    for (int32_t i = 0; i < k; ++i) first[job_slot[i] + 1]++;
    {
        std::vector<uint32_t> count(first.begin() + 1, first.end());
        uint32_t at = 0;
        for (uint32_t sl : slot_order) {
            first[sl] = at;
            at += count[sl];
        }
    }
    std::vector<uint32_t> key(static_cast<size_t>(k));   // job indices in (class, slot, index) order
    for (int32_t i = 0; i < k; ++i) key[first[job_slot[i]]++] = static_cast<uint32_t>(i);
    uint64_t tiles_of[kBatchClasses] = {};
    for (int32_t i = 0; i < k; ++i) {
        const int c = cls_of[job_slot[i]];
        tiles_of[c] += (jobs[i].n + ctx->batch_shape[c].layout.tile - 1) / ctx->batch_shape[c].layout.tile;
    }
    // units of up to kUnitTilesMax tiles, fewer when a class has too little
    // work for about four units per CTA
    for (int c = 0; c < kBatchClasses; ++c) {
        const uint64_t per = tiles_of[c] / (4ull * std::max(1, ctx->batch_shape[c].grid));
        pl.unit_tiles[c] = static_cast<uint32_t>(std::min<uint64_t>(kUnitTilesMax, std::max<uint64_t>(1, per)));
    }
    int cur = -1;
    pl.jobs.reserve(static_cast<size_t>(k));
    for (int32_t r = 0; r < k; ++r) {
        const int32_t x = static_cast<int32_t>(key[r]);
        const pfsm_job &j = jobs[x];
        const uint32_t slot = job_slot[x];
        const int c = cls_of[slot];
        if (c != cur) {
            if (cur >= 0) pl.job_hi[cur] = static_cast<uint32_t>(pl.jobs.size());
            pl.job_lo[c] = static_cast<uint32_t>(pl.jobs.size());
            cur = c;
        }
        const uint32_t tile = ctx->batch_shape[c].layout.tile;
        BatchJob b{};
        b.text = j.text;
        b.n = static_cast<uint32_t>(j.n);
        b.mach = slot;
        b.orig = static_cast<uint32_t>(x);
        b.ntiles = static_cast<uint32_t>((j.n + tile - 1) / tile);
        b.unit_begin = pl.nunits[c];
        const uint64_t units = (b.ntiles + pl.unit_tiles[c] - 1) / pl.unit_tiles[c];
        if (pl.nunits[c] + units >= (1ull << 32)) return PFSM_E_INVAL;
        pl.nunits[c] += static_cast<uint32_t>(units);
        pl.jobs.push_back(b);
    }
    if (cur >= 0) pl.job_hi[cur] = static_cast<uint32_t>(pl.jobs.size());
    for (int c = 0; c < kBatchClasses; ++c)
        if (pl.nunits[c] > 0) pl.mask |= 1u << c;
    return PFSM_OK;
}

// The graph of one class set: resets, one branch per class, the carry kernel.
static int graph_for(pfsm_ctx *ctx, BatchState *b, uint32_t mask, cudaGraphExec_t *out) {
    BatchGraph &bg = b->graphs[mask];
    if (bg.exec && bg.gen == ctx->batch_gen) {
        *out = bg.exec;
        return PFSM_OK;
    }
    if (bg.exec) {
        cudaGraphExecDestroy(bg.exec);
        bg.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PFSM_E_CUDA;
    const BatchArgs *dargs = reinterpret_cast<const BatchArgs *>(b->dev);
    cudaError_t e = cudaMemsetAsync(b->ctr, 0, 256, b->capture);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, (b->cap_jobs + 2) * 8, b->capture);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->capture);
    int carry_cls = -1;
    for (int c = 0; c < kBatchClasses && e == cudaSuccess; ++c) {
        if (!(mask & (1u << c))) continue;
        if (c < 6 && carry_cls < 0) carry_cls = c;
        const BatchShape &sh = ctx->batch_shape[c];
        e = cudaStreamWaitEvent(b->aux[c], b->fork, 0);
        if (e == cudaSuccess) e = launch_units(c, dargs + c, sh.threads, sh.grid, sh.smem, b->aux[c]);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[c], b->aux[c]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, b->join[c], 0);
    }
    if (e == cudaSuccess && carry_cls >= 0)
        e = launch_carry_batch(dargs + carry_cls, 2 * ctx->nsm, b->capture);
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    e = cudaGraphInstantiate(&bg.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bg.exec = nullptr;
        return PFSM_E_CUDA;
    }
    bg.gen = ctx->batch_gen;
    *out = bg.exec;
    return PFSM_OK;
}

// Enqueue one batch on `s`; on return the batch's status block lives in
// b->status (device): [0] total, [1] error bits, [2 + i] count of job i.
static int batch_enqueue(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, pfsm_bmatch *out,
                         uint64_t cap, cudaStream_t s, BatchState **bs) {
    NvtxRange nr("pfsm batch (plan, graph launch)");
    BatchPlan pl;
    int st = plan_batch(ctx, jobs, k, pl, s);
    // the pins protect this batch's machines while it is planned; once its
    // pointers are recorded they may be evicted again (an eviction frees
    // device memory with cudaFree, which waits for work in flight)
    ctx->epoch++;
    if (st) return st;
    BatchState *b = nullptr;
    st = state_reserve(ctx, s, std::max<size_t>(1, pl.jobs.size()), std::max<size_t>(1, pl.machs.size()), &b);
    if (st) return st;
    if (b->staged_pending) cudaEventSynchronize(b->staged);   // staging buffer is free again
    // warp bitsets of the NFA classes, one region per class
    size_t coop_need = 0, coop_off[kBatchClasses] = {};
    for (int c = 6; c < kBatchClasses; ++c) {
        if (!(pl.mask & (1u << c)) || pl.wq[c] <= 0) continue;
        const BatchShape &sh = ctx->batch_shape[c];
        coop_off[c] = coop_need;
        coop_need += static_cast<size_t>(sh.grid) * (sh.threads / 32) * 2 * pl.wq[c];
    }
    if (coop_need && ensure_words(&b->coop, &b->coop_words, coop_need)) return PFSM_E_NOMEM;
    BatchArgs args[kBatchClasses];
    memset(args, 0, sizeof(args));
    // every class gets valid arguments: the graph launches all of them, and
    // a class without units claims nothing and exits
    for (int c = 0; c < kBatchClasses; ++c) {
        const BatchShape &sh = ctx->batch_shape[c];
        BatchArgs &A = args[c];
        A.sa = sh.layout;
        A.sa.out = reinterpret_cast<uint32_t *>(out);
        A.sa.cap = cap;
        A.sa.status = b->status;
        A.sa.carry = b->carry;
        A.sa.carry_n = b->ctr + kCarryCtr;
        A.sa.carry_cap = kCarryCap;
        A.sa.Wq = pl.wq[c];
        A.sa.coop_g = (c >= 6 && pl.wq[c] > 0) ? b->coop + coop_off[c] : nullptr;
        A.nunits = pl.nunits[c];
        A.job_lo = pl.job_lo[c];
        A.job_hi = pl.job_hi[c];
        A.unit_tiles = pl.unit_tiles[c];
        A.sm_arena = 0;   // the arena is the first region (see class_shape)
        A.unit_counter = b->ctr + c;
        A.jobs = reinterpret_cast<const BatchJob *>(b->dev + b->off_jobs);
        A.machs = reinterpret_cast<const DevMachine *>(b->dev + b->off_machs);
        A.job_counts = b->status + 2;
    }
    memcpy(b->host, args, sizeof(args));
    if (!pl.jobs.empty())
        memcpy(b->host + b->off_jobs, pl.jobs.data(), pl.jobs.size() * sizeof(BatchJob));
    if (!pl.machs.empty())
        memcpy(b->host + b->off_machs, pl.machs.data(), pl.machs.size() * sizeof(DevMachine));
    const size_t used = b->off_machs + pl.machs.size() * sizeof(DevMachine);
    if (cudaMemcpyAsync(b->dev, b->host, used, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PFSM_E_CUDA;
    cudaEventRecord(b->staged, s);
    b->staged_pending = true;
    cudaGraphExec_t exec = nullptr;
    st = graph_for(ctx, b, kAllClasses, &exec);
    if (st) return st;
    int ev = -1;
    Slot *slot = ctx->timing ? get_slot(ctx, s) : nullptr;
    if (slot) {
        collect_timing(ctx, slot, kEventRing - 1);
        ev = slot->ev_head;
        cudaEventRecord(slot->ev[2 * ev], s);
    }
    if (cudaGraphLaunch(exec, s) != cudaSuccess) return PFSM_E_CUDA;
    st = mark_use(ctx, s, pl.used.data(), pl.used.size());
    if (st) return st;
    if (slot) {
        cudaEventRecord(slot->ev[2 * ev + 1], s);
        slot->ev_head = (slot->ev_head + 1) % kEventRing;
        slot->ev_pending++;
    }
    *bs = b;
    return PFSM_OK;
}

}  // namespace pfsm

using namespace pfsm;

extern "C" int pfsm_scan_batch_async(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k,
                                     pfsm_bmatch *out_dev, uint64_t cap, uint64_t *status_dev,
                                     void *stream) {
    if (!ctx || k < 0 || (k > 0 && !jobs) || !status_dev || (cap > 0 && !out_dev))
        return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchState *b = nullptr;
    int st = batch_enqueue(ctx, jobs, k, out_dev, cap, s, &b);
    if (st) return st;
    if (cudaMemcpyAsync(status_dev, b->status, (static_cast<size_t>(k) + 2) * 8,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PFSM_E_CUDA;
    return PFSM_OK;
}

extern "C" int pfsm_set_batch_params(pfsm_ctx *ctx, const pfsm_params *p) {
    if (!ctx) return PFSM_E_INVAL;
    const int threads = p ? p->threads : 0;
    const int tile = p ? p->tile : 0;
    const int ctas = p ? p->ctas_per_sm : 0;
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512) return PFSM_E_INVAL;
    if (tile != 0 && (tile < 4096 || tile > 32768 || tile % 4096)) return PFSM_E_INVAL;
    if (ctas < 0 || ctas > 4) return PFSM_E_INVAL;
    ctx->batch_threads = threads;
    ctx->batch_ctas = ctas;
    ctx->batch_tile = tile ? static_cast<uint32_t>(tile) : kBatchTile;
    for (int c = 0; c < kBatchClasses; ++c) ctx->batch_shape[c].ready = false;
    ctx->batch_gen++;   // captured graphs hold the old shapes
    return PFSM_OK;
}

extern "C" int pfsm_scan_batch(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k,
                               pfsm_bmatch *out_dev, uint64_t cap, uint64_t *counts,
                               uint64_t *total, void *stream) {
    if (!ctx || k < 0 || (k > 0 && !jobs) || !total || (cap > 0 && !out_dev)) return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchState *b = nullptr;
    int st = batch_enqueue(ctx, jobs, k, out_dev, cap, s, &b);
    if (st) return st;
    if (cudaMemcpyAsync(b->host_status, b->status, (static_cast<size_t>(k) + 2) * 8,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PFSM_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PFSM_E_CUDA;
    b->staged_pending = false;
    if (counts)
        for (int32_t i = 0; i < k; ++i) counts[i] = b->host_status[2 + i];
    return finish_status(b->host_status, cap, total);
}

// A union machine (Sec. III.A): k automata over one text. The union through
// an ancillary initial state with epsilon edges to every component's q0 has
// exactly the union of the components' match sets, so it runs as a batch of
// k jobs on the same text; a match's text field is its component's index.
extern "C" int pfsm_scan_union_async(pfsm_ctx *ctx, const pfsm_aut *auts, int32_t k,
                                     const uint8_t *text_dev, uint64_t n, pfsm_bmatch *out_dev,
                                     uint64_t cap, uint64_t *status_dev, void *stream) {
    if (!ctx || k < 0 || (k > 0 && !auts) || (n > 0 && !text_dev)) return PFSM_E_INVAL;
    std::vector<pfsm_job> jobs(static_cast<size_t>(k));
    for (int32_t i = 0; i < k; ++i) jobs[i] = pfsm_job{auts[i], 0u, text_dev, n};
    return pfsm_scan_batch_async(ctx, jobs.data(), k, out_dev, cap, status_dev, stream);
}

extern "C" int pfsm_scan_union(pfsm_ctx *ctx, const pfsm_aut *auts, int32_t k,
                               const uint8_t *text_dev, uint64_t n, pfsm_bmatch *out_dev,
                               uint64_t cap, uint64_t *counts, uint64_t *total, void *stream) {
    if (!ctx || k < 0 || (k > 0 && !auts) || (n > 0 && !text_dev)) return PFSM_E_INVAL;
    std::vector<pfsm_job> jobs(static_cast<size_t>(k));
    for (int32_t i = 0; i < k; ++i) jobs[i] = pfsm_job{auts[i], 0u, text_dev, n};
    return pfsm_scan_batch(ctx, jobs.data(), k, out_dev, cap, counts, total, stream);
}
