// Batched scans: many texts, each with its own machine, in one persistent
// launch. This combines the two partitionings of Sec. III.D: the set of
// machines is split across texts (regex partitioning) and every text is cut
// into tiles (data partitioning); every (text, tile) pair is one work item
// pulled by persistent CTAs from a global counter.
//
// The launch sequence (counter and status resets, the persistent kernel, the
// carry kernel) is captured once per stream and layout as a CUDA graph and
// replayed for every batch; the per-batch job table, machine table and
// kernel arguments are copied to a fixed device block before each replay.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pfsm_host.h"

namespace pfsm {

constexpr uint32_t kBatchTile = 16384;
constexpr uint32_t kBatchHalo = 2048;
constexpr uint32_t kBatchTabMax = 32768;   // DFA tables up to this size go to smem

struct BatchState {
    cudaStream_t capture = nullptr;   // private stream used to capture the graph
    size_t cap_jobs = 0, cap_machs = 0;
    size_t off_jobs = 0, off_machs = 0, block_bytes = 0;
    uint8_t *dev = nullptr;           // BatchArgs | jobs | machines
    uint8_t *host = nullptr;          // pinned staging of the same layout
    uint32_t *ctr = nullptr;          // device: [0] item counter, [1] carry count
    unsigned long long *status = nullptr;       // device: total, errors, per-job counts
    unsigned long long *host_status = nullptr;  // pinned copy of status
    uint32_t *carry = nullptr;
    uint32_t *coop = nullptr;         // warp-wide NFA bitsets
    size_t coop_words = 0;
    cudaEvent_t staged = nullptr;     // previous staging copy has been consumed
    bool staged_pending = false;
    cudaGraphExec_t exec = nullptr;
    uint32_t g_smem = 0;
    int g_threads = 0, g_grid = 0;
};

static void state_free(BatchState *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->staged) cudaEventDestroy(b->staged);
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
        if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess) {
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
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
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
    b->off_jobs = align256(sizeof(BatchArgs));
    b->off_machs = align256(b->off_jobs + b->cap_jobs * sizeof(BatchJob));
    b->block_bytes = align256(b->off_machs + b->cap_machs * sizeof(DevMachine));
    const size_t ctr_bytes = 256 + (b->cap_jobs + 2) * 8 + static_cast<size_t>(kCarryCap) * 16;
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

struct BatchPlan {
    std::vector<BatchJob> jobs;
    std::vector<DevMachine> machs;
    ScanArgs sa{};
    uint32_t nitems = 0;
    int threads = 256, grid = 1;
    uint32_t smem = 0;
};

// Validate the jobs, make their machines resident and lay out the launch.
static int plan_batch(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, BatchPlan &pl) {
    ctx->epoch++;
    std::map<int, uint32_t> slot_of;
    std::vector<int> ids;
    for (int32_t i = 0; i < k; ++i) {
        const pfsm_job &j = jobs[i];
        if (j.reserved != 0 || j.n >= (1ull << 32) || (j.n > 0 && !j.text)) return PFSM_E_INVAL;
        auto it = ctx->machines.find(j.aut);
        if (it == ctx->machines.end()) return PFSM_E_NOENT;
        if (!slot_of.count(j.aut)) {
            slot_of[j.aut] = static_cast<uint32_t>(ids.size());
            ids.push_back(j.aut);
            it->second.pin = ctx->epoch;
        }
    }
    for (int id : ids) {
        int st = make_resident(ctx, id, ctx->machines[id]);
        if (st) return st;
    }
    uint32_t memo_max = 0, tab_max = 0, band_max = 0, pool_max = 0, surv_max = 0;
    int32_t wq_max = 0;
    int kmask = 0;
    for (int id : ids) {
        Machine &m = ctx->machines[id];
        DevMachine d = m.dm;
        const uint32_t tab_bytes = m.kind == 0 ? ((static_cast<uint32_t>(m.Q) * m.S + 1) / 2) * 4 : 0;
        d.tab_smem = (m.kind == 0 && tab_bytes <= kBatchTabMax) ? 1 : 0;
        if (d.tab_smem) tab_max = std::max(tab_max, tab_bytes);
        const uint32_t band_bytes = static_cast<uint32_t>(m.band.size() * 4);
        const uint32_t pool_bytes = m.kind == 1 ? static_cast<uint32_t>(m.pool.size() * 4) : 0;
        d.band_smem = band_bytes > 0 && band_bytes <= kBatchTabMax * 2;
        d.pool_smem = pool_bytes > 0 && pool_bytes <= kBatchTabMax * 2;
        if (d.band_smem) band_max = std::max(band_max, band_bytes);
        if (d.pool_smem) pool_max = std::max(pool_max, pool_bytes);
        d.memo_smem = m.surv2.empty() && d.memo_n > 0;
        if (d.memo_smem) memo_max = std::max(memo_max, d.memo_n);
        if (!m.surv2.empty()) d.pool_smem = 0;
        surv_max = std::max(surv_max, static_cast<uint32_t>(m.surv.size() * 4));
        if (m.kind == 1) wq_max = std::max(wq_max, d.Wq);
        kmask |= m.kind == 0 ? 1 : 2;
        pl.machs.push_back(d);
    }
    // jobs ordered by machine, so that consecutive items share tables
    std::vector<int32_t> order(k);
    for (int32_t i = 0; i < k; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return slot_of[jobs[x].aut] < slot_of[jobs[y].aut];
    });
    // launch geometry: shrink until the layout fits one CTA's shared memory
    ScanArgs &a = pl.sa;
    memset(&a, 0, sizeof(a));
    a.memo_n = memo_max;
    a.Wq = wq_max;
    a.stage_n = (kmask & 1) ? STAGE : 32;
    a.settle_steps = 8;
    uint32_t tile = ctx->batch_tile ? ctx->batch_tile : kBatchTile;
    int threads = ctx->batch_threads ? ctx->batch_threads : 256;
    uint32_t smem = 0;
    bool fit = false;
    a.qcap = static_cast<uint32_t>(FILTER_SPT) * threads;
    for (int attempt = 0; attempt < 12 && !fit; ++attempt) {
        a.tile = tile;
        a.halo = kBatchHalo;
        a.text_buf = (tile + kBatchHalo + 16 + 127) & ~127u;
        const SmemNeed need{memo_max ? ((memo_max + 1) / 2) * 4 + 4 : 0u, tab_max, band_max,
                            pool_max, surv_max};
        smem = layout_smem(a, kmask, threads, need);
        if (smem <= kSmemMax - kSmemStatic) { fit = true; break; }
        if (a.stage_n > 32) {
            a.stage_n = 32;
        } else if (pool_max) {
            pool_max = 0;
            for (auto &d : pl.machs) d.pool_smem = 0;
        } else if (tile > 8192) {
            tile = 8192;
        } else if (band_max) {
            band_max = 0;
            for (auto &d : pl.machs) d.band_smem = 0;
        } else if (tab_max) {
            tab_max = 0;
            for (auto &d : pl.machs) d.tab_smem = 0;
        } else if (threads > 128) {
            threads /= 2;
            a.qcap = static_cast<uint32_t>(FILTER_SPT) * threads;
        } else {
            break;
        }
    }
    if (!fit) return PFSM_E_INVAL;
    uint32_t item = 0;
    for (int32_t x : order) {
        const pfsm_job &j = jobs[x];
        BatchJob b{};
        b.text = j.text;
        b.n = static_cast<uint32_t>(j.n);
        b.mach = slot_of[j.aut];
        b.orig = static_cast<uint32_t>(x);
        b.tile_begin = item;
        const uint64_t tiles = (j.n + a.tile - 1) / a.tile;
        if (item + tiles >= (1ull << 32)) return PFSM_E_INVAL;
        item += static_cast<uint32_t>(tiles);
        pl.jobs.push_back(b);
    }
    pl.nitems = item;
    int occ = max_batch_ctas_per_sm(threads, smem);
    if (occ <= 0) return PFSM_E_INVAL;
    pl.threads = threads;
    pl.smem = smem;
    pl.grid = ctx->nsm * occ;
    return PFSM_OK;
}

static int capture_graph(BatchState *b, const BatchPlan &pl, int nsm) {
    if (b->exec && b->g_smem == pl.smem && b->g_threads == pl.threads && b->g_grid == pl.grid)
        return PFSM_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PFSM_E_CUDA;
    const BatchArgs *dargs = reinterpret_cast<const BatchArgs *>(b->dev);
    cudaMemsetAsync(b->ctr, 0, 8, b->capture);
    cudaMemsetAsync(b->status, 0, (b->cap_jobs + 2) * 8, b->capture);
    cudaError_t e = launch_batch(dargs, pl.threads, pl.grid, pl.smem, b->capture);
    if (e == cudaSuccess) e = launch_carry_batch(dargs, 2 * nsm, b->capture);
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->exec = nullptr;
        return PFSM_E_CUDA;
    }
    b->g_smem = pl.smem;
    b->g_threads = pl.threads;
    b->g_grid = pl.grid;
    return PFSM_OK;
}

// Enqueue one batch on `s`; on return the batch's status block lives in
// b->status (device): [0] total, [1] error bits, [2 + i] count of job i.
static int batch_enqueue(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k, pfsm_bmatch *out,
                         uint64_t cap, cudaStream_t s, BatchState **bs) {
    BatchPlan pl;
    int st = plan_batch(ctx, jobs, k, pl);
    // the pins protect this batch's machines while it is planned; once its
    // pointers are recorded they may be evicted again (an eviction frees
    // device memory with cudaFree, which waits for work in flight)
    ctx->epoch++;
    if (st) return st;
    BatchState *b = nullptr;
    st = state_reserve(ctx, s, std::max<size_t>(1, pl.jobs.size()), std::max<size_t>(1, pl.machs.size()), &b);
    if (st) return st;
    if (b->staged_pending) cudaEventSynchronize(b->staged);   // staging buffer is free again
    // kernel arguments
    BatchArgs args{};
    args.sa = pl.sa;
    args.sa.out = reinterpret_cast<uint32_t *>(out);
    args.sa.cap = cap;
    args.sa.status = b->status;
    args.sa.carry = b->carry;
    args.sa.carry_n = b->ctr + 1;
    args.sa.carry_cap = kCarryCap;
    args.nitems = pl.nitems;
    args.njobs = static_cast<uint32_t>(pl.jobs.size());
    args.item_counter = b->ctr;
    args.jobs = reinterpret_cast<const BatchJob *>(b->dev + b->off_jobs);
    args.machs = reinterpret_cast<const DevMachine *>(b->dev + b->off_machs);
    args.job_counts = b->status + 2;
    if (pl.sa.Wq > 0) {
        const size_t need = static_cast<size_t>(pl.grid) * (pl.threads / 32) * 2 * pl.sa.Wq;
        if (ensure_words(&b->coop, &b->coop_words, need)) return PFSM_E_NOMEM;
        args.sa.coop_g = b->coop;
    }
    memcpy(b->host, &args, sizeof(args));
    if (!pl.jobs.empty())
        memcpy(b->host + b->off_jobs, pl.jobs.data(), pl.jobs.size() * sizeof(BatchJob));
    if (!pl.machs.empty())
        memcpy(b->host + b->off_machs, pl.machs.data(), pl.machs.size() * sizeof(DevMachine));
    const size_t used = b->off_machs + pl.machs.size() * sizeof(DevMachine);
    if (cudaMemcpyAsync(b->dev, b->host, used, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PFSM_E_CUDA;
    cudaEventRecord(b->staged, s);
    b->staged_pending = true;
    st = capture_graph(b, pl, ctx->nsm);
    if (st) return st;
    int ev = -1;
    Slot *slot = ctx->timing ? get_slot(ctx, s) : nullptr;
    if (slot) {
        collect_timing(ctx, slot, kEventRing - 1);
        ev = slot->ev_head;
        cudaEventRecord(slot->ev[2 * ev], s);
    }
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return PFSM_E_CUDA;
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
    if (threads != 0 && threads != 128 && threads != 256) return PFSM_E_INVAL;
    if (tile != 0 && (tile < 4096 || tile > 32768 || tile % 4096)) return PFSM_E_INVAL;
    ctx->batch_threads = threads ? threads : 256;
    ctx->batch_tile = tile ? static_cast<uint32_t>(tile) : kBatchTile;
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
