// Host-side state of libpfsm shared by the API translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pfsm_internal.h"

namespace pfsm {

constexpr uint64_t kDefaultBudget = 8ull << 30;
constexpr uint32_t kCarryCap = 1u << 20;     // carry entries per stream slot
constexpr uint32_t kSmemMax = 232448;        // opt-in shared memory per CTA
constexpr uint32_t kSmemStatic = 1024;       // room left for static shared memory (single-text kernels: none)
constexpr uint32_t kBatchSmemStatic = 2048;  // the batch class kernels' static shared memory (1.5 KB)
constexpr int kEventRing = 256;              // timed launches kept in flight per stream

struct Machine {
    int kind = 0;  // 0 DFA, 1 NFA
    int Q = 0, S = 0, q0 = 0, dead = -1;
    std::vector<uint8_t> fin;
    // device encodings (host images)
    std::vector<uint16_t> dtab;       // DFA [Q][S]
    std::vector<uint32_t> off;        // NFA CSR [Q*S+1]
    std::vector<uint16_t> tgt;        // NFA targets
    // NFA with epsilon edges kept (step 2 of Sec. III.B at run time): the
    // states each state reaches through epsilon edges (itself excluded),
    // CSR by state, final bit as in tgt; empty without epsilon edges
    std::vector<uint32_t> ecl_off;
    std::vector<uint16_t> ecl_tgt;
    // start-prefix table
    int k = 0, sbits = 1;
    std::vector<uint16_t> memo;
    std::vector<uint16_t> tail;       // NFA: records of the j-grams, 0 < j < k (text ends)
    std::vector<uint32_t> pool;
    std::vector<uint16_t> l2tab;      // NFA: second-level tables (see L2_SYMS) or empty
    std::vector<uint32_t> pool2;      // NFA: second-level records
    std::vector<uint16_t> memox;      // NFA: second-level set index per k-gram, or empty
    std::vector<uint32_t> band;   // NFA band image (S <= 4) or empty
    // survival bitmap over m-grams (m = 0: none)
    int sm_m = 0, sm_m2 = 0;
    std::vector<uint32_t> surv, surv2;   // shallow (shared memory) and deep (global) bitmaps
    pfsm_params params{};
    // residency: the device image is built once in pinned host memory and
    // copied in on the scan's stream whenever the machine becomes resident
    void *dev = nullptr;
    size_t dev_bytes = 0;
    uint8_t *host_img = nullptr;      // pinned copy of the device image
    size_t img_bytes = 0;
    size_t o_memo = 0, o_tail = 0, o_surv = 0, o_surv2 = 0, o_tab = 0, o_off = 0,
           o_tgt = 0, o_pool = 0, o_band = 0, o_eoff = 0, o_etgt = 0, o_l2tab = 0,
           o_pool2 = 0, o_memox = 0;   // section offsets
    cudaEvent_t ready = nullptr;      // recorded after the last upload
    // last use per stream (an event recorded after a launch that read the
    // image); an eviction orders its free after every one of them
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
    DevMachine dm{};
    uint64_t last_use = 0;
    uint64_t pin = 0;        // batch epoch that needs it resident
    bool was_resident = false;
};

struct Slot {   // per-stream scratch
    unsigned long long *status = nullptr;   // device [2]
    uint32_t *carry_n = nullptr;
    uint32_t *carry = nullptr;              // kCarryCap entries of 4 words
    unsigned long long *host_status = nullptr;   // pinned [2]
    uint32_t *coop = nullptr;               // warp-wide NFA bitsets
    size_t coop_words = 0;
    // ring of (start, end) events around timed tile-kernel launches
    cudaEvent_t ev[2 * kEventRing] = {};
    int ev_head = 0, ev_pending = 0;
};

struct BatchState;   // batch.cu

constexpr int kUseRing = 64;   // use events kept per stream
struct UseRing {             // events marking launches that read machine images
    cudaEvent_t ev[kUseRing] = {};
    int head = 0;
};

// Launch shape of one batch class (batch.cu), fixed per context until the
// batch parameters change: the layout of everything but the table arena,
// and the arena's size.
struct BatchShape {
    bool ready = false;
    int threads = 0, grid = 0;
    uint32_t smem = 0, arena = 0;
    ScanArgs layout{};
};

// An NVTX range over a scope (load, table build, scan, carry, batch planning
// and launch, reload, eviction), for timeline profilers; without a profiler
// attached each push and pop is a call that returns at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace pfsm

struct pfsm_ctx {
    int device = 0;
    int nsm = 0;
    uint64_t budget = pfsm::kDefaultBudget;
    uint64_t resident_bytes = 0;
    uint64_t clock = 0;
    uint64_t epoch = 0;
    uint64_t n_loads = 0, n_evict = 0, n_reload = 0;
    std::map<int, pfsm::Machine> machines;
    int next_id = 1;
    std::map<cudaStream_t, pfsm::Slot> slots;
    cudaMemPool_t pool = nullptr;     // stream-ordered pool of machine images
    // unloaded machines whose images scans in flight still read: freed when
    // their last uses complete (or evicted in stream order when room is needed)
    std::vector<pfsm::Machine> retired;
    std::map<cudaStream_t, pfsm::UseRing> use_rings;
    std::mutex mu;
    bool timing = false;
    bool hold_tiles = false;   // test hook: scans time out (see pfsm_test_hold_tiles)
    uint32_t test_carry_cap = 0, test_cpool_cap = 0;   // see pfsm_test_carry_cap
    double time_ms = 0.0;
    uint64_t time_launches = 0;
    // batch executors, one per stream (batch.cu), and their launch shape
    std::map<cudaStream_t, pfsm::BatchState *> batch;
    int batch_threads = 0;        // 0: per-class default
    int batch_ctas = 0;           // CTAs per SM, 0: per-class default
    uint32_t batch_tile = 16384;
    uint64_t batch_gen = 1;       // bumped when the batch parameters change
    pfsm::BatchShape batch_shape[pfsm::kBatchClasses];
    uint32_t smem_sm = 233472;    // shared memory per SM
    uint32_t smem_rsv = 1024;     // shared memory the system reserves per CTA
};

namespace pfsm {

int ceil_log2(int S);
bool build_memo(Machine &m);
void build_survival(Machine &m);
size_t align256(size_t x);
void release(pfsm_ctx *ctx, Machine &m);
void drop_host_image(Machine &m);
void sweep_retired(pfsm_ctx *ctx);
int make_resident(pfsm_ctx *ctx, int id, Machine &m, cudaStream_t s);
int mark_use(pfsm_ctx *ctx, cudaStream_t s, Machine *const *ms, size_t k);
Slot *get_slot(pfsm_ctx *ctx, cudaStream_t s);
int ensure_words(uint32_t **buf, size_t *have, size_t need);
void collect_timing(pfsm_ctx *ctx, Slot *slot, int keep);
int finish_status(const unsigned long long *hs, uint64_t cap, uint64_t *n_matches);
void batch_free(pfsm_ctx *ctx);

}  // namespace pfsm
