// Allocation-free DFA scan.
//
// Some callers cannot allocate device memory at all: plugins handed
// pre-allocated buffers by a host application, processes whose device memory
// is entirely owned by another allocator (a framework's caching pool), or
// latency-critical loops that must never call cudaMalloc/cudaFree because
// those calls synchronise the device. pfsm_scan_dfa_noalloc serves them: it
// takes the DFA table, the text and the outputs as the caller's device
// buffers, and keeps everything else it needs (status words, the encoded
// table, the carry queue) in one file-scope __device__ array below, so it
// calls no allocating routine.
//
// The array is a fixed kNoAllocBytes per device, held by every device that
// loads this library until the process exits. The driver reserves it when it
// loads this file's module: with lazy module loading (the CUDA default) that
// is the first call on a device, so such callers make that first call before
// another allocator takes the device's memory (CUDA_MODULE_LOADING=EAGER
// reserves it when the library is loaded). All calls on a device share
// it: calls whose work overlaps on the GPU (for example on two streams)
// race on it, so a caller issues them on one stream or waits between them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "pfsm_host.h"

namespace pfsm {

constexpr size_t kNoAllocBytes = 4u << 20;          // the whole array: 4 MiB
constexpr size_t kNoAllocHeader = 256;              // status[2], carry count
constexpr size_t kNoAllocTable = 1u << 20;          // encoded table: Q*S <= 512 Ki entries
constexpr size_t kNoAllocCarry = kNoAllocBytes - kNoAllocHeader - kNoAllocTable;
constexpr unsigned long long ERR_TABLE = 4ull;      // the caller's table is malformed

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

namespace {
struct NoAllocDevice {
    uint8_t *scratch = nullptr;   // device address of g_noalloc_scratch
    int nsm = 0;
};
std::mutex g_noalloc_mu;
int g_noalloc_nsm[128];   // SM count per device index (0: not read yet)

// The array's device address for the current device. The name is only a
// host-side stand-in in host code, so the address is looked up on every
// call: after cudaDeviceReset, or when the primary context is released and
// created again, the module is loaded anew and the array may sit elsewhere.
// Once the module is loaded the lookup allocates nothing.
int noalloc_setup(int dev, NoAllocDevice *out) {
    if (dev < 0 || dev >= 128) return PFSM_E_INVAL;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (g_noalloc_nsm[dev] == 0) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            nsm <= 0) {
            cudaGetLastError();
            return PFSM_E_CUDA;
        }
        g_noalloc_nsm[dev] = nsm;
    }
    out->scratch = static_cast<uint8_t *>(p);
    out->nsm = g_noalloc_nsm[dev];
    return PFSM_OK;
}
}  // namespace

// Encodes the caller's int16 table into the scan's uint16 form inside the
// scratch array and checks it (entries in range; the dead state absorbing
// and not final). A malformed table raises ERR_TABLE in the status.
__global__ void encode_dfa_noalloc(const int16_t *delta, int32_t Q, int32_t S, int32_t dead,
                                   const uint8_t *is_final, uint16_t *tab,
                                   unsigned long long *status) {
    const uint32_t total = static_cast<uint32_t>(Q) * S;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        const int t = delta[i];
        if (t < 0 || t >= Q) {
            atomicOr(&status[1], ERR_TABLE);
            tab[i] = DEAD16;
            continue;
        }
        if (dead >= 0 && static_cast<int>(i / S) == dead && t != dead)
            atomicOr(&status[1], ERR_TABLE);
        tab[i] = t == dead ? DEAD16 : static_cast<uint16_t>(t | (is_final[t] ? FINAL_BIT : 0));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && dead >= 0 && is_final[dead])
        atomicOr(&status[1], ERR_TABLE);
}

__global__ void noalloc_status_out(const unsigned long long *scratch_status,
                                   unsigned long long *status_out) {
    if (threadIdx.x < 2) {
        unsigned long long v = scratch_status[threadIdx.x];
        // a malformed table reports as a bad-argument error (bit 0)
        if (threadIdx.x == 1 && (v & ERR_TABLE)) v = (v & ~ERR_TABLE) | ERR_SYMBOL;
        status_out[threadIdx.x] = v;
    }
}

}  // namespace pfsm

using namespace pfsm;

extern "C" int pfsm_scan_dfa_noalloc(const int16_t *delta_dev, int32_t Q, int32_t S, int32_t q0,
                                     int32_t dead, const uint8_t *is_final_dev,
                                     const uint8_t *text_dev, uint64_t n, pfsm_match *out_dev,
                                     uint64_t cap, uint64_t *status_dev, void *stream) {
    if (Q < 1 || Q > 32767 || S < 1 || S > 256) return PFSM_E_INVAL;
    if (q0 < 0 || q0 >= Q || dead < -1 || dead >= Q || dead == q0) return PFSM_E_INVAL;
    if (static_cast<size_t>(Q) * S * 2 > kNoAllocTable) return PFSM_E_INVAL;   // above the limit
    if (!delta_dev || !is_final_dev || !status_dev) return PFSM_E_INVAL;
    if (n >= (1ull << 32) || (n > 0 && !text_dev) || (cap > 0 && !out_dev)) return PFSM_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PFSM_E_CUDA;
    NoAllocDevice dd;
    int st = noalloc_setup(dev, &dd);
    if (st) return st;
    const NoAllocDevice *d = &dd;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(d->scratch);
    uint32_t *carry_n = reinterpret_cast<uint32_t *>(d->scratch + 16);
    uint16_t *tab = reinterpret_cast<uint16_t *>(d->scratch + kNoAllocHeader);
    uint32_t *carry = reinterpret_cast<uint32_t *>(d->scratch + kNoAllocHeader + kNoAllocTable);
    // the array keeps the previous call's contents: clear the counters
    if (cudaMemsetAsync(d->scratch, 0, kNoAllocHeader, s) != cudaSuccess) return PFSM_E_CUDA;
    encode_dfa_noalloc<<<2 * d->nsm, 256, 0, s>>>(delta_dev, Q, S, dead, is_final_dev, tab, status);
    if (cudaGetLastError() != cudaSuccess) return PFSM_E_CUDA;
    if (n > 0) {
        ScanArgs a;
        memset(&a, 0, sizeof(a));
        a.text = text_dev;
        a.n = static_cast<uint32_t>(n);
        a.tile = 16384;
        a.halo = 2048;
        a.ntiles = static_cast<uint32_t>((n + a.tile - 1) / a.tile);
        a.text_buf = (a.tile + a.halo + 32 + 127) & ~127u;
        a.nbuf = 3;
        a.shift = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(text_dev) & 15);
        a.Q = Q;
        a.S = S;
        a.q0 = q0;
        a.k = 0;   // every instance steps from q0 (no start-prefix table)
        a.sbits = 8;
        a.dtab = tab;
        const uint32_t tab_bytes = ((static_cast<uint32_t>(Q) * S + 1) / 2) * 4;
        a.tab_smem = tab_bytes <= 48 * 1024;
        a.out = reinterpret_cast<uint32_t *>(out_dev);
        a.cap = cap;
        a.status = status;
        a.carry = carry;
        a.carry_n = carry_n;
        a.carry_cap = static_cast<uint32_t>(kNoAllocCarry / 16);
        a.stage_n = STAGE;
        const int threads = 512;
        SmemNeed need{0u, a.tab_smem ? tab_bytes : 0u, 0u, 0u, 0u, 0u};
        const uint32_t smem = layout_smem(a, 1, threads, need);
        if (smem > kSmemMax - kSmemStatic) return PFSM_E_INVAL;
        const int occ = max_ctas_per_sm(0, 0, threads, smem, a.tab_smem != 0);
        if (occ <= 0) return PFSM_E_CUDA;
        const int grid = static_cast<int>(
            std::min<uint64_t>(a.ntiles, static_cast<uint64_t>(d->nsm) * occ));
        if (launch_scan(a, 0, threads, grid, smem, s) != cudaSuccess) return PFSM_E_CUDA;
        if (launch_carry(a, 2 * d->nsm, s) != cudaSuccess) return PFSM_E_CUDA;
    }
    noalloc_status_out<<<1, 32, 0, s>>>(status, reinterpret_cast<unsigned long long *>(status_dev));
    if (cudaGetLastError() != cudaSuccess) return PFSM_E_CUDA;
    return PFSM_OK;
}
