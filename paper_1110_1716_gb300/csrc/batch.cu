// Batched scans: many texts, each with its own machine, in one launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pfsm_internal.h"

namespace pfsm {
void batch_free(pfsm_ctx *) {}
}  // namespace pfsm

extern "C" int pfsm_scan_batch(pfsm_ctx *ctx, const pfsm_job *jobs, int32_t k,
                               pfsm_bmatch *out_dev, uint64_t cap, uint64_t *counts,
                               uint64_t *total, void *stream) {
    (void)ctx; (void)jobs; (void)k; (void)out_dev; (void)cap; (void)counts; (void)total;
    (void)stream;
    return PFSM_E_INVAL;
}
