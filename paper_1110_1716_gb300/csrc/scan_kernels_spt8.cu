// The single-text scan kernel instantiated for 8 starts per thread per
// filter round (short texts), compiled apart from the 32-start kernels.
#include "scan_tiles.cuh"

namespace pfsm {

cudaError_t launch_scan_spt8(const ScanArgs &a, int kind, int threads, int grid, uint32_t smem,
                             cudaStream_t s) {
    return launch_scan_spt<8>(a, kind, threads, grid, smem, s);
}

int max_ctas_per_sm_spt8(int kind, int sbits, int threads, uint32_t smem, bool tab_smem) {
    return occupancy_spt<8>(kind, sbits, threads, smem, tab_smem);
}

}  // namespace pfsm
