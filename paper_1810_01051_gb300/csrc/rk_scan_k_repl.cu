// Scan kernel variants with the prefix bit set replicated into all 32
// shared-memory banks (and the sampled grams' set in the same layout).
#include "rk_scan_kernel.cuh"

namespace rk {
namespace scan {

cudaError_t launch_replicated(const ScanParams &p, uint32_t grid, uint32_t threads,
                              uint32_t smem, cudaStream_t st, bool q4, bool samp) {
    return q4 ? launch_one<kFilterReplicated, true>(p, grid, threads, smem, st, samp)
              : launch_one<kFilterReplicated, false>(p, grid, threads, smem, st, samp);
}

}  // namespace scan
}  // namespace rk
