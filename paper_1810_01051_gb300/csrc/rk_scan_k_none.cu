// Scan kernel variants without a stage-1 filter (every window hashed at
// every pattern length).
#include "rk_scan_kernel.cuh"

namespace rk {
namespace scan {

cudaError_t launch_none(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, bool q4) {
    return q4 ? launch_one<kFilterNone, true>(p, grid, threads, smem, st, false)
              : launch_one<kFilterNone, false>(p, grid, threads, smem, st, false);
}

}  // namespace scan
}  // namespace rk
