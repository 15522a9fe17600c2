// Scan kernel variants with one flat prefix bit set (and the sampled
// grams' set in the same layout).
#include "rk_scan_kernel.cuh"

namespace rk {
namespace scan {

cudaError_t launch_flat(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, bool q4, bool samp) {
    return q4 ? launch_one<kFilterFlat, true>(p, grid, threads, smem, st, samp)
              : launch_one<kFilterFlat, false>(p, grid, threads, smem, st, samp);
}

}  // namespace scan
}  // namespace rk
