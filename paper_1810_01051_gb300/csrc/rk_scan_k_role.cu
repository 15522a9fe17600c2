// Scan kernel variants with a role filter: stage 1 looks up every 2nd or
// 4th position's 4-byte gram (DevTable::rf_step), in scans that verify
// their survivors themselves or list them for the verification kernel.
#include "rk_scan_kernel.cuh"

namespace rk {
namespace scan {

cudaError_t launch_role(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, uint32_t step) {
    const bool defer = p.cand.list != nullptr;
    if (step == 2)
        return defer ? launch_d<kFilterFlat, true, true, 2>(p, grid, threads, smem, st)
                     : launch_d<kFilterFlat, true, false, 2>(p, grid, threads, smem, st);
    return defer ? launch_d<kFilterFlat, true, true, 4>(p, grid, threads, smem, st)
                 : launch_d<kFilterFlat, true, false, 4>(p, grid, threads, smem, st);
}

}  // namespace scan
}  // namespace rk
