// The role-filter scan kernel's variants: its kind (step 2, step 4, step 4
// with a side set), survivors verified in the scan or listed for the
// verification kernel.
#include "rk_scan_rf.cuh"

namespace rk {
namespace scan {

cudaError_t launch_role(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, uint32_t step, bool side) {
    const bool defer = p.cand.list != nullptr;
    if (step == 2)
        return defer ? launch_rf_d<2, true>(p, grid, threads, smem, st)
                     : launch_rf_d<2, false>(p, grid, threads, smem, st);
    if (side)
        return defer ? launch_rf_d<6, true>(p, grid, threads, smem, st)
                     : launch_rf_d<6, false>(p, grid, threads, smem, st);
    return defer ? launch_rf_d<4, true>(p, grid, threads, smem, st)
                 : launch_rf_d<4, false>(p, grid, threads, smem, st);
}

}  // namespace scan
}  // namespace rk
