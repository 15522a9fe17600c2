// rk_search_device_noalloc: the device-buffer search for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: a host
// application whose own allocator has already reserved all of the device's
// memory (a foreign cudaMalloc then fails), or a latency-bound loop that must
// not pay for cudaMalloc/cudaFree, which can synchronise the device and take
// milliseconds.  This entry point runs the same scan and sort kernels as
// rk_search_device, but the sort's scratch space (ping-pong key buffer and
// digit histograms) is a fixed array in the library's own device memory,
// reserved when the library's device code is loaded on a GPU and held there
// until the process exits.  No call allocates.
#include <mutex>

#include "rk_internal.cuh"
#include "rk_sortws.cuh"

namespace {

// Scratch for an output of up to RK_NOALLOC_MAX_KEYS keys: the sort's
// workspace for that capacity (ping-pong key buffer, digit totals and
// look-back words).
constexpr uint64_t kNoAllocBytes = rk::sort_ws_bytes(RK_NOALLOC_MAX_KEYS);
static_assert(kNoAllocBytes == RK_NOALLOC_SCRATCH_BYTES, "rk.h states the scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a stand-in, so the
// address must come from the runtime.  The address kept here dies with the
// device's primary context (a device reset unloads the array); rk.h tells
// callers not to use this entry point after resetting a device.
int scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return RK_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RK_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RK_OK;
}

}  // namespace

extern "C" int rk_search_device_noalloc(const rk_table *t, const uint8_t *d_text, uint64_t n,
                                        uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                                        void *stream) {
    if (!t) return RK_EINVAL;
    if (capacity > RK_NOALLOC_MAX_KEYS) return RK_EINVAL;  // beyond the fixed scratch
    if (rk::sort_workspace_bytes(capacity) > kNoAllocBytes) return RK_EINVAL;
    int rc = rk::check_device(t);
    if (rc) return rc;
    void *scratch = nullptr;
    if ((rc = scratch_address(t->device, &scratch))) return rc;
    rc = rk_scan_device(t, d_text, n, d_keys, capacity, d_info, stream);
    if (rc) return rc;
    // The sort clears its counters, digit totals and look-back words itself
    // before using them, and writes every buffered key before reading it, so
    // leftovers from an earlier call do no harm.
    return rk::launch_sort(t, n, d_keys, capacity, d_info, scratch, kNoAllocBytes,
                           reinterpret_cast<cudaStream_t>(stream));
}
