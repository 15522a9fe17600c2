// The paper's own GPU matcher (Section 3.1, GPU listing), kept as a measured
// comparison point: one pattern; one thread per text offset x <= n - m; the
// shift-add hash hy = (hy << 1) + T[x + i] recomputed over the whole window
// from global memory; a byte comparison when hy equals the pattern hash hx
// (computed once on the host and passed in); result[x] = 1 on a match.  The
// hash is kept in 64 bits (the paper does not state a width); it wraps for
// long patterns, which only adds hash collisions that the comparison removes.
#include "rk_internal.cuh"

namespace {

struct PaperParams {
    const uint8_t *text;
    uint64_t n;
    uint8_t *result;
    uint64_t hx;
    uint32_t m;
    uint8_t pattern[RK_MAX_PATTERN_LEN];
};

__global__ void rk_paper_kernel(const __grid_constant__ PaperParams P) {
    const uint64_t last = P.n - P.m;  // windows x = 0 .. n - m (the GPU listing's bound)
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x <= last;
         x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t hy = 0;
        for (uint32_t i = 0; i < P.m; ++i) hy = (hy << 1) + P.text[x + i];
        if (hy == P.hx) {
            uint32_t i = 0;
            while (i < P.m && P.text[x + i] == P.pattern[i]) ++i;
            if (i == P.m) P.result[x] = 1;
        }
    }
}

}  // namespace

extern "C" int rk_paper_search_device(const uint8_t *d_text, uint64_t n, const uint8_t *h_pattern,
                                      uint32_t m, uint8_t *d_result,
                                      uint32_t threads_per_block, void *stream) {
    if (m < 1 || m > RK_MAX_PATTERN_LEN || !h_pattern || n > RK_MAX_TEXT_LEN) return RK_EINVAL;
    if (threads_per_block == 0) threads_per_block = 1024;
    if (threads_per_block > 1024 || threads_per_block % 32) return RK_EINVAL;
    if (n == 0) return RK_OK;
    if (!d_text || !d_result) return RK_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_result, 0, n, st) != cudaSuccess) return RK_ECUDA;
    if (m > n) return RK_OK;
    PaperParams p;  // passed by value: the launch copies it
    p.text = d_text;
    p.n = n;
    p.result = d_result;
    p.m = m;
    p.hx = 0;
    for (uint32_t i = 0; i < m; ++i) {
        p.hx = (p.hx << 1) + h_pattern[i];  // the pattern hash, once, on the host
        p.pattern[i] = h_pattern[i];
    }
    const uint64_t windows = n - m + 1;
    const uint64_t blocks = std::min<uint64_t>((windows + threads_per_block - 1) / threads_per_block,
                                               1ull << 30);
    rk_paper_kernel<<<(uint32_t)blocks, threads_per_block, 0, st>>>(p);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}
