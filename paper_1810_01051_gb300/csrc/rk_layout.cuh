// Shared-memory layout of the scan kernel, computed identically on host
// (launch size) and device (carving the dynamic shared memory).
#pragma once

#include <stdint.h>

namespace rk {

constexpr uint32_t kMaxTileBytes = 1u << 16;  // survivor positions are 16-bit
constexpr uint32_t kQueueCap = 288;           // queued survivor windows per warp (u16 positions)
constexpr uint32_t kMatchCap = 128;           // buffered match keys per warp
constexpr uint32_t kStagePad = 16;            // readable slack after each staged tile

struct SmemLayout {
    uint32_t filter_off, s2_off, bar_off, queue_off, mcount_off, match_off, stage_off;
    uint32_t stage_stride;
    uint32_t total;
};

__host__ __device__ constexpr uint32_t align_up(uint32_t x, uint32_t a) {
    return (x + a - 1) / a * a;
}

// s2_bytes: bytes of the survivor-stage tables copied into shared memory (0 =
// they stay in global memory).
__host__ __device__ inline SmemLayout smem_layout(uint32_t filter_bytes, uint32_t s2_bytes,
                                                  uint32_t warps, uint32_t stages,
                                                  uint32_t tile_bytes, uint32_t halo) {
    SmemLayout L{};
    uint32_t off = 0;
    L.filter_off = off;
    off = align_up(off + filter_bytes, 128);
    L.s2_off = off;
    off = align_up(off + s2_bytes, 128);
    L.bar_off = off;
    off = align_up(off + 2 * stages * 8, 16);
    L.queue_off = off;
    off = align_up(off + warps * kQueueCap * 2, 16);
    L.mcount_off = off;
    off = align_up(off + warps * 4, 16);
    L.match_off = off;
    off = align_up(off + warps * kMatchCap * 8, 128);
    L.stage_off = off;
    L.stage_stride = align_up(tile_bytes + halo + kStagePad, 128);
    off += stages * L.stage_stride;
    L.total = off;
    return L;
}

// Shared memory of the role-filter scan kernel (warp-specialised: stage-1
// warps, survivor warps, a producer warp).  Survivors pass from the stage-1
// warps to the survivor warps through a ring of 64-bit text positions.
constexpr uint32_t kRfRing = 1024;  // ring entries (a power of two)

constexpr uint32_t kRfXCap = 64;    // positions a survivor warp sets aside (see rk_scan_rf.cuh)

struct RfSmemLayout {
    uint32_t filter_off, s2_off, bar_off, ring_off, ctl_off, mcount_off, match_off, xbuf_off,
        stage_off;
    uint32_t stage_stride;
    uint32_t total;
};

__host__ __device__ inline RfSmemLayout rf_smem_layout(uint32_t filter_bytes, uint32_t s2_bytes,
                                                       uint32_t sv_warps, uint32_t stages,
                                                       uint32_t tile_bytes, uint32_t halo) {
    RfSmemLayout L{};
    uint32_t off = 0;
    L.filter_off = off;
    off = align_up(off + filter_bytes, 128);
    L.s2_off = off;
    off = align_up(off + s2_bytes, 128);
    L.bar_off = off;
    off = align_up(off + 2 * stages * 8, 16);
    L.ring_off = off;
    off = align_up(off + kRfRing * 8, 16);
    L.ctl_off = off;  // 16 bytes of counters, then 16 per ring (one per survivor warp)
    off = align_up(off + 16 + 16 * sv_warps, 16);
    L.mcount_off = off;
    off = align_up(off + sv_warps * 4, 16);
    L.match_off = off;
    off = align_up(off + sv_warps * kMatchCap * 8, 128);
    L.xbuf_off = off;  // per survivor warp: kRfXCap positions, then a count
    off = align_up(off + sv_warps * (kRfXCap * 8 + 16), 128);
    L.stage_off = off;
    L.stage_stride = align_up(tile_bytes + halo + kStagePad, 128);
    off += stages * L.stage_stride;
    L.total = off;
    return L;
}

}  // namespace rk
