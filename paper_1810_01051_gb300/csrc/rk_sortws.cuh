// Workspace layout of the match-key sort, shared by the sort and by the
// entry point that keeps its scratch in a fixed device array.
#pragma once

#include <stdint.h>

namespace rk {

constexpr uint32_t kSortTile = 2048;      // keys per tile of a sort pass
constexpr uint32_t kMaxSortPasses = 8;    // 8-bit digits: 5 offset + 3 id digits at most

struct SortWsLayout {
    uint64_t tmp_off;     // ping-pong key buffer, capacity x 8 bytes
    uint64_t ctrl_off;    // per pass: tile counter
    uint64_t ghist_off;   // per pass: 256 digit totals
    uint64_t status_off;  // per pass: one look-back word per (tile, digit)
    uint64_t tiles;       // tiles of a full output
    uint64_t total;
};

__host__ __device__ constexpr uint64_t ws_align(uint64_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ constexpr SortWsLayout sort_ws_layout(uint64_t capacity) {
    const uint64_t tiles = (capacity + kSortTile - 1) / kSortTile;
    const uint64_t tmp = ws_align(capacity * 8);
    const uint64_t ctrl = 256;
    const uint64_t ghist = ws_align((uint64_t)kMaxSortPasses * 256 * 4);
    const uint64_t status = (uint64_t)kMaxSortPasses * tiles * 256 * 8;
    return SortWsLayout{0, tmp, tmp + ctrl, tmp + ctrl + ghist, tiles,
                        tmp + ctrl + ghist + status + 256};
}

__host__ __device__ constexpr uint64_t sort_ws_bytes(uint64_t capacity) {
    return sort_ws_layout(capacity).total;
}

// Workspace of a scan of n text bytes whose survivors are verified in a
// second pass: a candidate count and a list of up to n / 64 + 4096
// candidates (16 bytes each; a scan offered more probes the rest itself).
struct ScanWsLayout {
    uint64_t count_off;  // unsigned long long: candidates offered
    uint64_t list_off;   // 16-byte entries [cap]
    uint64_t cap;
    uint64_t total;
};

__host__ __device__ constexpr ScanWsLayout scan_ws_layout(uint64_t n) {
    return ScanWsLayout{0, 256, n / 64 + 4096, 256 + ws_align((n / 64 + 4096) * 16)};
}

}  // namespace rk
