// fsp_batch_scan.cuh -- the couple-lanes scan of the batched kernels
// (fsp_batch.cu, fsp_noalloc.cu), whose warps read their instance's records
// from global memory (L1/L2) rather than from a shared-memory tile.
#pragma once

#include "fsp_lanes_device.cuh"

namespace fspgb {

// scan_compact over records read from global memory (L1/L2): the records
// of the next kScanAhead positions are loaded while the current ones are
// applied, so each load's latency (longer than a shared-memory read's) is
// covered by the updates before it is needed.  npos (a couple row's padded
// length) is a multiple of kScanAhead, so every round applies all of them.
constexpr int kScanAhead = 4;
static_assert(kScanAhead == kRecAlign, "a round of the ring covers one padding unit of a couple row");
__device__ __forceinline__ void scan_compact_global(const uint2 *R, int npos, const uint32_t *F, int (&u)[32]) {
    uint2 buf[kScanAhead];
#pragma unroll
    for (int t = 0; t < kScanAhead; ++t) buf[t] = t < npos ? __ldg(R + t * 32) : make_uint2(0u, 0u);
    for (int i = 0; i < npos; i += kScanAhead) {
#pragma unroll
        for (int t = 0; t < kScanAhead; ++t) {
            const uint2 r = buf[t];
            const int nx = i + kScanAhead + t;
            buf[t] = nx < npos ? __ldg(R + nx * 32) : make_uint2(0u, 0u);
            lanes_step(r, F, u);
        }
    }
}

}  // namespace fspgb
