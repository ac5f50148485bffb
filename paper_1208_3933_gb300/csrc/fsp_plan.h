// fsp_plan.h -- host-visible argument blocks of the couple-lanes kernels and
// the batch-plan interface shared by fsp_batch.cu and fsp_server.cpp.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>
#include <vector>

#include "fsp_internal.h"

namespace fspgb {

// Shared-memory words of one warp's flag array: one per job, rounded up to
// whole 32-word blocks (the setup's membership bitmaps use them all).
__host__ __device__ inline int flag_words(int n) { return (n + 31) & ~31; }

// Arguments of one pool for the couple-lanes kernels (one per launch for the
// single-pool kernels, one per pool in a batch plan).
struct LanesArgs {
    const unsigned char *grec;
    const uint8_t *gpairs;
    const int2 *hsort, *tsort;
    const int32_t *ptot;
    const int32_t *pp;    // [n][mpad] processing times, rows padded with zeros
    const int16_t *nodes;
    const int32_t *depths;
    int32_t *out;
    int32_t *status;
    int64_t N;
    int64_t num_batches;  // streamed: block batches of 32 * warps nodes; resident: warp batches of 32
    int32_t n, m, G, npad;
    int32_t mpad;         // row stride of pp (<= the kernel's MP)
    int32_t chunk;        // streamed: Johnson positions per tile (multiple of 4)
    int32_t nchunks;      // streamed: tiles per couple group
    int32_t ntiles;       // streamed: G * nchunks
    uint32_t rec_bytes;
    uint32_t off_tables;  // records (resident: all groups; streamed: two tile buffers)
    uint32_t tile_stride;
    uint32_t off_flags, off_aq;  // split scan: off_flags = the prepared-state region
    uint32_t off_cache;   // first 32 entries of each machine's head/tail-sorted list (0 = none)
    uint32_t off_ptab;    // shared-memory copy of pp as bytes, [n][mpad] uint8 (0 = none: read pp from global)
    const int32_t *order; // slot -> node (depth order), or null: slot i bounds node i
    uint32_t *scratch;    // split kernels: prepared state, [32-node batch][sb_words]
    int32_t sb_words;
    int32_t aq_stride;    // ints per node row (odd): A as int32 [m], then q as int16 [m] (int32 if q32)
    int32_t q32;          // q stored as int32: instances with 128-bit records, whose tails may pass 2^15
    int32_t release;      // 0: release times from the head minima; 1: per-job earliest starts
    int32_t gper;         // streamed: couple groups per work item (slices of a block batch)
    int32_t gslices;      // streamed: work items per sliced block batch, ceil(G / gper); 0 or 1 = no split
    int64_t full_batches; // streamed, gslices > 1: block batches [0, full_batches) are whole work items
    long long wait_limit;
};

// A batch plan's launch parameters.
struct PlanParams {
    int64_t nitems = 0, nodes = 0;
    int mp = 8, n_max = 1, stride = 1, warps = 16, grid = 1;
    int couples_per_item = 0;  // 0: every couple of a node batch in one work item
    uint32_t off_aq = 0;
    size_t smem = 0;
    // bounds of pools split by couples: zeroed before the kernel, whose
    // slices then meet in an atomic max
    std::vector<std::pair<int32_t *, int64_t>> zero;
};

// Builds a batch plan on the host: per-pool arguments and the work items,
// ordered longest first (fsp_batch.cu).  A work item is a 32-node batch of a
// pool and, with couples_per_item > 0, a slice of ceil(couples_per_item / 32)
// of its instance's couple groups.
fsp_status build_plan(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block, int32_t couples_per_item,
                      int device, std::vector<LanesArgs> &args, std::vector<int2> &items, PlanParams &pp);
// Launchers of the couple-lanes kernels that live in translation units of
// their own (mp = the kernel's padded machine count 8, 12, 16, 20, 24 or 32):
// streamed staging with ns sets of 28 nodes per warp (fsp_bound_streamed28.cu)
// and global staging (fsp_bound_global.cu, a.off_ptab != 0: the processing
// times in shared memory).
cudaError_t launch_streamed28_mp(const LanesArgs &a, int mp, int ns, int grid, int threads, size_t smem,
                                 cudaStream_t s);
cudaError_t launch_global_mp(const LanesArgs &a, int mp, int grid, int threads, size_t smem, cudaStream_t s);
// resident staging (fsp_bound_resident.cu), wide: 128-bit records
cudaError_t launch_resident_mp(const LanesArgs &a, bool wide, int mp, int grid, int threads, size_t smem,
                               cudaStream_t s);

// Enqueues a plan already copied to the device: counter reset + kernel.
fsp_status launch_plan(const LanesArgs *d_args, const int2 *d_items, int32_t *d_counter, const PlanParams &pp,
                       cudaStream_t s);

}  // namespace fspgb
