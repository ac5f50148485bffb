// fsp_internal.h -- instance layout shared by the library's translation units.
//
// Device tables of one instance (Section II-D of Melab et al.; Table I gives
// their sizes and access counts).  Everything lives in one cudaMalloc block,
// each array 256-byte aligned so the bulk copies that stage them into shared
// memory start on a 16-byte boundary.
//
//   rec    [P][npad]      Johnson order of every couple with the per-entry
//                         constants of the bounding recurrence (see below);
//                         couples ordered by their second machine l, then k
//   pairs  [P][2]         uint8 (k,l) of each couple, in the same order (MM)
//   grec   [G][npad][32]  the same records regrouped for the couple-lanes
//                         kernel: couple c sits in group c/32, lane c%32;
//                         the slots past P are empty couples
//   gpairs [G*32][2]      (k,l) per group slot; empty slots read (0,1)
//   hsort  [m][n]         int2 (job, sum_{h<k} p_jh) sorted by the sum (RM)
//   tsort  [m][n]         int2 (job, sum_{h>k} p_jh) sorted by the sum (QM)
//   ptot   [m]            sum over all jobs of p_jk
//   pp     [n][mpad]      p with rows zero-padded to mpad (vector loads)
//   p      [n][m]         int32 processing times (PTM), job-major
//   head   [m][n]         int32 sum_{h<k} p_jh, machine-major (for RM)
//   tail   [m][n]         int32 sum_{h>l} p_jh, machine-major (for QM)
//   ptm    [m][n]         int32 p_jk, machine-major (column sums over U)
//
// One Johnson entry of couple c=(k,l) for job j carries
//   delta = p_jl - p_jk   and   s = lag_j + p_jl,   lag_j = sum_{k<h<l} p_jh,
// because the kernels run the pseudo-code's two-machine recurrence on the
// slack u = timeOnM2 - timeOnM1:  u <- max(u + delta, s)  for j in U.
//
// Compact 32-bit record (n <= 1024, 0 <= s < 8192, -256 <= delta < 256):
//   bits  0..9   j
//   bits 10..22  s
//   bits 23..31  delta (two's complement)
// The couple-lanes copy (grec) stores each compact record as two int32 words
// the scan uses directly: word 0 = 1024 s + j, word 1 = 1024 delta.  The scan
// keeps the slack scaled by 1024 with a job in its low 10 bits (a fraction
// below one unit) and runs one fused integer add-max per entry; with
// s < 2^13, |delta| <= 256 and n <= 1024 every scaled value stays below
// 2^29.  The no-op record (padding, empty couples) is (0, 0).
// Wide record: int4 {j, s, delta, 0}.
// Padding entries and empty couples are all-zero records: for any u >= 0,
// max(u + 0, 0) = u, so they never change the result, and an empty couple
// read as (0,1) contributes A_0 + q_1, which never exceeds couple (0,1)'s
// own value.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "fsp.h"

namespace fspgb {

// Lets a kernel take the device's opt-in maximum of dynamic shared memory
// (the current device; callers do this once per kernel and device).
template <typename K>
inline cudaError_t set_smem_attr(K kernel) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

constexpr int kThreads = 128;          // threads per bounding block
constexpr int kRecAlign = 4;           // couple rows padded to 4 entries (16 B compact)

struct DeviceTables {
    const void *rec = nullptr;
    const uint8_t *pairs = nullptr;
    const void *grec = nullptr;
    const uint8_t *gpairs = nullptr;
    const int32_t *hsort = nullptr;  // int2 pairs
    const int32_t *tsort = nullptr;  // int2 pairs
    const int32_t *ptot = nullptr;
    const int32_t *pp = nullptr;     // [n][mpad] p with zero-padded rows
    const int32_t *p = nullptr;
    const int32_t *head = nullptr;
    const int32_t *tail = nullptr;
    const int32_t *ptm = nullptr;
};

}  // namespace fspgb

struct fsp_instance {
    int32_t n = 0, m = 0, P = 0, npad = 0;
    int32_t G = 0;                  // couple groups of 32 (couple-lanes layout)
    int32_t mpad = 0;               // m rounded up to 8, 12, 16, 20, 24 or 32
    int32_t compact = 1;
    int32_t device = 0;
    int32_t rec_bytes = 4;          // bytes per Johnson record (lockstep layout)
    int32_t grec_bytes = 8;         // bytes per couple-lanes record
    uint32_t flags = 0;             // FSP_INSTANCE_* options of fsp_instance_create_ex
    std::vector<int32_t> p;         // host copy [n][m]
    std::vector<uint8_t> pairs;     // host copy [P][2]
    void *dev_block = nullptr;      // owns every device table
    size_t dev_bytes = 0;
    int32_t *host_status = nullptr; // pinned, mapped word: last device-side error (0 = none)
    int32_t *dev_status = nullptr;  // the same word as the device sees it
    fspgb::DeviceTables t;
    int32_t num_sms = 0;
    // fsp_bound_pool_host's copy and second compute stream and its events,
    // made on first use and kept; host_mu serialises that entry point's calls
    mutable std::mutex host_mu;
    mutable cudaStream_t host_streams[2] = {nullptr, nullptr};
    mutable cudaEvent_t host_events[10] = {};  // start, done, one per chunk (at most 8)
    mutable std::mutex mu;          // guards the tuning cache below
    mutable std::vector<std::pair<int64_t, fsp_launch_config>> tuned;  // pool-size bucket -> shape
};

namespace fspgb {

// Launch-shape resolution and the kernel launcher (fsp_bound.cu).
fsp_status resolve_config(const fsp_instance *inst, int64_t N, const fsp_launch_config *req,
                          fsp_launch_config *out, size_t *smem_bytes);
fsp_status launch_bound(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                        int64_t N, int32_t *out_lb, void *stream, const fsp_launch_config *cfg);
// Couple-lanes kernel (fsp_bound_lanes.cu).
fsp_status lanes_layout(const fsp_instance *inst, const fsp_launch_config &cfg, size_t *smem_bytes);
// Couple groups of 32 per streamed work item for a requested pairs_per_tile
// (0 or >= P: all G groups; else rounded up to whole groups).
int lanes_groups_per_item(const fsp_instance *inst, int pairs_per_tile);
// Nodes per warp of a couple-lanes shape (its nodes_per_thread field): 32 (0
// also means 32), 28 or 56 (one or two sets of 28); 0 for any other value.
int lanes_nodes_per_warp(const fsp_launch_config &c);
fsp_status launch_lanes(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *stream, const fsp_launch_config &cfg);
// The same bound as a prep kernel and a scan kernel (fsp_bound_split.cu).
fsp_status split_layout(const fsp_instance *inst, const fsp_launch_config &cfg, size_t *smem_bytes);
fsp_status launch_split(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *stream, const fsp_launch_config &cfg);
// The same bound with a record-tile pipeline per warp (fsp_bound_warp.cu).
fsp_status warp_layout(const fsp_instance *inst, const fsp_launch_config &cfg, size_t *smem_bytes);
fsp_status launch_warp(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                       int32_t *out_lb, void *stream, const fsp_launch_config &cfg);
// Depth order of a pool (fsp_order.cu): *order = a device permutation slot ->
// node, allocated from the scratch pool on stream s (free it with
// cudaFreeAsync on s after the launch that reads it), or null (identity) for
// pools below kDepthOrderMin nodes or instances below kDepthOrderMinJobs jobs.
constexpr int64_t kDepthOrderMin = 8192;
constexpr int kDepthOrderMinJobs = 64;
fsp_status depth_order(const fsp_instance *inst, const int32_t *depths, int64_t N, cudaStream_t s, int32_t **order);
// Per-device stream-ordered memory pool for launch scratch (keeps its memory).
fsp_status scratch_pool(int dev, cudaMemPool_t *out);
// Counts kernels the library enqueues (fsp_kernel_launches).
void note_launches(int k);
int max_smem_per_block(int device);
int max_smem_per_sm(int device);
int num_sms(int device);
fsp_status check_device(const fsp_instance *inst);
fsp_status take_device_status(const fsp_instance *inst);

}  // namespace fspgb
