// fsp_bound_resident.cu -- the couple-lanes bound with resident staging
// (sm_103a): every record group copied to shared memory once per block, warps
// independent.  The host side (layout, launch shape, depth order) is in
// fsp_bound_lanes.cu; this file holds the kernel and its launcher so that the
// library's translation units compile in parallel.
#include <cuda_runtime.h>

#include <mutex>

#include "fsp_internal.h"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

template <bool WIDE, int MP>
__global__ void __launch_bounds__(512, 1) fsp_lanes_resident(const LanesArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *ctr = reinterpret_cast<int *>(smem + 8);
    uint8_t *sgp = smem + 16;
    int2 *hcache = reinterpret_cast<int2 *>(smem + a.off_cache);
    int2 *tcache = hcache + a.m * 32;
    const unsigned char *tables = smem + a.off_tables;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem + a.off_flags) + (size_t)warp * flag_words(a.n);
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + a.off_aq) + (size_t)warp * 32 * a.aq_stride;

    // this block's share of the warp batches
    const int64_t b0 = (int64_t)blockIdx.x * a.num_batches / gridDim.x;
    const int64_t b1 = (int64_t)(blockIdx.x + 1) * a.num_batches / gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        *ctr = 0;
    }
    for (int i = threadIdx.x; i < a.G * 64; i += blockDim.x) sgp[i] = a.gpairs[i];
    load_sorted_heads(a, hcache, tcache);
    __syncthreads();
    const size_t group_bytes = (size_t)a.npad * 32 * a.rec_bytes;
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(group_bytes * a.G));
        for (int g = 0; g < a.G; ++g)
            bulk_g2s(smem + a.off_tables + g * group_bytes, a.grec + g * group_bytes, (uint32_t)group_bytes, bar);
    }
    bool ready = false;
    for (;;) {
        int claim = 0;
        if (lane == 0) claim = atomicAdd(ctr, 1);
        const int64_t bt = b0 + __shfl_sync(kFull, claim, 0);
        if (bt >= b1) break;
        const int64_t x = node_at(a, bt * 32 + lane);
        int bterm = 0;
        const bool valid = lanes_setup<MP>(a, x, lane, F, AQ + lane * a.aq_stride, bterm, hcache, tcache);
        if (!ready) {
            if (!mbar_wait_bounded(bar, 0, a.wait_limit)) {
                if (lane == 0) report_status(a.status, (int32_t)FSP_ETIMEDOUT);
                if (threadIdx.x == 0) mbar_wait_bounded(bar, 0, a.wait_limit);  // let the copy land
                return;
            }
            ready = true;
        }
        int lb[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) lb[b] = 0;
        for (int g = 0; g < a.G; ++g) {
            const int kk = sgp[2 * (g * 32 + lane)], ll = sgp[2 * (g * 32 + lane) + 1];
            if (!WIDE) {
                int u[32];
#pragma unroll
                for (int b = 0; b < 32; ++b) u[b] = 0;
                scan_compact(reinterpret_cast<const uint2 *>(tables + g * group_bytes) + lane, a.npad, F, u);
                couple_epilogue<WIDE>(AQ, a.aq_stride, a.m, kk, ll, u, lb);
            } else {
                int u[32];
#pragma unroll
                for (int b = 0; b < 32; ++b) u[b] = 0;
                scan_wide(reinterpret_cast<const int4 *>(tables + g * group_bytes) + lane, a.npad, F, u);
                couple_epilogue<WIDE>(AQ, a.aq_stride, a.m, kk, ll, u, lb);
            }
        }
        const int best = transpose_max(lb, lane);
        if (x < a.N) a.out[x] = valid ? max(best, bterm) : FSP_LB_INVALID;
        __syncwarp();  // the flag and row arrays are rewritten by the next batch
    }
    // the issuing thread never leaves while its copy may still be landing
    if (threadIdx.x == 0 && !ready) mbar_wait_bounded(bar, 0, a.wait_limit);
}

namespace {

template <bool WIDE, int MP>
cudaError_t launch_resident_variant(const LanesArgs &a, int grid, int threads, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] { attr_err = set_smem_attr(fsp_lanes_resident<WIDE, MP>); });
    if (attr_err != cudaSuccess) return attr_err;
    note_launches(1);
    fsp_lanes_resident<WIDE, MP><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_resident_w(const LanesArgs &a, int mp, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (mp) {
        case 8: return launch_resident_variant<WIDE, 8>(a, grid, threads, smem, s);
        case 12: return launch_resident_variant<WIDE, 12>(a, grid, threads, smem, s);
        case 16: return launch_resident_variant<WIDE, 16>(a, grid, threads, smem, s);
        case 20: return launch_resident_variant<WIDE, 20>(a, grid, threads, smem, s);
        case 24: return launch_resident_variant<WIDE, 24>(a, grid, threads, smem, s);
        default: return launch_resident_variant<WIDE, 32>(a, grid, threads, smem, s);
    }
}

}  // namespace

cudaError_t launch_resident_mp(const LanesArgs &a, bool wide, int mp, int grid, int threads, size_t smem,
                               cudaStream_t s) {
    return wide ? launch_resident_w<true>(a, mp, grid, threads, smem, s)
                : launch_resident_w<false>(a, mp, grid, threads, smem, s);
}

}  // namespace fspgb
