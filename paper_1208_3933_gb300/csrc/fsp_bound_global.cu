// fsp_bound_global.cu -- the couple-lanes bound with global staging (sm_103a).
//
// No shared-memory record tiles: every warp reads its couple groups' records
// from L2/L1 through the register ring of scan_compact_global and takes its
// own work items (a 32-node batch and a couple slice), so a small pool can
// spread one warp per item over the whole GPU.  The host side (layout,
// launch shape, depth order) is in fsp_bound_lanes.cu; this file holds the
// kernel and its launcher so that the library's translation units compile in
// parallel.
#include <cuda_runtime.h>

#include <mutex>

#include "fsp_internal.h"
#include "fsp_batch_scan.cuh"
#include "fsp_lanes_device.cuh"

namespace fspgb {

// No shared-memory tiles: every warp reads its couple groups' records from
// global memory (L2/L1) through the register ring of scan_compact_global, so
// the warps of a block never wait for each other and a pool too small to fill
// the GPU with block batches can give each work item a warp of its own.  Work
// item it = 32-node batch it / S, couple slice it % S (S = gslices, slices of
// gper groups); the grid's T warps take items w, w + T, w + 2T, ... in order.
template <int MP, int PS>
__global__ void __launch_bounds__(512, 1) fsp_lanes_global(const LanesArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem + a.off_flags) + (size_t)warp * flag_words(a.n);
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + a.off_aq) + (size_t)warp * 32 * a.aq_stride;
    const int64_t S = a.gslices > 1 ? a.gslices : 1;
    const int64_t items = a.num_batches * S;
    const int64_t T = (int64_t)gridDim.x * W;
    // kPtabByte: the block's shared-memory copy of the processing times
    void *ptab = PS == kPtabByte ? smem + a.off_ptab : nullptr;
    if constexpr (PS == kPtabByte) {
        load_ptab(a, ptab);
        __syncthreads();
    }
    for (int64_t it = (int64_t)blockIdx.x * W + warp; it < items; it += T) {
        const int64_t bt = it / S;
        const int sl = (int)(it - bt * S);
        const int64_t x = node_at(a, bt * 32 + lane);
        int bterm = 0;
        const bool valid = lanes_setup<MP, PS>(a, x, lane, F, AQ + lane * a.aq_stride, bterm, nullptr, nullptr, ptab);
        int lb[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) lb[b] = 0;
        const int g0 = S > 1 ? sl * a.gper : 0, g1 = S > 1 ? min(a.G, g0 + a.gper) : a.G;
        for (int g = g0; g < g1; ++g) {
            const int kk = __ldg(a.gpairs + 2 * (g * 32 + lane)), ll = __ldg(a.gpairs + 2 * (g * 32 + lane) + 1);
            int u[32];
#pragma unroll
            for (int b = 0; b < 32; ++b) u[b] = 0;
            const uint2 *R = reinterpret_cast<const uint2 *>(a.grec) + (size_t)g * a.npad * 32 + lane;
            scan_compact_global(R, a.npad, F, u);
            couple_epilogue<false>(AQ, a.aq_stride, a.m, kk, ll, u, lb);
        }
        const int best = transpose_max(lb, lane);
        if (x < a.N) {
            if (S == 1)
                a.out[x] = valid ? max(best, bterm) : FSP_LB_INVALID;
            else if (!valid)
                a.out[x] = FSP_LB_INVALID;  // every slice finds the row invalid
            else
                atomicMax(a.out + x, max(best, bterm));  // out was zeroed; bounds are >= 0
        }
        __syncwarp();  // the flag and row arrays are rewritten by the next item
    }
}
namespace {

template <int MP>
cudaError_t launch_global_variant(const LanesArgs &a, int grid, int threads, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = set_smem_attr(fsp_lanes_global<MP, kPtabNone>);
        if (attr_err == cudaSuccess) attr_err = set_smem_attr(fsp_lanes_global<MP, kPtabByte>);
    });
    if (attr_err != cudaSuccess) return attr_err;
    note_launches(1);
    if (a.off_ptab)
        fsp_lanes_global<MP, kPtabByte><<<grid, threads, smem, s>>>(a);
    else
        fsp_lanes_global<MP, kPtabNone><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_global_mp(const LanesArgs &a, int mp, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (mp) {
        case 8: return launch_global_variant<8>(a, grid, threads, smem, s);
        case 12: return launch_global_variant<12>(a, grid, threads, smem, s);
        case 16: return launch_global_variant<16>(a, grid, threads, smem, s);
        case 20: return launch_global_variant<20>(a, grid, threads, smem, s);
        case 24: return launch_global_variant<24>(a, grid, threads, smem, s);
        default: return launch_global_variant<32>(a, grid, threads, smem, s);
    }
}

}  // namespace fspgb
