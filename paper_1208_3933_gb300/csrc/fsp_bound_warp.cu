// fsp_bound_warp.cu -- the couple-lanes bound with a record pipeline per
// warp (sm_103a).
//
// Same computation as fsp_bound_lanes.cu (one warp = 32 nodes, lanes = 32
// machine couples, slack scan over each couple's Johnson order), but no block
// barrier on the scan path: every warp streams the record tiles it needs
// through its own ring of kWarpBufs shared-memory buffers, each filled by one
// bulk copy (cp.async.bulk) completing on the buffer's mbarrier, and refilled
// by lane 0 as soon as the warp has read it.  The tile sequence is cyclic
// (group 0 chunk 0, ..., group G-1 last chunk, group 0 chunk 0, ...), so the
// first tiles of a warp's next 32 nodes are already in flight while it sets
// them up.  Warps of a block claim 32-node batches from a shared counter over
// the block's share of the pool; one warp's setup (latency bound: dependent
// loads and the prefix recurrence) therefore overlaps the other warps' scans
// instead of stalling them at a tile barrier.
//
// Shared memory: block part [counter | couple list (G x 32 x 2 bytes) | first
// 32 entries of every machine's head/tail-sorted list]; then per warp
// [kWarpBufs mbarriers | flag words F[n] | node rows 32 x stride | kWarpBufs
// record tiles].
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "fsp_internal.h"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

namespace {

constexpr int kWarpBufs = 3;  // record tiles in flight per warp

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <bool WIDE, int MP>
__global__ void __launch_bounds__(512, 1) fsp_lanes_warp(const LanesArgs a, uint32_t warp_stride, uint32_t w_off_aq,
                                                         uint32_t w_off_tiles) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *ctr = reinterpret_cast<int *>(smem);
    uint8_t *sgp = smem + 16;
    int2 *hcache = reinterpret_cast<int2 *>(smem + a.off_cache);
    int2 *tcache = hcache + a.m * 32;
    unsigned char *wr = smem + a.off_flags + (size_t)warp * warp_stride;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wr);
    uint32_t *F = reinterpret_cast<uint32_t *>(wr + 128);
    int32_t *AQ = reinterpret_cast<int32_t *>(wr + w_off_aq);
    unsigned char *tiles = wr + w_off_tiles;

    // this block's share of the 32-node batches
    const int64_t b0 = (int64_t)blockIdx.x * a.num_batches / gridDim.x;
    const int64_t b1 = (int64_t)(blockIdx.x + 1) * a.num_batches / gridDim.x;
    if (threadIdx.x == 0) *ctr = 0;
    if (lane == 0) {
        for (int i = 0; i < kWarpBufs; ++i) mbar_init(&bar[i], 1);
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < a.G * 64; i += blockDim.x) sgp[i] = a.gpairs[i];
    load_sorted_heads(a, hcache, tcache);
    __syncthreads();

    // the warp's tile ring: `issued` tiles requested, `consumed` read; tile k
    // of the sequence is tile k mod ntiles and lives in buffer k mod kWarpBufs
    uint32_t issued = 0, consumed = 0;
    auto issue = [&]() {  // lane 0
        const uint32_t bi = issued % kWarpBufs;
        const int t = (int)(issued % (uint32_t)a.ntiles);
        const int g = t / a.nchunks, ch = t - g * a.nchunks;
        const int pos = min(a.chunk, a.npad - ch * a.chunk);
        const unsigned char *src = a.grec + ((size_t)g * a.npad + (size_t)ch * a.chunk) * 32 * a.rec_bytes;
        const uint32_t bytes = (uint32_t)pos * 32u * a.rec_bytes;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[bi], bytes);
        bulk_g2s(tiles + (size_t)bi * a.tile_stride, src, bytes, &bar[bi]);
        ++issued;
    };

    int claim = 0;
    if (lane == 0) claim = atomicAdd(ctr, 1);
    int64_t bt = b0 + __shfl_sync(kFull, claim, 0);
    if (bt < b1 && lane == 0)
        for (int i = 0; i < kWarpBufs; ++i) issue();
    bool failed = false;
    while (bt < b1) {
        const int64_t x = node_at(a, bt * 32 + lane);
        int bterm = 0;
        const bool valid = lanes_setup<MP>(a, x, lane, F, AQ + lane * a.aq_stride, bterm, hcache, tcache);
        int lb[32];
        int uf[32];
        int ui[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) {
            lb[b] = 0;
            uf[b] = 0;
            ui[b] = 0;
        }
        int kk = 0, ll = 1;
        for (int t = 0; t < a.ntiles; ++t) {
            const uint32_t bi = consumed % kWarpBufs;
            const bool ok = mbar_wait_bounded(&bar[bi], (consumed / kWarpBufs) & 1u, a.wait_limit);
            if (!__all_sync(kFull, ok)) {
                failed = true;
                break;
            }
            const unsigned char *tb = tiles + (size_t)bi * a.tile_stride;
            const int g = t / a.nchunks, ch = t - g * a.nchunks;
            if (ch == 0) {
#pragma unroll
                for (int b = 0; b < 32; ++b) {
                    uf[b] = 0;
                    ui[b] = 0;
                }
                kk = sgp[2 * (g * 32 + lane)];
                ll = sgp[2 * (g * 32 + lane) + 1];
            }
            const int npos = min(a.chunk, a.npad - ch * a.chunk);
            if (!WIDE)
                scan_compact(reinterpret_cast<const uint2 *>(tb) + lane, npos, F, uf);
            else
                scan_wide(reinterpret_cast<const int4 *>(tb) + lane, npos, F, ui);
            if (ch == a.nchunks - 1) {
                if (!WIDE)
                    couple_epilogue<WIDE>(AQ, a.aq_stride, a.m, kk, ll, uf, lb);
                else
                    couple_epilogue<WIDE>(AQ, a.aq_stride, a.m, kk, ll, ui, lb);
            }
            ++consumed;
            __syncwarp();  // every lane is done with buffer bi
            if (lane == 0) issue();
        }
        if (failed) break;
        const int best = transpose_max(lb, lane);
        if (x < a.N) a.out[x] = valid ? max(best, bterm) : FSP_LB_INVALID;
        __syncwarp();  // the flag and row arrays are rewritten by the next batch
        if (lane == 0) claim = atomicAdd(ctr, 1);
        bt = b0 + __shfl_sync(kFull, claim, 0);
    }
    // copies still in flight land before the warp leaves (bounded)
    if (lane == 0) {
        if (failed) report_status(a.status, (int32_t)FSP_ETIMEDOUT);
        for (; consumed < issued; ++consumed)
            mbar_wait_bounded(&bar[consumed % kWarpBufs], (consumed / kWarpBufs) & 1u, a.wait_limit);
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ints per node row: A_k as int32, then q_l as int16 (compact records) or int32
int aq_stride_for(int m, bool q32) { return (m + (q32 ? m : (m + 1) / 2)) | 1; }

struct WarpLayout {
    uint32_t off_cache, off_warps, warp_stride, w_off_aq, w_off_tiles, tile_stride;
    size_t total;
};

WarpLayout warp_layout_for(const fsp_instance *inst, int warps, int chunk) {
    WarpLayout L;
    L.off_cache = (uint32_t)align_up(16 + (size_t)inst->G * 64, 128);
    L.off_warps = (uint32_t)align_up(L.off_cache + (size_t)inst->m * 32 * 8 * 2, 128);
    L.tile_stride = (uint32_t)align_up((size_t)chunk * 32 * inst->grec_bytes, 128);
    L.w_off_aq = (uint32_t)align_up(128 + (size_t)flag_words(inst->n) * 4, 128);
    L.w_off_tiles = (uint32_t)align_up(L.w_off_aq + (size_t)32 * aq_stride_for(inst->m, !inst->compact) * 4, 128);
    L.warp_stride = (uint32_t)align_up(L.w_off_tiles + (size_t)kWarpBufs * L.tile_stride, 128);
    L.total = (size_t)L.off_warps + (size_t)warps * L.warp_stride;
    return L;
}

template <bool WIDE, int MP>
cudaError_t launch_warp_variant(const LanesArgs &a, const WarpLayout &L, int grid, int threads, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] { attr_err = set_smem_attr(fsp_lanes_warp<WIDE, MP>); });
    if (attr_err != cudaSuccess) return attr_err;
    fsp_lanes_warp<WIDE, MP><<<grid, threads, L.total, s>>>(a, L.warp_stride, L.w_off_aq, L.w_off_tiles);
    note_launches(1);
    return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_warp_mp(int mp, const LanesArgs &a, const WarpLayout &L, int grid, int threads, cudaStream_t s) {
    switch (mp) {
        case 8: return launch_warp_variant<WIDE, 8>(a, L, grid, threads, s);
        case 12: return launch_warp_variant<WIDE, 12>(a, L, grid, threads, s);
        case 16: return launch_warp_variant<WIDE, 16>(a, L, grid, threads, s);
        case 20: return launch_warp_variant<WIDE, 20>(a, L, grid, threads, s);
        case 24: return launch_warp_variant<WIDE, 24>(a, L, grid, threads, s);
        default: return launch_warp_variant<WIDE, 32>(a, L, grid, threads, s);
    }
}

}  // namespace

fsp_status warp_layout(const fsp_instance *inst, const fsp_launch_config &c, size_t *smem_bytes) {
    const int W = c.warps_per_block;
    const int bps = c.blocks_per_sm ? c.blocks_per_sm : 1;
    if (W < 1 || W > 16 || bps < 1 || bps > 2 || W * bps > 16) return FSP_EINVAL;
    if (c.positions_per_tile < 4 || (c.positions_per_tile & 3)) return FSP_EINVAL;
    const WarpLayout L = warp_layout_for(inst, W, std::min(c.positions_per_tile, inst->npad));
    const size_t budget = bps == 1 ? (size_t)max_smem_per_block(inst->device)
                                   : std::min((size_t)max_smem_per_block(inst->device),
                                              (size_t)max_smem_per_sm(inst->device) / 2 - 1024);
    if (L.total > budget) return FSP_EINVAL;
    *smem_bytes = L.total;
    return FSP_OK;
}

fsp_status launch_warp(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                       int32_t *out_lb, void *stream, const fsp_launch_config &cfg) {
    size_t smem = 0;
    fsp_status st = warp_layout(inst, cfg, &smem);
    if (st != FSP_OK) return st;
    if (N <= 0) return FSP_OK;
    const int W = cfg.warps_per_block;
    const int bps = cfg.blocks_per_sm ? cfg.blocks_per_sm : 1;
    const int chunk = std::min(cfg.positions_per_tile, inst->npad);
    const WarpLayout L = warp_layout_for(inst, W, chunk);
    LanesArgs a = {};
    a.grec = static_cast<const unsigned char *>(inst->t.grec);
    a.gpairs = inst->t.gpairs;
    a.hsort = reinterpret_cast<const int2 *>(inst->t.hsort);
    a.tsort = reinterpret_cast<const int2 *>(inst->t.tsort);
    a.ptot = inst->t.ptot;
    a.pp = inst->t.pp;
    a.nodes = nodes;
    a.depths = depths;
    a.out = out_lb;
    a.status = inst->dev_status;
    a.N = N;
    a.num_batches = (N + 31) / 32;
    a.n = inst->n;
    a.m = inst->m;
    a.G = inst->G;
    a.npad = inst->npad;
    a.mpad = inst->mpad;
    a.chunk = chunk;
    a.nchunks = (inst->npad + chunk - 1) / chunk;
    a.ntiles = inst->G * a.nchunks;
    a.rec_bytes = (uint32_t)inst->grec_bytes;
    a.off_cache = L.off_cache;
    a.off_flags = L.off_warps;
    a.tile_stride = L.tile_stride;
    a.aq_stride = aq_stride_for(inst->m, !inst->compact);
    a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
    a.q32 = inst->compact ? 0 : 1;
    a.wait_limit = 4000000000LL;
    // whole blocks' worth of warps per SM; at least one batch per warp of the grid
    const int64_t per_block = W;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((a.num_batches + per_block - 1) / per_block, (int64_t)num_sms(inst->device) * bps));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *order = nullptr;
    st = depth_order(inst, depths, N, s, &order);
    if (st != FSP_OK) return st;
    a.order = order;
    const cudaError_t e = inst->compact ? launch_warp_mp<false>(inst->mpad, a, L, grid, 32 * W, s)
                                        : launch_warp_mp<true>(inst->mpad, a, L, grid, 32 * W, s);
    const cudaError_t ef = order ? cudaFreeAsync(order, s) : cudaSuccess;
    return (e == cudaSuccess && ef == cudaSuccess) ? FSP_OK : FSP_ECUDA;
}

}  // namespace fspgb
