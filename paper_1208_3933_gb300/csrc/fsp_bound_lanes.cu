// fsp_bound_lanes.cu -- the couple-lanes bounding kernels (sm_103a).
//
// Same operator as fsp_bound.cu (Section III-A: one evaluation of the
// two-machine bound of Section II-C per sub-problem), mapped the other way
// round: a warp owns 32 nodes, and its 32 lanes take 32 different machine
// couples (k,l).  Each lane walks its couple's Johnson order (records laid
// out [group][position][lane], so the 32 lanes read 32 consecutive records)
// and updates the slack of all 32 nodes of the warp in registers,
//     u_b <- max(u_b + delta_j, s_j)   when job j is unscheduled in node b,
// where bit b of the warp's flag word for job j says so.  A lane's couple
// value for node b is A_k + q_l + u_b (the slack form, see fsp_bound.cu); a
// transpose-max over the 32 lanes (31 shuffles) then gives lane b the maximum
// over all couples for node b, combined with the one-machine terms
// max_l (A_l + q_l).
//
// With compact records (two int32 words: 1024 s + j and 1024 delta) the scan
// keeps every slack scaled by 1024 with a job in its low bits and runs one
// fused integer add-max per entry (fsp_lanes_device.cuh); the epilogue's
// shift by 10 gives the exact integer slack.  128-bit records (large
// processing times) use the plain int32 path.
//
// Per node the shared memory holds one flag bit per job and a row with A_k
// (int32) and q_l (int16 with compact records, whose tails stay below 2^15;
// int32 with 128-bit ones), so a block keeps hundreds of nodes in flight.
// Large pools are bounded in depth order (fsp_order.cu).  The streamed kernel
// and the host side of all the couple-lanes modes are here; the kernels of
// the other modes are in files of their own:
//   resident  all record groups are copied to shared memory once per block
//             (one cp.async.bulk per group on one mbarrier); warps are then
//             independent and claim 32-node batches from a per-block counter,
//             so one warp's setup overlaps the others' scans
//             (fsp_bound_resident.cu);
//   streamed  records too large for shared memory are staged in tiles of
//             (group, positions) through two buffers, the whole block moving
//             from tile to tile together (the paper's "does not fit" case).
//             A pool too small to occupy every SM splits each block batch by
//             couple groups over several work items, whose couple maxima meet
//             in an atomic max on the zeroed bounds.  A variant holds one or
//             two sets of 28 nodes per warp instead of 32
//             (fsp_bound_streamed28.cu);
//   global    no tiles: every warp reads its groups' records from L2/L1
//             through a register ring and takes its own work items, so a
//             small pool spreads one warp per item over the GPU
//             (fsp_bound_global.cu);
//   split     and warp staging: fsp_bound_split.cu, fsp_bound_warp.cu.
// Global, one-set streamed and split staging (its prep kernel) keep the
// processing times in shared memory, one byte each, when they fit.
//
// Setup, one lane per node (fsp_lanes_device.cuh): (1) one pass over the
// prefix for the membership bitmaps, row validation, the prefix recurrence
// C(sigma,k) (Section II-B) and the prefix's column sums, (2) the flag words
// by bit-matrix transposes, (3) the minima of RM and QM as the first
// unscheduled job of each machine's head- (tail-) sorted job list, 32 list
// entries per round, or, for nodes with at most 32 unscheduled jobs, by
// walking those jobs.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "fsp_internal.h"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

// ---------------------------------------------------------------- streamed
// PS: the block holds a shared-memory copy of the processing times as bytes
// (a.off_ptab), which the setup reads instead of global memory.
template <bool WIDE, int MP, bool PS>
__global__ void __launch_bounds__(512, 1) fsp_lanes_streamed(const LanesArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint8_t *sgp = smem + 16;
    int2 *hcache = reinterpret_cast<int2 *>(smem + a.off_cache);
    int2 *tcache = hcache + a.m * 32;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem + a.off_flags) + (size_t)warp * flag_words(a.n);
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + a.off_aq) + (size_t)warp * 32 * a.aq_stride;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < a.G * 64; i += blockDim.x) sgp[i] = a.gpairs[i];
    load_sorted_heads(a, hcache, tcache);
    void *ptab = PS ? smem + a.off_ptab : nullptr;
    if constexpr (PS) load_ptab(a, ptab);
    __syncthreads();

    TilePipe tp{bar, smem + a.off_tables, a.tile_stride, a.ntiles <= 2};
    auto tile_issue = [&](uint32_t fill, int t) {
        const int g = t / a.nchunks, ch = t - g * a.nchunks;
        const int pos = min(a.chunk, a.npad - ch * a.chunk);
        const unsigned char *src = a.grec + ((size_t)g * a.npad + (size_t)ch * a.chunk) * 32 * a.rec_bytes;
        tp.issue(fill, src, (uint32_t)pos * 32u * a.rec_bytes);
    };
    // Work items: block batches of 32 W nodes, the first `full` of them whole
    // (all couple groups), each later one split into S slices of gper couple
    // groups.  S = 1 unless a small pool is split by couples throughout
    // (full = 0) to occupy more SMs, or the batches of the last partial wave
    // are (full = the batches before it).  Sliced item it = batch full +
    // (it - full) / S, slice (it - full) % S; the host keeps the sliced item
    // count below 2^31.
    const uint32_t S = a.gslices > 1 ? (uint32_t)a.gslices : 1u;
    const int64_t full = S > 1 ? a.full_batches : a.num_batches;
    const int gper = S > 1 ? a.gper : a.G;
    const int64_t items = full + (a.num_batches - full) * S;
    auto slice_of = [&](int64_t it) { return it < full ? -1 : (int)((uint32_t)(it - full) % S); };
    auto first_tile = [&](int sl) { return sl < 0 ? 0 : sl * gper * a.nchunks; };
    if (threadIdx.x == 0 && (int64_t)blockIdx.x < items) {
        if (tp.resident) {
            tile_issue(0, 0);
            if (a.ntiles == 2) tile_issue(1, 1);
        } else {
            tile_issue(0, first_tile(slice_of(blockIdx.x)));
        }
    }

    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int sl = slice_of(it);
        const int64_t bt = sl < 0 ? it : full + (int64_t)((uint32_t)(it - full) / S);
        const int64_t x = node_at(a, bt * (int64_t)(32 * W) + warp * 32 + lane);
        int bterm = 0;
        const bool valid = lanes_setup<MP, PS ? kPtabByte : kPtabNone>(a, x, lane, F, AQ + lane * a.aq_stride, bterm,
                                                                       hcache, tcache, ptab);
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
        const int t1 = sl < 0 ? a.ntiles : min(a.G, (sl + 1) * gper) * a.nchunks;
        for (int t = first_tile(sl); t < t1; ++t) {
            const int g = t / a.nchunks, ch = t - g * a.nchunks;
            if (!tp.resident && threadIdx.x == 0) {
                // the next tile of this item, else the first of the block's next item
                const int next = t + 1 < t1 ? t + 1
                                 : (it + gridDim.x < items ? first_tile(slice_of(it + gridDim.x)) : -1);
                if (next >= 0) tile_issue(tp.fill + 1, next);
            }
            if (!tp.wait(t, a.wait_limit)) {
                if (threadIdx.x == 0) {
                    report_status(a.status, (int32_t)FSP_ETIMEDOUT);
                    tp.drain(a.wait_limit);
                }
                return;
            }
            const unsigned char *tb = tp.buf + tp.current(t) * tp.stride;
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
            if (!tp.resident) {
                __syncthreads();
                ++tp.fill;
            }
        }
        const int best = transpose_max(lb, lane);
        if (x < a.N) {
            if (sl < 0)
                a.out[x] = valid ? max(best, bterm) : FSP_LB_INVALID;
            else if (!valid)
                a.out[x] = FSP_LB_INVALID;  // every slice finds the row invalid
            else
                atomicMax(a.out + x, max(best, bterm));  // out was zeroed; bounds are >= 0
        }
        __syncwarp();  // the flag and row arrays are rewritten by the next batch
    }
}

// ---------------------------------------------------------------- host side
namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct LanesLayout {
    uint32_t off_cache, off_tables, tile_stride, off_flags, off_aq;
    uint32_t off_ptab;  // shared-memory copy of the processing times (0 = none)
    int32_t aq_stride;
    size_t total;
};

// Global and one-set streamed staging copy the processing-time rows (pp,
// [n][mpad], as bytes) to shared memory when they fit the block's budget beside
// everything else (at most 64 KB): the setup's prefix recurrence, walks and
// release times then read a row in one shared-memory latency instead of an
// L1 miss.  One byte per entry (compact instances: every p < 256).
constexpr size_t kPtabMaxBytes = 64 * 1024;
void add_ptab(LanesLayout &L, const fsp_instance *inst, size_t budget) {
    const size_t bytes = (size_t)inst->n * inst->mpad;
    const size_t off = align_up(L.total, 128);
    L.off_ptab = 0;
    if (bytes <= kPtabMaxBytes && off + bytes <= budget) {
        L.off_ptab = (uint32_t)off;
        L.total = align_up(off + bytes, 128);
    }
}

// ints per node row: A_k as int32, then q_l as int16 (compact records) or int32
int aq_stride_for(int m, bool q32) { return (m + (q32 ? m : (m + 1) / 2)) | 1; }

// npw: nodes per warp (32; or 28 and 56, one and two sets of 28, streamed only)
LanesLayout lanes_layout_for(const fsp_instance *inst, int warps, bool resident, int chunk, size_t budget,
                             int npw = 32) {
    const int sets = npw == 56 ? 2 : 1;
    LanesLayout L = {};
    L.off_cache = (uint32_t)align_up(16 + (size_t)inst->G * 64, 128);
    L.off_tables = (uint32_t)align_up(L.off_cache + (size_t)inst->m * 32 * 8 * 2, 128);
    const size_t group_bytes = (size_t)inst->npad * 32 * inst->grec_bytes;
    if (resident) {
        L.tile_stride = (uint32_t)group_bytes;
        L.off_flags = (uint32_t)align_up(L.off_tables + group_bytes * inst->G, 128);
    } else {
        L.tile_stride = (uint32_t)align_up((size_t)chunk * 32 * inst->grec_bytes, 128);
        L.off_flags = L.off_tables + 2 * L.tile_stride;
    }
    L.off_aq = (uint32_t)align_up(L.off_flags + (size_t)warps * sets * flag_words(inst->n) * 4, 128);
    L.aq_stride = aq_stride_for(inst->m, !inst->compact);
    L.total = align_up(L.off_aq + (size_t)warps * sets * 32 * L.aq_stride * 4, 128);
    // the one-set streamed kernel keeps a shared copy of the processing times
    // when it fits (compact records); the others read them from global memory
    L.off_ptab = 0;
    if (!resident && npw == 32 && inst->compact) add_ptab(L, inst, budget);
    return L;
}

template <bool WIDE, int MP>
cudaError_t launch_lanes_variant(const LanesArgs &a, bool resident, int npw, int grid, int threads, size_t smem,
                                 cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    if (resident) return launch_resident_mp(a, WIDE, MP, grid, threads, smem, s);
    if (npw != 32) return launch_streamed28_mp(a, MP, npw == 56 ? 2 : 1, grid, threads, smem, s);
    std::call_once(once, [] {
        attr_err = set_smem_attr(fsp_lanes_streamed<WIDE, MP, false>);
        if (!WIDE && attr_err == cudaSuccess) attr_err = set_smem_attr(fsp_lanes_streamed<WIDE, MP, !WIDE>);
    });
    if (attr_err != cudaSuccess) return attr_err;
    note_launches(1);
    if (!WIDE && a.off_ptab)
        fsp_lanes_streamed<WIDE, MP, !WIDE><<<grid, threads, smem, s>>>(a);
    else
        fsp_lanes_streamed<WIDE, MP, false><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_lanes_mp(const LanesArgs &a, int mp, bool resident, int npw, int grid, int threads, size_t smem,
                            cudaStream_t s) {
    switch (mp) {
        case 8: return launch_lanes_variant<WIDE, 8>(a, resident, npw, grid, threads, smem, s);
        case 12: return launch_lanes_variant<WIDE, 12>(a, resident, npw, grid, threads, smem, s);
        case 16: return launch_lanes_variant<WIDE, 16>(a, resident, npw, grid, threads, smem, s);
        case 20: return launch_lanes_variant<WIDE, 20>(a, resident, npw, grid, threads, smem, s);
        case 24: return launch_lanes_variant<WIDE, 24>(a, resident, npw, grid, threads, smem, s);
        default: return launch_lanes_variant<WIDE, 32>(a, resident, npw, grid, threads, smem, s);
    }
}

// Global staging: flag words and node rows of every warp, nothing else.
LanesLayout global_layout_for(const fsp_instance *inst, int warps, size_t budget) {
    LanesLayout L = {};
    L.off_flags = 0;
    L.off_aq = (uint32_t)align_up((size_t)warps * flag_words(inst->n) * 4, 128);
    L.aq_stride = aq_stride_for(inst->m, !inst->compact);
    L.total = align_up(L.off_aq + (size_t)warps * 32 * L.aq_stride * 4, 128);
    if (inst->compact) add_ptab(L, inst, budget);
    return L;
}

// Shared memory a block may take: the opt-in maximum, or an equal share of
// the SM for several blocks per SM.
size_t lanes_budget(const fsp_instance *inst, int bps) {
    return bps <= 1 ? (size_t)max_smem_per_block(inst->device)
                    : std::min((size_t)max_smem_per_block(inst->device),
                               (size_t)max_smem_per_sm(inst->device) / bps - 1024);
}


}  // namespace

int lanes_nodes_per_warp(const fsp_launch_config &c) {
    const int v = c.nodes_per_thread;
    return v == 0 ? 32 : (v == 32 || v == 28 || v == 56) ? v : 0;
}

int lanes_groups_per_item(const fsp_instance *inst, int pairs_per_tile) {
    if (pairs_per_tile <= 0 || pairs_per_tile >= inst->P) return inst->G;
    return std::min(inst->G, (pairs_per_tile + 31) / 32);
}

fsp_status lanes_layout(const fsp_instance *inst, const fsp_launch_config &c, size_t *smem_bytes) {
    if (c.staging == FSP_STAGING_SPLIT) return split_layout(inst, c, smem_bytes);
    if (c.staging == FSP_STAGING_WARP) return warp_layout(inst, c, smem_bytes);
    const int W = c.warps_per_block;
    const int bps = c.blocks_per_sm ? c.blocks_per_sm : 1;
    if (c.staging == FSP_STAGING_GLOBAL) {
        // compact records only (the register ring holds two-word records)
        if (!inst->compact || W < 1 || W > 16 || bps < 1 || W * bps > 16) return FSP_EINVAL;
        const size_t budget = lanes_budget(inst, bps);
        const LanesLayout L = global_layout_for(inst, W, budget);
        if (L.total > budget) return FSP_EINVAL;
        *smem_bytes = L.total;
        return FSP_OK;
    }
    const bool resident = c.staging == FSP_STAGING_RESIDENT;
    // up to 8 blocks per SM for streamed staging (small node tiles of small
    // pools), 2 otherwise
    if (W < 1 || W > 16 || bps < 1 || bps > (resident ? 2 : 8) || W * bps > 16) return FSP_EINVAL;
    if (!resident && (c.positions_per_tile < 4 || (c.positions_per_tile & 3))) return FSP_EINVAL;
    // nodes per warp: 32, or 28 and 56 (one and two sets of 28: streamed
    // staging, compact records)
    const int npw = lanes_nodes_per_warp(c);
    if (!npw || (npw != 32 && (resident || !inst->compact))) return FSP_EINVAL;
    const int chunk = resident ? inst->npad : std::min(c.positions_per_tile, inst->npad);
    const size_t budget = lanes_budget(inst, bps);
    const LanesLayout L = lanes_layout_for(inst, W, resident, chunk, budget, npw);
    if (L.total > budget) return FSP_EINVAL;
    // the resident copy completes on one mbarrier: its byte count must fit the transaction counter
    if (resident && (size_t)inst->npad * 32 * inst->grec_bytes * inst->G >= (1u << 20)) return FSP_EINVAL;
    *smem_bytes = L.total;
    return FSP_OK;
}

namespace {

fsp_status launch_global(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                         int32_t *out_lb, void *stream, const fsp_launch_config &cfg, size_t smem) {
    const int W = cfg.warps_per_block;
    const int bps = cfg.blocks_per_sm ? cfg.blocks_per_sm : 1;
    const LanesLayout L = global_layout_for(inst, W, lanes_budget(inst, bps));
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
    a.n = inst->n;
    a.m = inst->m;
    a.G = inst->G;
    a.npad = inst->npad;
    a.mpad = inst->mpad;
    a.rec_bytes = (uint32_t)inst->grec_bytes;
    a.off_flags = L.off_flags;
    a.off_aq = L.off_aq;
    a.off_ptab = L.off_ptab;
    a.aq_stride = L.aq_stride;
    a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
    a.q32 = 0;
    a.wait_limit = 4000000000LL;
    a.num_batches = (N + 31) / 32;
    a.gper = lanes_groups_per_item(inst, cfg.pairs_per_tile);
    a.gslices = (inst->G + a.gper - 1) / a.gper;
    const int64_t items = a.num_batches * a.gslices;
    const int64_t slots = (int64_t)num_sms(inst->device) * bps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((items + W - 1) / W, slots));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // couple slices combine by atomic max into zeroed bounds
    if (a.gslices > 1 && cudaMemsetAsync(out_lb, 0, sizeof(int32_t) * (size_t)N, s) != cudaSuccess)
        return FSP_ECUDA;
    int32_t *order = nullptr;
    fsp_status st = depth_order(inst, depths, N, s, &order);
    if (st != FSP_OK) return st;
    a.order = order;
    const cudaError_t e = launch_global_mp(a, inst->mpad, grid, 32 * W, smem, s);
    const cudaError_t ef = order ? cudaFreeAsync(order, s) : cudaSuccess;
    return (e == cudaSuccess && ef == cudaSuccess) ? FSP_OK : FSP_ECUDA;
}

}  // namespace

fsp_status launch_lanes(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *stream, const fsp_launch_config &cfg) {
    if (cfg.staging == FSP_STAGING_SPLIT) return launch_split(inst, nodes, depths, N, out_lb, stream, cfg);
    if (cfg.staging == FSP_STAGING_WARP) return launch_warp(inst, nodes, depths, N, out_lb, stream, cfg);
    size_t smem = 0;
    fsp_status st = lanes_layout(inst, cfg, &smem);
    if (st != FSP_OK) return st;
    if (cfg.staging == FSP_STAGING_GLOBAL) return launch_global(inst, nodes, depths, N, out_lb, stream, cfg, smem);
    const int W = cfg.warps_per_block;
    const bool resident = cfg.staging == FSP_STAGING_RESIDENT;
    const int chunk = resident ? inst->npad : std::min(cfg.positions_per_tile, inst->npad);
    const int npw = lanes_nodes_per_warp(cfg);
    const LanesLayout L = lanes_layout_for(inst, W, resident, chunk,
                                           lanes_budget(inst, cfg.blocks_per_sm ? cfg.blocks_per_sm : 1), npw);
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
    a.off_tables = L.off_tables;
    a.tile_stride = L.tile_stride;
    a.off_flags = L.off_flags;
    a.off_aq = L.off_aq;
    a.off_ptab = resident ? 0u : L.off_ptab;
    a.aq_stride = L.aq_stride;
    a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
    a.q32 = inst->compact ? 0 : 1;
    a.wait_limit = 4000000000LL;
    int grid;
    if (resident) {
        a.num_batches = (N + 31) / 32;
        // at least one warp batch per warp of the grid
        const int64_t per_block = std::max<int64_t>(1, W);
        grid = (int)std::min<int64_t>((a.num_batches + per_block - 1) / per_block, (int64_t)num_sms(inst->device));
    } else {
        a.num_batches = (N + (int64_t)npw * W - 1) / ((int64_t)npw * W);
        const int bps = cfg.blocks_per_sm ? cfg.blocks_per_sm : 1;
        const int64_t slots = (int64_t)num_sms(inst->device) * bps;
        a.gper = lanes_groups_per_item(inst, cfg.pairs_per_tile);
        a.gslices = (inst->G + a.gper - 1) / a.gper;
        a.full_batches = 0;
        if (a.gslices == 1 && cfg.tail_slices > 1 && a.num_batches > slots) {
            // whole batches in full waves, the last partial wave's batches sliced
            const int st = std::min(cfg.tail_slices, inst->G);
            a.gper = (inst->G + st - 1) / st;
            a.gslices = (inst->G + a.gper - 1) / a.gper;
            a.full_batches = a.num_batches - a.num_batches % slots;
            if (a.full_batches == a.num_batches) a.gslices = 1;
        }
        if (a.gslices > 1 && (a.num_batches - a.full_batches) * a.gslices >= ((int64_t)1 << 31)) return FSP_EINVAL;
        grid = (int)std::min<int64_t>(a.full_batches + (a.num_batches - a.full_batches) * a.gslices, slots);
    }
    grid = std::max(grid, 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // couple slices combine by atomic max into zeroed bounds
    if (a.gslices > 1 && cudaMemsetAsync(out_lb, 0, sizeof(int32_t) * (size_t)N, s) != cudaSuccess)
        return FSP_ECUDA;
    int32_t *order = nullptr;
    st = depth_order(inst, depths, N, s, &order);
    if (st != FSP_OK) return st;
    a.order = order;
    const cudaError_t e = inst->compact ? launch_lanes_mp<false>(a, inst->mpad, resident, npw, grid, 32 * W, smem, s)
                                        : launch_lanes_mp<true>(a, inst->mpad, resident, npw, grid, 32 * W, smem, s);
    const cudaError_t ef = order ? cudaFreeAsync(order, s) : cudaSuccess;
    return (e == cudaSuccess && ef == cudaSuccess) ? FSP_OK : FSP_ECUDA;
}

}  // namespace fspgb
