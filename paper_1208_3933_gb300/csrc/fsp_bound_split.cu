// fsp_bound_split.cu -- the couple-lanes bound in two kernels: node setup,
// then the Johnson scan (sm_103a).
//
// The fused streamed kernel (fsp_bound_lanes.cu) runs each batch's setup and
// scan in one block that moves from record tile to record tile together, so
// the setup -- a chain of dependent loads and adds per node, latency bound --
// holds every warp of the block at the first tile barrier.  Here the two
// halves are separate launches on the same stream:
//
//   fsp_lanes_prep   one warp per 32 nodes, warps independent and many per SM
//                    (latency hidden by occupancy).  Per 32-node batch it
//                    builds the same state the fused kernel keeps in shared
//                    memory -- the job flag words F[j], the node rows
//                    (A_k int32, q_l int16 or int32), the one-machine term and the node
//                    index -- and writes it as one contiguous block of scratch
//                    (large pools are taken in depth order, fsp_order.cu).
//   fsp_lanes_scan   the block-synchronous tile scan of the fused kernel, with
//                    each batch's prepared state brought into shared memory by
//                    one bulk copy (cp.async.bulk on an mbarrier).
//
// The scratch is [batch][F: n words | rows: 32 * stride words | one-machine
// term: 32 | node index: 32], each batch block padded to 16 bytes; it comes
// from a per-device stream-ordered memory pool and is released on the stream
// after the scan.  Pools larger than kSplitChunk nodes are bounded chunk by
// chunk through one scratch allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "fsp_internal.h"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

namespace {

constexpr int kPrepWarps = 8;                 // warps (32-node batches) per prep block
constexpr int64_t kSplitChunk = int64_t(1) << 20;  // nodes per prep+scan pair

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ prep
// PS = kPtabByte: the block first copies the processing times of a compact
// instance to shared memory as bytes (when they fit beside the warps' state),
// so the prefix pass reads each job's row in one shared-memory latency
// instead of an L1 miss, a quarter of the bytes of an int32 copy.
template <int MP, int PS>
__global__ void __launch_bounds__(32 * kPrepWarps, 2) fsp_lanes_prep(const LanesArgs a, int64_t nbatch32) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int2 *hcache = reinterpret_cast<int2 *>(smem + a.off_cache);
    int2 *tcache = hcache + a.m * 32;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem + a.off_flags) + (size_t)warp * flag_words(a.n);
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + a.off_aq) + (size_t)warp * 32 * a.aq_stride;
    void *ptab = PS == kPtabByte ? smem + a.off_ptab : nullptr;
    load_sorted_heads(a, hcache, tcache);
    if constexpr (PS == kPtabByte) load_ptab(a, ptab);
    __syncthreads();
    const int rows_words = 32 * a.aq_stride;
    // warps are independent: warp w of block i takes the 32-node batches
    // w * gridDim.x + i, then every gridDim.x * kPrepWarps after it, so the
    // batches of a depth-ordered pool (deeper = longer setup) are dealt
    // across the blocks instead of the deepest ones landing on a few SMs
    for (int64_t b32 = (int64_t)warp * gridDim.x + blockIdx.x; b32 < nbatch32;
         b32 += (int64_t)gridDim.x * kPrepWarps) {
        const int64_t x = node_at(a, b32 * 32 + lane);
        int bterm = 0;
        const bool valid = lanes_setup<MP, PS>(a, x, lane, F, AQ + lane * a.aq_stride, bterm, hcache, tcache, ptab);
        uint32_t *dst = a.scratch + (size_t)b32 * a.sb_words;
        for (int j = lane; j < a.n; j += 32) dst[j] = F[j];
        const uint32_t *rows = reinterpret_cast<const uint32_t *>(AQ);
        for (int i = lane; i < rows_words; i += 32) dst[a.n + i] = rows[i];
        dst[a.n + rows_words + lane] = (uint32_t)(valid ? bterm : INT_MIN);
        dst[a.n + rows_words + 32 + lane] = (uint32_t)(x < a.N ? (int32_t)x : -1);
        __syncwarp();  // F and the rows are rewritten by the next batch
    }
}

// ------------------------------------------------------------------ scan
template <bool WIDE, int MP>
__global__ void __launch_bounds__(512, 1) fsp_lanes_scan(const LanesArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // [0], [1]: record tiles; [2]: prepared state
    uint8_t *sgp = smem + 32;
    unsigned char *prep = smem + a.off_flags;
    const uint32_t prep_bytes = (uint32_t)W * (uint32_t)a.sb_words * 4u;
    const int rows_words = 32 * a.aq_stride;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < a.G * 64; i += blockDim.x) sgp[i] = a.gpairs[i];
    __syncthreads();

    TilePipe tp{bar, smem + a.off_tables, a.tile_stride, a.ntiles <= 2};
    auto tile_issue = [&](uint32_t fill, int t) {
        const int g = t / a.nchunks, ch = t - g * a.nchunks;
        const int pos = min(a.chunk, a.npad - ch * a.chunk);
        const unsigned char *src = a.grec + ((size_t)g * a.npad + (size_t)ch * a.chunk) * 32 * a.rec_bytes;
        tp.issue(fill, src, (uint32_t)pos * 32u * a.rec_bytes);
    };
    // Work items: block batch bt = it / S, couple slice it % S of gper groups
    // (S = 1: every couple); the slices of a batch read the same prepared
    // state and meet in an atomic max on the zeroed bounds.
    const int S = a.gslices > 1 ? a.gslices : 1;
    const int gper = S > 1 ? a.gper : a.G;
    const int64_t items = a.num_batches * S;
    auto first_tile = [&](int64_t it) { return (int)(it % S) * gper * a.nchunks; };
    auto end_tile = [&](int64_t it) { return min(a.G, ((int)(it % S) + 1) * gper) * a.nchunks; };
    if (threadIdx.x == 0 && (int64_t)blockIdx.x < items) {
        if (tp.resident) {
            tile_issue(0, 0);
            if (a.ntiles == 2) tile_issue(1, 1);
        } else {
            tile_issue(0, first_tile(blockIdx.x));
        }
    }

    const uint32_t *F = reinterpret_cast<const uint32_t *>(prep) + (size_t)warp * a.sb_words;
    const int32_t *AQ = reinterpret_cast<const int32_t *>(F + a.n);
    uint32_t prep_phase = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x, prep_phase ^= 1u) {
        const int64_t bt = it / S;
        __syncthreads();  // the previous batch is done with the prepared state
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[2], prep_bytes);
            bulk_g2s(prep, a.scratch + (size_t)bt * W * a.sb_words, prep_bytes, &bar[2]);
        }
        const bool got = mbar_wait_bounded(&bar[2], prep_phase, a.wait_limit);
        if (!__syncthreads_and(got)) {
            if (threadIdx.x == 0) {
                report_status(a.status, (int32_t)FSP_ETIMEDOUT);
                mbar_wait_bounded(&bar[2], prep_phase, a.wait_limit);
                tp.drain(a.wait_limit);
            }
            return;
        }
        const int bterm = (int)F[a.n + rows_words + lane];
        const int xid = (int)F[a.n + rows_words + 32 + lane];
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
        const int t1 = end_tile(it);
        for (int t = first_tile(it); t < t1; ++t) {
            const int g = t / a.nchunks, ch = t - g * a.nchunks;
            if (!tp.resident && threadIdx.x == 0) {
                // the next tile of this item, else the first of the block's next item
                const int next = t + 1 < t1 ? t + 1 : (it + gridDim.x < items ? first_tile(it + gridDim.x) : -1);
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
        if (xid >= 0) {
            if (bterm == INT_MIN)
                a.out[xid] = FSP_LB_INVALID;  // every slice finds the row invalid
            else if (S == 1)
                a.out[xid] = max(best, bterm);
            else
                atomicMax(a.out + xid, max(best, bterm));  // out was zeroed; bounds are >= 0
        }
    }
}

// ------------------------------------------------------------------ host
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ints per node row: A_k as int32, then q_l as int16 (compact records) or int32
int aq_stride_for(int m, bool q32) { return (m + (q32 ? m : (m + 1) / 2)) | 1; }

// Words of one 32-node batch block of scratch (a multiple of 4: 16 bytes).
int sb_words_for(const fsp_instance *inst) {
    return (int)align_up((size_t)inst->n + 32 * (size_t)aq_stride_for(inst->m, !inst->compact) + 64, 4);
}

struct PrepLayout {
    uint32_t off_cache, off_flags, off_aq, off_ptab;  // off_ptab 0: no shared copy of the processing times
    size_t total;
};

// The prep block's shared memory; the processing times of a compact instance
// ([n][mpad] bytes) join it when the total stays within half an SM (two prep
// blocks per SM) and the table within 64 KB.
PrepLayout prep_layout_for(const fsp_instance *inst) {
    PrepLayout L;
    L.off_cache = 0;
    L.off_flags = (uint32_t)align_up((size_t)inst->m * 32 * 8 * 2, 128);
    L.off_aq = (uint32_t)align_up(L.off_flags + (size_t)kPrepWarps * flag_words(inst->n) * 4, 128);
    L.total = align_up(L.off_aq + (size_t)kPrepWarps * 32 * aq_stride_for(inst->m, !inst->compact) * 4, 128);
    L.off_ptab = 0;
    const size_t pbytes = (size_t)inst->n * inst->mpad;  // one byte per processing time
    const size_t budget = std::min((size_t)max_smem_per_block(inst->device),
                                   (size_t)max_smem_per_sm(inst->device) / 2 - 1024);
    if (inst->compact && pbytes <= 64 * 1024 && L.total + pbytes <= budget) {
        L.off_ptab = (uint32_t)L.total;
        L.total = align_up(L.total + pbytes, 128);
    }
    return L;
}

struct ScanLayout {
    uint32_t off_tables, tile_stride, off_prep;
    size_t total;
};

ScanLayout scan_layout_for(const fsp_instance *inst, int warps, int chunk) {
    ScanLayout L;
    L.off_tables = (uint32_t)align_up(32 + (size_t)inst->G * 64, 128);
    L.tile_stride = (uint32_t)align_up((size_t)chunk * 32 * inst->grec_bytes, 128);
    L.off_prep = (uint32_t)align_up(L.off_tables + 2 * (size_t)L.tile_stride, 128);
    L.total = align_up(L.off_prep + (size_t)warps * sb_words_for(inst) * 4, 128);
    return L;
}

// Launches prep then scan for one chunk; the prep grid fills the device once
// (resident blocks per SM from the occupancy calculator).
template <bool WIDE, int MP>
cudaError_t launch_pair(const LanesArgs &ap, int64_t nbatch32, size_t prep_smem, const LanesArgs &ac, int scan_grid,
                        int threads, size_t scan_smem, int sms, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = set_smem_attr(fsp_lanes_prep<MP, kPtabNone>);
        if (attr_err == cudaSuccess) attr_err = set_smem_attr(fsp_lanes_prep<MP, kPtabByte>);
        if (attr_err == cudaSuccess) attr_err = set_smem_attr(fsp_lanes_scan<WIDE, MP>);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const bool ps = ap.off_ptab != 0;
    int per_sm = 0;
    if ((ps ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fsp_lanes_prep<MP, kPtabByte>, 32 * kPrepWarps,
                                                            prep_smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fsp_lanes_prep<MP, kPtabNone>, 32 * kPrepWarps,
                                                            prep_smem)) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    // every SM takes per_sm blocks (the batches are dealt across them), but no
    // block is launched without a batch of its own
    const int prep_grid = (int)std::max<int64_t>(1, std::min<int64_t>(nbatch32, (int64_t)sms * per_sm));
    note_launches(2);
    if (ps)
        fsp_lanes_prep<MP, kPtabByte><<<prep_grid, 32 * kPrepWarps, prep_smem, s>>>(ap, nbatch32);
    else
        fsp_lanes_prep<MP, kPtabNone><<<prep_grid, 32 * kPrepWarps, prep_smem, s>>>(ap, nbatch32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fsp_lanes_scan<WIDE, MP><<<scan_grid, threads, scan_smem, s>>>(ac);
    return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_pair_mp(int mp, const LanesArgs &ap, int64_t nbatch32, size_t prep_smem, const LanesArgs &ac,
                           int scan_grid, int threads, size_t scan_smem, int sms, cudaStream_t s) {
    switch (mp) {
        case 8: return launch_pair<WIDE, 8>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
        case 12: return launch_pair<WIDE, 12>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
        case 16: return launch_pair<WIDE, 16>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
        case 20: return launch_pair<WIDE, 20>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
        case 24: return launch_pair<WIDE, 24>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
        default: return launch_pair<WIDE, 32>(ap, nbatch32, prep_smem, ac, scan_grid, threads, scan_smem, sms, s);
    }
}

}  // namespace

fsp_status split_layout(const fsp_instance *inst, const fsp_launch_config &c, size_t *smem_bytes) {
    const int W = c.warps_per_block;
    const int bps = c.blocks_per_sm ? c.blocks_per_sm : 1;
    if (W < 1 || W > 16 || bps < 1 || bps > 2 || W * bps > 16) return FSP_EINVAL;
    if (c.positions_per_tile < 4 || (c.positions_per_tile & 3)) return FSP_EINVAL;
    const int chunk = std::min(c.positions_per_tile, inst->npad);
    const ScanLayout L = scan_layout_for(inst, W, chunk);
    const size_t budget = bps == 1 ? (size_t)max_smem_per_block(inst->device)
                                   : std::min((size_t)max_smem_per_block(inst->device),
                                              (size_t)max_smem_per_sm(inst->device) / 2 - 1024);
    if (L.total > budget) return FSP_EINVAL;
    if (prep_layout_for(inst).total > (size_t)max_smem_per_block(inst->device)) return FSP_EINVAL;
    // the prepared state of a block batch completes on one mbarrier
    if ((size_t)W * sb_words_for(inst) * 4 >= (1u << 20)) return FSP_EINVAL;
    *smem_bytes = L.total;
    return FSP_OK;
}

fsp_status launch_split(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *stream, const fsp_launch_config &cfg) {
    size_t scan_smem = 0;
    fsp_status st = split_layout(inst, cfg, &scan_smem);
    if (st != FSP_OK) return st;
    if (N <= 0) return FSP_OK;
    const int W = cfg.warps_per_block;
    const int bps = cfg.blocks_per_sm ? cfg.blocks_per_sm : 1;
    const int chunk = std::min(cfg.positions_per_tile, inst->npad);
    const ScanLayout SL = scan_layout_for(inst, W, chunk);
    const PrepLayout PL = prep_layout_for(inst);
    const int sb = sb_words_for(inst);
    const int64_t per_call = std::min<int64_t>(N, kSplitChunk);
    const int64_t max_b32 = (per_call + 32 * W - 1) / (32 * W) * W;  // 32-node batches, whole block batches
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaMemPool_t pool = nullptr;
    st = scratch_pool(inst->device, &pool);
    if (st != FSP_OK) return st;
    uint32_t *scratch = nullptr;
    if (cudaMallocFromPoolAsync((void **)&scratch, (size_t)max_b32 * sb * 4, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return FSP_ENOMEM;
    }

    LanesArgs a = {};
    a.grec = static_cast<const unsigned char *>(inst->t.grec);
    a.gpairs = inst->t.gpairs;
    a.hsort = reinterpret_cast<const int2 *>(inst->t.hsort);
    a.tsort = reinterpret_cast<const int2 *>(inst->t.tsort);
    a.ptot = inst->t.ptot;
    a.pp = inst->t.pp;
    a.status = inst->dev_status;
    a.n = inst->n;
    a.m = inst->m;
    a.G = inst->G;
    a.npad = inst->npad;
    a.mpad = inst->mpad;
    a.chunk = chunk;
    a.nchunks = (inst->npad + chunk - 1) / chunk;
    a.ntiles = inst->G * a.nchunks;
    a.rec_bytes = (uint32_t)inst->grec_bytes;
    a.aq_stride = aq_stride_for(inst->m, !inst->compact);
    a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
    a.q32 = inst->compact ? 0 : 1;
    a.scratch = scratch;
    a.sb_words = sb;
    a.wait_limit = 4000000000LL;
    LanesArgs ap = a, ac = a;
    ap.off_cache = PL.off_cache;
    ap.off_flags = PL.off_flags;
    ap.off_aq = PL.off_aq;
    ap.off_ptab = PL.off_ptab;
    ac.off_tables = SL.off_tables;
    ac.tile_stride = SL.tile_stride;
    ac.off_flags = SL.off_prep;

    cudaError_t e = cudaSuccess;
    for (int64_t off = 0; off < N && e == cudaSuccess; off += per_call) {
        const int64_t n_here = std::min<int64_t>(per_call, N - off);
        const int64_t nb32 = (n_here + 32 * W - 1) / (32 * W) * W;
        ap.nodes = ac.nodes = nodes + off * inst->n;
        ap.depths = ac.depths = depths + off;
        ap.out = ac.out = out_lb + off;
        ap.N = ac.N = n_here;
        ap.num_batches = (nb32 + kPrepWarps - 1) / kPrepWarps;  // prep blocks' worth of batches
        ac.num_batches = nb32 / W;
        // couple slices of every block batch (pairs_per_tile below P): the
        // bounds are zeroed first and the slices meet in an atomic max
        const int gper = lanes_groups_per_item(inst, cfg.pairs_per_tile);
        const int S = gper < inst->G ? (inst->G + gper - 1) / gper : 1;
        ac.gper = gper;
        ac.gslices = S;
        if (S > 1 && cudaMemsetAsync(out_lb + off, 0, sizeof(int32_t) * (size_t)n_here, s) != cudaSuccess) {
            e = cudaErrorUnknown;
            break;
        }
        int32_t *order = nullptr;
        st = depth_order(inst, depths + off, n_here, s, &order);
        if (st != FSP_OK) break;
        ap.order = order;
        const int sms = num_sms(inst->device);
        const int scan_grid =
            (int)std::max<int64_t>(1, std::min<int64_t>(ac.num_batches * S, (int64_t)sms * bps));
        e = inst->compact ? launch_pair_mp<false>(inst->mpad, ap, nb32, PL.total, ac, scan_grid, 32 * W, scan_smem,
                                                  sms, s)
                          : launch_pair_mp<true>(inst->mpad, ap, nb32, PL.total, ac, scan_grid, 32 * W, scan_smem,
                                                 sms, s);
        if (order && cudaFreeAsync(order, s) != cudaSuccess && e == cudaSuccess) e = cudaErrorUnknown;
    }
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (st != FSP_OK) return st;
    return (e == cudaSuccess && ef == cudaSuccess) ? FSP_OK : FSP_ECUDA;
}

}  // namespace fspgb
