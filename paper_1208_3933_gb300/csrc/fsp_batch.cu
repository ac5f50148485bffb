// fsp_batch.cu -- many pools of many instances bounded in one persistent
// launch (the batched form of the bounding operator of Section III-A).
//
// A batch plan lists every pool's 32-node work items, longest first (cost =
// couple groups x Johnson positions of the pool's instance), and uploads the
// list and the per-pool arguments to the device once.  One persistent launch
// of fsp_lanes_batch then covers the whole plan: each warp claims work items
// from a device counter, sets up its 32 nodes (lane = node), and scans the
// instance's couple groups (lane = couple) reading the Johnson records from
// L2/L1, so warps of one block may work on different instances.  The launch
// can be captured once in a CUDA graph (counter reset + kernel) and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fsp_internal.h"
#include "fsp_batch_scan.cuh"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

template <int MP>
__global__ void __launch_bounds__(512, 1)
    fsp_lanes_batch(const LanesArgs *__restrict__ pools, const int2 *__restrict__ items, int64_t nitems,
                    int32_t *counter, int32_t n_max, int32_t aq_stride, uint32_t off_aq) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem) + (size_t)warp * n_max;
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + off_aq) + (size_t)warp * 32 * aq_stride;
    for (;;) {
        int claim = 0;
        if (lane == 0) claim = atomicAdd(counter, 1);
        claim = __shfl_sync(kFull, claim, 0);
        if ((int64_t)claim >= nitems) break;
        const int2 it = __ldg(items + claim);
        const LanesArgs &a = pools[it.x];
        // a pool split by couples: item y = batch * S + slice, the slice
        // covering couple groups [slice * gper, (slice + 1) * gper)
        const int S = a.gslices > 1 ? a.gslices : 1;
        const int batch = S > 1 ? it.y / S : it.y, slice = S > 1 ? it.y - batch * S : 0;
        const int64_t x = (int64_t)batch * 32 + lane;
        int bterm = 0;
        const bool valid = lanes_setup<MP>(a, x, lane, F, AQ + lane * aq_stride, bterm);
        int lb[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) lb[b] = 0;
        const int npad = a.npad, m = a.m;
        const int g0 = S > 1 ? slice * a.gper : 0, G = S > 1 ? min(a.G, g0 + a.gper) : a.G;
        for (int g = g0; g < G; ++g) {
            const int kk = __ldg(a.gpairs + 2 * (g * 32 + lane)), ll = __ldg(a.gpairs + 2 * (g * 32 + lane) + 1);
            int u[32];
#pragma unroll
            for (int b = 0; b < 32; ++b) u[b] = 0;
            const uint2 *R = reinterpret_cast<const uint2 *>(a.grec) + (size_t)g * npad * 32 + lane;
            scan_compact_global(R, npad, F, u);
            couple_epilogue<false>(AQ, aq_stride, m, kk, ll, u, lb);
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

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int MP>
cudaError_t launch_batch_variant(const LanesArgs *pools, const int2 *items, int64_t nitems, int32_t *counter,
                                 int n_max, int stride, uint32_t off_aq, int grid, int threads, size_t smem,
                                 cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        attr_err = cudaFuncSetAttribute(fsp_lanes_batch<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    });
    if (attr_err != cudaSuccess) return attr_err;
    fsp_lanes_batch<MP><<<grid, threads, smem, s>>>(pools, items, nitems, counter, n_max, stride, off_aq);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

}  // namespace fspgb

using namespace fspgb;

struct fsp_batch {
    int device = 0;
    fspgb::PlanParams pp;
    void *dev_block = nullptr;  // pools, items and the work counter
    LanesArgs *d_pools = nullptr;
    int2 *d_items = nullptr;
    int32_t *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::mutex mu;
};

namespace {

fsp_status enqueue(fsp_batch *b, cudaStream_t s) { return launch_plan(b->d_pools, b->d_items, b->d_counter, b->pp, s); }

}  // namespace

namespace fspgb {

fsp_status build_plan(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block, int32_t couples_per_item,
                      int device, std::vector<LanesArgs> &args, std::vector<int2> &items, PlanParams &pp) {
    if (count < 0 || (count > 0 && !pools) || warps_per_block < 0 || warps_per_block > 16 || couples_per_item < 0)
        return FSP_EINVAL;
    int n_max = 1, m_max = 2, mp = 8;
    for (int32_t i = 0; i < count; ++i) {
        const fsp_pool_desc &p = pools[i];
        if (!p.inst || p.N < 0 || (p.N > 0 && (!p.nodes || !p.depths || !p.out_lb))) return FSP_EINVAL;
        if (p.inst->device != device || !p.inst->compact) return FSP_EINVAL;
        n_max = std::max(n_max, p.inst->n);
        m_max = std::max(m_max, p.inst->m);
        mp = std::max(mp, p.inst->mpad);
    }
    pp = PlanParams();
    pp.couples_per_item = couples_per_item;
    const int gper = couples_per_item ? (couples_per_item + 31) / 32 : 0;  // couple groups per item
    pp.mp = mp;
    pp.n_max = flag_words(n_max);  // flag words per warp
    pp.stride = (m_max + (m_max + 1) / 2) | 1;
    // work items, longest first: couple groups x Johnson positions of the instance
    items.clear();
    args.assign((size_t)count, LanesArgs());
    for (int32_t i = 0; i < count; ++i) {
        const fsp_pool_desc &p = pools[i];
        const fsp_instance *inst = p.inst;
        LanesArgs &a = args[i];
        std::memset(&a, 0, sizeof a);
        a.grec = static_cast<const unsigned char *>(inst->t.grec);
        a.gpairs = inst->t.gpairs;
        a.hsort = reinterpret_cast<const int2 *>(inst->t.hsort);
        a.tsort = reinterpret_cast<const int2 *>(inst->t.tsort);
        a.ptot = inst->t.ptot;
        a.pp = inst->t.pp;
        a.nodes = p.nodes;
        a.depths = p.depths;
        a.out = p.out_lb;
        a.status = inst->dev_status;
        a.N = p.N;
        a.n = inst->n;
        a.m = inst->m;
        a.G = inst->G;
        a.npad = inst->npad;
        a.mpad = inst->mpad;
        a.rec_bytes = (uint32_t)inst->grec_bytes;
        a.aq_stride = pp.stride;
        a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
        a.q32 = inst->compact ? 0 : 1;
        a.wait_limit = 4000000000LL;
        const int S = (gper && inst->G > gper) ? (inst->G + gper - 1) / gper : 1;
        a.gper = S > 1 ? gper : inst->G;
        a.gslices = S;
        const int64_t nb = (p.N + 31) / 32;
        if (nb * S > INT32_MAX) return FSP_EINVAL;
        for (int64_t k = 0; k < nb * S; ++k) items.push_back(make_int2(i, (int)k));
        if (S > 1 && p.N > 0) pp.zero.emplace_back(p.out_lb, p.N);
        pp.nodes += p.N;
    }
    // longest first: couple groups of the item x Johnson positions
    auto cost = [&](const int2 &w) {
        const LanesArgs &a = args[w.x];
        const int S = a.gslices;
        const int slice = S > 1 ? w.y % S : 0;
        const int groups = S > 1 ? std::min(a.G - slice * a.gper, a.gper) : a.G;
        return (int64_t)groups * a.npad;
    };
    std::stable_sort(items.begin(), items.end(), [&](const int2 &x, const int2 &y) { return cost(x) > cost(y); });
    pp.nitems = (int64_t)items.size();
    if (pp.nitems > INT32_MAX) return FSP_EINVAL;
    // shared memory: flags [warps][n_max] words, rows [warps][32][stride] ints
    const int smem_optin = max_smem_per_block(device);
    // Unless the caller fixes the node tile, a plan of fewer than 16 items
    // per SM takes the fewest warps per block that still put every item in
    // flight at once on at most one block per SM: the warps of one block sit
    // on different schedulers, so every warp runs its setup and scan without
    // sharing a scheduler, and no SM stays idle while another holds 16 warps
    // (a 140-item search batch in 16-warp blocks ran on 9 of 152 SMs).
    const int64_t sms = std::max(1, num_sms(device));
    int W = warps_per_block ? warps_per_block
                            : (int)std::min<int64_t>(16, std::max<int64_t>(1, (pp.nitems + sms - 1) / sms));
    for (; W >= 1; --W) {
        const uint32_t off_aq = (uint32_t)align_up((size_t)W * pp.n_max * 4, 128);
        const size_t total = align_up(off_aq + (size_t)W * 32 * pp.stride * 4, 128);
        if (total <= (size_t)smem_optin) {
            pp.off_aq = off_aq;
            pp.smem = total;
            break;
        }
        if (warps_per_block) break;
    }
    if (!pp.smem) return FSP_EINVAL;
    pp.warps = W;
    const int64_t blocks_needed = (pp.nitems + W - 1) / W;
    pp.grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, num_sms(device)));
    return FSP_OK;
}

fsp_status launch_plan(const LanesArgs *d_args, const int2 *d_items, int32_t *d_counter, const PlanParams &pp,
                       cudaStream_t s) {
    if (pp.nitems == 0) return FSP_OK;
    if (cudaMemsetAsync(d_counter, 0, sizeof(int32_t), s) != cudaSuccess) return FSP_ECUDA;
    for (const auto &z : pp.zero)
        if (cudaMemsetAsync(z.first, 0, sizeof(int32_t) * (size_t)z.second, s) != cudaSuccess) return FSP_ECUDA;
    cudaError_t e;
    switch (pp.mp) {
#define FSP_BATCH_CASE(MPV)                                                                                    \
    case MPV:                                                                                                   \
        e = launch_batch_variant<MPV>(d_args, d_items, pp.nitems, d_counter, pp.n_max, pp.stride, pp.off_aq, \
                                      pp.grid, 32 * pp.warps, pp.smem, s);                                    \
        break;
        FSP_BATCH_CASE(8)
        FSP_BATCH_CASE(12)
        FSP_BATCH_CASE(16)
        FSP_BATCH_CASE(20)
        FSP_BATCH_CASE(24)
#undef FSP_BATCH_CASE
        default:
            e = launch_batch_variant<32>(d_args, d_items, pp.nitems, d_counter, pp.n_max, pp.stride, pp.off_aq,
                                         pp.grid, 32 * pp.warps, pp.smem, s);
            break;
    }
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

}  // namespace fspgb

extern "C" fsp_status fsp_batch_create(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block,
                                       fsp_batch **out) {
    return fsp_batch_create_ex(pools, count, warps_per_block, 0, out);
}

extern "C" fsp_status fsp_batch_create_ex(const fsp_pool_desc *pools, int32_t count, int32_t warps_per_block,
                                          int32_t couples_per_item, fsp_batch **out) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    std::vector<LanesArgs> args;
    std::vector<int2> items;
    PlanParams pp;
    fsp_status st = build_plan(pools, count, warps_per_block, couples_per_item, dev, args, items, pp);
    if (st != FSP_OK) return st;
    fsp_batch *b = new (std::nothrow) fsp_batch();
    if (!b) return FSP_ENOMEM;
    b->device = dev;
    b->pp = pp;
    const size_t off_items = align_up(sizeof(LanesArgs) * std::max(1, count), 256);
    const size_t off_ctr = align_up(off_items + sizeof(int2) * std::max<int64_t>(1, pp.nitems), 256);
    const size_t bytes = off_ctr + 256;
    unsigned char *blk = nullptr;
    if (cudaMalloc((void **)&blk, bytes) != cudaSuccess) {
        delete b;
        return FSP_ENOMEM;
    }
    if ((count && cudaMemcpy(blk, args.data(), sizeof(LanesArgs) * count, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (pp.nitems &&
         cudaMemcpy(blk + off_items, items.data(), sizeof(int2) * pp.nitems, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(blk + off_ctr, 0, 256) != cudaSuccess) {
        cudaFree(blk);
        delete b;
        return FSP_ECUDA;
    }
    b->dev_block = blk;
    b->d_pools = reinterpret_cast<LanesArgs *>(blk);
    b->d_items = reinterpret_cast<int2 *>(blk + off_items);
    b->d_counter = reinterpret_cast<int32_t *>(blk + off_ctr);
    *out = b;
    return FSP_OK;
}

extern "C" fsp_status fsp_batch_launch(fsp_batch *b, void *cuda_stream) {
    if (!b) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != b->device) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(b->mu);
    return enqueue(b, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" fsp_status fsp_batch_launch_graph(fsp_batch *b, void *cuda_stream) {
    if (!b) return FSP_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    if (dev != b->device) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(b->mu);
    if (!b->exec) {
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return FSP_ECUDA;
        fsp_status st = FSP_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = FSP_ECUDA;
        } else {
            st = enqueue(b, cap);
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(cap, &graph);
            if (st == FSP_OK && e != cudaSuccess) st = FSP_ECUDA;
            if (st == FSP_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
                st = FSP_ECUDA;
                b->exec = nullptr;
            }
            if (graph) {
                if (st == FSP_OK)
                    b->graph = graph;
                else
                    cudaGraphDestroy(graph);
            }
        }
        cudaStreamDestroy(cap);
        if (st != FSP_OK) return st;
    }
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

extern "C" fsp_status fsp_batch_query_ex(const fsp_batch *b, int64_t *work_items, int64_t *nodes,
                                         int32_t *warps_per_block, int32_t *blocks, int32_t *couples_per_item) {
    if (!b) return FSP_EINVAL;
    if (couples_per_item) *couples_per_item = b->pp.couples_per_item;
    return fsp_batch_query(b, work_items, nodes, warps_per_block, blocks);
}

extern "C" fsp_status fsp_batch_query(const fsp_batch *b, int64_t *work_items, int64_t *nodes,
                                      int32_t *warps_per_block, int32_t *blocks) {
    if (!b) return FSP_EINVAL;
    if (work_items) *work_items = b->pp.nitems;
    if (nodes) *nodes = b->pp.nodes;
    if (warps_per_block) *warps_per_block = b->pp.warps;
    if (blocks) *blocks = b->pp.grid;
    return FSP_OK;
}

extern "C" void fsp_batch_destroy(fsp_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dev_block) cudaFree(b->dev_block);
    delete b;
}

// Times one plan shape on the stream: one warm-up launch, then three timed
// ones.  *ms = -1 when the shape does not fit the batch.
static fsp_status time_plan(const fsp_pool_desc *pools, int32_t count, int W, int cpi, cudaStream_t s,
                            cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    *ms = -1.f;
    fsp_batch *b = nullptr;
    const fsp_status cs = fsp_batch_create_ex(pools, count, W, cpi, &b);
    if (cs == FSP_EINVAL) return FSP_OK;  // the shape does not fit this batch
    if (cs != FSP_OK) return cs;
    constexpr int kReps = 3;
    float t = 0.f;
    fsp_status st = fsp_batch_launch(b, s);
    if (st == FSP_OK && cudaEventRecord(e0, s) != cudaSuccess) st = FSP_ECUDA;
    for (int r = 0; r < kReps && st == FSP_OK; ++r) st = fsp_batch_launch(b, s);
    if (st == FSP_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = FSP_ECUDA;
    cudaStreamSynchronize(s);
    fsp_batch_destroy(b);
    if (st == FSP_OK) *ms = t / kReps;
    return st;
}

// Node tile first: plans of the same pools with 16, 12, 8, 6, 4 and 2 warps
// per block, every couple of a batch in one work item; then the couple
// split: the two fastest tiles again with 32, 64, 96 and 128 couples per
// work item (pools of more couple groups are split into that many slices).
// Every candidate writes the same bounds.
extern "C" fsp_status fsp_batch_autotune_ex(const fsp_pool_desc *pools, int32_t count, void *cuda_stream,
                                            int32_t *best_warps, int32_t *best_couples_per_item, float *best_ms) {
    if (!pools || count < 1 || !best_warps) return FSP_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FSP_ECUDA;
    }
    fsp_status st = FSP_OK;
    std::vector<std::pair<float, int>> tiles;  // (ms, warps)
    for (int W : {16, 12, 8, 6, 4, 2}) {
        float ms = -1.f;
        st = time_plan(pools, count, W, 0, s, e0, e1, &ms);
        if (st != FSP_OK) break;
        if (ms >= 0.f) tiles.emplace_back(ms, W);
    }
    float best = 1e30f;
    int bw = 0, bc = 0;
    if (st == FSP_OK && !tiles.empty()) {
        std::sort(tiles.begin(), tiles.end());
        best = tiles[0].first;
        bw = tiles[0].second;
        if (best_couples_per_item) {
            for (size_t t = 0; t < std::min<size_t>(2, tiles.size()) && st == FSP_OK; ++t)
                for (int cpi : {32, 64, 96, 128}) {
                    float ms = -1.f;
                    st = time_plan(pools, count, tiles[t].second, cpi, s, e0, e1, &ms);
                    if (st != FSP_OK) break;
                    if (ms >= 0.f && ms < best) {
                        best = ms;
                        bw = tiles[t].second;
                        bc = cpi;
                    }
                }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FSP_OK) return st;
    if (!bw) return FSP_EINVAL;
    *best_warps = bw;
    if (best_couples_per_item) *best_couples_per_item = bc;
    if (best_ms) *best_ms = best;
    return FSP_OK;
}

extern "C" fsp_status fsp_batch_autotune(const fsp_pool_desc *pools, int32_t count, void *cuda_stream,
                                         int32_t *best_warps, float *best_ms) {
    return fsp_batch_autotune_ex(pools, count, cuda_stream, best_warps, nullptr, best_ms);
}
