// fsp_bound.cu -- the bounding operator of Section III-A on sm_103a: one
// launch bounds a whole pool of sub-problems with the two-machine lower bound
// of Section II-C (figure "Pseudo-code implementing the LB function").
//
// Work decomposition.  A block of 128 threads owns a tile of 128*K nodes;
// thread t bounds nodes t, t+128, ..., t+128(K-1) of the tile in lockstep,
// so every thread of a warp reads the same Johnson record at the same time
// (a shared-memory broadcast) and only the per-node membership byte differs.
// Blocks are persistent: each walks node tiles blockIdx.x, +gridDim.x, ...
//
// Per node (prefix sigma of depth d, unscheduled set U):
//   1. flags:  byte flags[j][t] holds bit b = "job j in U for node b of t";
//   2. prefix: C(sigma,k) by the flow-shop recurrence (Section II-B);
//   3. A_k = r_k + S_k with r_k = max(C(sigma,k), min_{j in U} sum_{h<k} p_jh)
//      (RM) and S_k = sum_{j in U} p_jk;
//   4. for every machine l: q_l = min_{j in U} sum_{h>l} p_jh (QM) and the
//      term A_l + q_l;
//   5. for every couple (k,l): the filtered Johnson scan, run on the slack
//      u = timeOnM2 - timeOnM1 of the pseudo-code.  Its two-machine update is
//      timeOnM1 += p_jk; timeOnM2 = max(timeOnM2, timeOnM1 + lag_j) + p_jl,
//      which is u <- max(u + delta_j, s_j) with delta_j = p_jl - p_jk and
//      s_j = lag_j + p_jl.  That map composes to u_end = max(u_0 + S_l - S_k,
//      F(0)), where F(0) is the scan started from u = 0, and since
//      u_0 = r_l - r_k >= 0 the couple's value (timeOnM2 plus the latency) is
//          max(A_l + q_l, A_k + q_l + F(0)).
//      The scan therefore needs neither release time: it starts at 0 and
//      is the only O(n) loop per couple;
//   6. LB = max over all terms, or FSP_LB_INVALID for a bad row.
// Scheduled jobs and padding entries leave u unchanged: for a scheduled job
// the update is skipped, and padding records (delta = s = 0) map u >= 0 to
// itself.
//
// Shared memory: the Johnson records of a tile of couples (double-buffered,
// staged with cp.async.bulk and an mbarrier), the couple list, A [m][K][128]
// and the flags [n][128].  When all couples fit in the two buffers they are
// staged once per block and stay resident; otherwise the couple tiles are
// re-staged for every node tile, overlapped with the scan of the previous
// tile (the paper's "does not fit" case, Section IV-B).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "fsp_internal.h"
#include "fsp_ptx.cuh"

namespace fspgb {

struct BoundArgs {
    const unsigned char *rec;
    const uint8_t *pairs;
    const int32_t *p, *head, *tail, *ptm;
    const int16_t *nodes;
    const int32_t *depths;
    int32_t *out;
    int32_t *status;        // first device-side error (host-mapped), may be null
    int64_t N;
    int64_t num_node_tiles;
    int32_t n, m, P, npad;
    int32_t ppt;            // couples per staged tile
    int32_t ntiles;         // number of couple tiles
    uint32_t rec_bytes;
    uint32_t off_tiles, tile_stride, off_A, off_flags;
    long long wait_limit;   // clock64 cycles for one bounded mbarrier wait
};

// ---------------------------------------------------------------- the kernel
template <int K>
__device__ __forceinline__ void johnson_step(int j, int s, int delta, const uint8_t *__restrict__ sflags, int tid,
                                             int (&u)[K]) {
    const uint32_t fb = sflags[(j << 7) + tid];
#pragma unroll
    for (int b = 0; b < K; ++b) {
        if ((fb >> b) & 1u) u[b] = max(u[b] + delta, s);
    }
}

template <int K, bool WIDE>
__global__ void __launch_bounds__(kThreads) fsp_bound_kernel(const BoundArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    static_assert(kThreads == 128, "flag addressing assumes 128 threads");
    constexpr int KT = K * kThreads;
    const int tid = threadIdx.x;
    const int n = a.n, m = a.m;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint8_t *spairs = smem + 16;
    unsigned char *tiles = smem + a.off_tiles;
    int32_t *sA = reinterpret_cast<int32_t *>(smem + a.off_A);
    uint8_t *sflags = smem + a.off_flags;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    for (int i = tid; i < 2 * a.P; i += kThreads) spairs[i] = a.pairs[i];
    __syncthreads();

    const bool resident = a.ntiles <= 2;
    // Copies in flight per buffer (tracked by thread 0, which issues them):
    // bit i of `pending` set = buffer i has an issued fill not yet waited for,
    // whose phase parity is bit i of `pend_par`.
    uint32_t pending = 0, pend_par = 0;
    auto issue = [&](uint32_t fill, int t) {
        const int c0 = t * a.ppt;
        const int np = min(a.ppt, a.P - c0);
        const uint32_t bytes = (uint32_t)np * (uint32_t)a.npad * a.rec_bytes;
        const uint32_t bi = fill & 1;
        uint64_t *b = &bar[bi];
        mbar_arrive_expect_tx(b, bytes);
        bulk_g2s(tiles + bi * a.tile_stride, a.rec + (size_t)c0 * a.npad * a.rec_bytes, bytes, b);
        pending |= 1u << bi;
        pend_par = (pend_par & ~(1u << bi)) | (((fill >> 1) & 1u) << bi);
    };
    if (tid == 0 && (int64_t)blockIdx.x < a.num_node_tiles) {
        issue(0, 0);
        if (a.ntiles == 2) issue(1, 1);
    }
    uint32_t fill = 0;  // fill being consumed (re-staging mode)

    for (int64_t nt = blockIdx.x; nt < a.num_node_tiles; nt += gridDim.x) {
        const int64_t base = nt * KT;
        // ---- 1. depths and the membership flags
        uint32_t vmask = 0;
        int dd[K];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const int64_t x = base + b * kThreads + tid;
            dd[b] = 0;
            if (x < a.N) {
                const int d = __ldg(a.depths + x);
                if (d >= 0 && d <= n) {
                    vmask |= 1u << b;
                    dd[b] = d;
                }
            }
        }
        for (int j = 0; j < n; ++j) sflags[(j << 7) + tid] = (uint8_t)vmask;

        // ---- 2. prefix completion times C(sigma,k), kept in A
#pragma unroll
        for (int b = 0; b < K; ++b) {
            int32_t *Ab = sA + b * kThreads + tid;
            for (int k = 0; k < m; ++k) Ab[k * KT] = 0;
            if ((vmask >> b) & 1u) {
                const int16_t *row = a.nodes + (base + b * kThreads + tid) * (int64_t)n;
                for (int i = 0; i < dd[b]; ++i) {
                    const int j = __ldg(row + i);
                    if ((unsigned)j >= (unsigned)n) {
                        vmask &= ~(1u << b);
                        break;
                    }
                    const uint32_t fv = sflags[(j << 7) + tid];
                    if (!((fv >> b) & 1u)) {  // job already in the prefix
                        vmask &= ~(1u << b);
                        break;
                    }
                    sflags[(j << 7) + tid] = (uint8_t)(fv & ~(1u << b));
                    const int32_t *pj = a.p + j * m;
                    int c = 0;
                    for (int k = 0; k < m; ++k) {
                        c = max(c, Ab[k * KT]) + __ldg(pj + k);
                        Ab[k * KT] = c;
                    }
                }
            }
        }

        // ---- 3. A_k = max(C_k, min head over U) + sum of p_jk over U
        for (int k = 0; k < m; ++k) {
            int mh[K], S[K];
#pragma unroll
            for (int b = 0; b < K; ++b) {
                mh[b] = INT_MAX;
                S[b] = 0;
            }
            const int32_t *hk = a.head + k * n;
            const int32_t *pk = a.ptm + k * n;
            for (int j = 0; j < n; ++j) {
                const uint32_t fb = sflags[(j << 7) + tid];
                const int h = __ldg(hk + j), pv = __ldg(pk + j);
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    if ((fb >> b) & 1u) {
                        mh[b] = min(mh[b], h);
                        S[b] += pv;
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < K; ++b) {
                int32_t *Ab = sA + (k * K + b) * kThreads + tid;
                const int C = *Ab;
                *Ab = (mh[b] == INT_MAX ? C : max(C, mh[b])) + S[b];
            }
        }

        // ---- 4/5. couples, tile by tile
        int lb[K], q[K];
#pragma unroll
        for (int b = 0; b < K; ++b) {
            lb[b] = 0;
            q[b] = 0;
        }
        for (int t = 0; t < a.ntiles; ++t) {
            const uint32_t f = resident ? (uint32_t)t : fill;
            if (!resident && tid == 0) {
                const bool has_next = (t + 1 < a.ntiles) || (nt + gridDim.x < a.num_node_tiles);
                if (has_next) issue(fill + 1, (t + 1) % a.ntiles);
            }
            const uint32_t parity = resident ? 0u : ((fill >> 1) & 1u);
            const bool ok = mbar_wait_bounded(&bar[f & 1], parity, a.wait_limit);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) {
                    report_status(a.status, (int32_t)FSP_ETIMEDOUT);
                    // let copies already issued land before the block exits
                    for (uint32_t bi = 0; bi < 2; ++bi)
                        if ((pending >> bi) & 1u) mbar_wait_bounded(&bar[bi], (pend_par >> bi) & 1u, a.wait_limit);
                }
                return;
            }
            pending &= ~(1u << (f & 1));
            const unsigned char *tb = tiles + (f & 1) * a.tile_stride;
            const int c0 = t * a.ppt;
            const int np = min(a.ppt, a.P - c0);
            for (int cc = 0; cc < np; ++cc) {
                const int c = c0 + cc;
                const int k = spairs[2 * c], l = spairs[2 * c + 1];
                if (k == 0) {
                    // first couple of machine l: latency q_l (QM) and A_l + q_l
#pragma unroll
                    for (int b = 0; b < K; ++b) q[b] = INT_MAX;
                    const int32_t *tl = a.tail + l * n;
                    for (int j = 0; j < n; ++j) {
                        const uint32_t fb = sflags[(j << 7) + tid];
                        const int tv = __ldg(tl + j);
#pragma unroll
                        for (int b = 0; b < K; ++b)
                            if ((fb >> b) & 1u) q[b] = min(q[b], tv);
                    }
#pragma unroll
                    for (int b = 0; b < K; ++b) {
                        if (q[b] == INT_MAX) q[b] = 0;
                        lb[b] = max(lb[b], sA[(l * K + b) * kThreads + tid] + q[b]);
                    }
                }
                int u[K];
#pragma unroll
                for (int b = 0; b < K; ++b) u[b] = 0;
                if (!WIDE) {
                    const uint4 *R = reinterpret_cast<const uint4 *>(tb + (size_t)cc * a.npad * 4);
                    const int nq = a.npad >> 2;
#pragma unroll 1
                    for (int i = 0; i < nq; ++i) {
                        const uint4 r4 = R[i];
                        const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const uint32_t r = rr[e];
                            johnson_step<K>((int)(r & 1023u), (int)((r >> 10) & 8191u), (int)r >> 23, sflags, tid, u);
                        }
                    }
                } else {
                    const int4 *R = reinterpret_cast<const int4 *>(tb + (size_t)cc * a.npad * 16);
#pragma unroll 1
                    for (int i = 0; i < a.npad; ++i) {
                        const int4 r = R[i];
                        johnson_step<K>(r.x, r.y, r.z, sflags, tid, u);
                    }
                }
#pragma unroll
                for (int b = 0; b < K; ++b) lb[b] = max(lb[b], sA[(k * K + b) * kThreads + tid] + q[b] + u[b]);
            }
            if (!resident) {
                __syncthreads();  // every thread is done with this buffer
                ++fill;
            }
        }

        // ---- 6. results
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const int64_t x = base + b * kThreads + tid;
            if (x < a.N) a.out[x] = ((vmask >> b) & 1u) ? lb[b] : FSP_LB_INVALID;
        }
    }
}

// ---------------------------------------------------------------- host side
namespace {

struct DeviceLimits {
    int smem_optin = 0;  // per block, opt-in maximum
    int smem_sm = 0;     // per SM
    int num_sms = 0;
};

DeviceLimits device_limits(int dev) {
    static std::mutex mu;
    static DeviceLimits cache[64];
    static bool have[64] = {};
    std::lock_guard<std::mutex> g(mu);
    if (dev >= 0 && dev < 64 && have[dev]) return cache[dev];
    DeviceLimits d;
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&d.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64 && d.num_sms > 0) {
        cache[dev] = d;
        have[dev] = true;
    }
    return d;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    uint32_t off_tiles, tile_stride, off_A, off_flags;
    size_t total;
};

Layout layout_for(const fsp_instance *inst, int K, int ppt) {
    Layout L;
    L.off_tiles = (uint32_t)align_up(16 + 2 * (size_t)inst->P, 128);
    L.tile_stride = (uint32_t)align_up((size_t)ppt * inst->npad * inst->rec_bytes, 128);
    L.off_A = L.off_tiles + 2 * L.tile_stride;
    L.off_flags = (uint32_t)align_up(L.off_A + (size_t)inst->m * K * kThreads * 4, 128);
    L.total = align_up(L.off_flags + (size_t)inst->n * kThreads, 128);
    return L;
}

// Shared-memory budget of one block when `bps` blocks share an SM.
size_t block_budget(const DeviceLimits &d, int bps) {
    const size_t per_block = bps <= 1 ? (size_t)d.smem_optin : (size_t)d.smem_sm / bps - 1024;
    return std::min(per_block, (size_t)d.smem_optin);
}

// Largest couple tile that fits; 0 if nothing fits.
int max_ppt(const fsp_instance *inst, int K, int bps, const DeviceLimits &d) {
    const size_t budget = block_budget(d, bps);
    const Layout L0 = layout_for(inst, K, 0);
    if (L0.total > budget) return 0;
    const size_t per_pair = (size_t)inst->npad * inst->rec_bytes;
    size_t ppt = (budget - L0.total) / (2 * per_pair + 1);
    while (ppt > 0 && layout_for(inst, K, (int)ppt).total > budget) --ppt;
    return (int)std::min<size_t>(ppt, (size_t)inst->P);
}

// Relative per-node efficiency of K nodes per thread (instruction overhead
// of a Johnson record is shared by the K nodes).
double k_efficiency(int K) {
    switch (K) {
        case 8: return 1.0;
        case 4: return 0.85;
        case 2: return 0.65;
        default: return 0.45;
    }
}

double wave_efficiency(double work_items, double slots) {
    const double waves = work_items / slots;
    return waves / std::ceil(waves);
}

fsp_status resolve_lockstep(const fsp_instance *inst, int64_t N, const DeviceLimits &d, fsp_launch_config &c) {
    if (c.nodes_per_thread && c.nodes_per_thread != 1 && c.nodes_per_thread != 2 && c.nodes_per_thread != 4 &&
        c.nodes_per_thread != 8)
        return FSP_EINVAL;
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 2 || c.pairs_per_tile < 0) return FSP_EINVAL;
    if (!c.nodes_per_thread || !c.blocks_per_sm) {
        double best = -1.0;
        int bK = 0, bB = 0;
        for (int K : {8, 4, 2, 1}) {
            if (c.nodes_per_thread && c.nodes_per_thread != K) continue;
            for (int bps : {1, 2}) {
                if (c.blocks_per_sm && c.blocks_per_sm != bps) continue;
                const int ppt = max_ppt(inst, K, bps, d);
                if (ppt < 1) continue;
                const bool res = (ppt * 2 >= inst->P);
                const double tiles = std::ceil((double)std::max<int64_t>(N, 1) / (K * kThreads));
                const double score = k_efficiency(K) * wave_efficiency(tiles, (double)d.num_sms * bps) *
                                     (bps == 2 ? 1.08 : 1.0) * (res ? 1.0 : 0.97);
                if (score > best) {
                    best = score;
                    bK = K;
                    bB = bps;
                }
            }
        }
        if (best < 0) return FSP_EINVAL;
        c.nodes_per_thread = bK;
        c.blocks_per_sm = bB;
    }
    const int mp = max_ppt(inst, c.nodes_per_thread, c.blocks_per_sm, d);
    if (mp < 1) return FSP_EINVAL;
    if (!c.pairs_per_tile) c.pairs_per_tile = (mp * 2 >= inst->P) ? std::max(1, (inst->P + 1) / 2) : mp;
    if (c.pairs_per_tile > mp) return FSP_EINVAL;
    return FSP_OK;
}

fsp_status resolve_lanes(const fsp_instance *inst, int64_t N, const DeviceLimits &d, fsp_launch_config &c) {
    if (c.warps_per_block < 0 || c.warps_per_block > 16 || c.positions_per_tile < 0 ||
        (c.positions_per_tile & 3) || c.staging < 0 || c.staging > 5 || c.blocks_per_sm < 0 ||
        c.blocks_per_sm > (c.staging == FSP_STAGING_GLOBAL ? 16 : 8) || c.pairs_per_tile < 0 || c.tail_slices < 0)
        return FSP_EINVAL;
    const int G = inst->G;
    // nodes per warp (nodes_per_thread for this kernel): 32, or 28 and 56 in
    // one and two sets of 28 (streamed staging, compact records)
    const int npw = lanes_nodes_per_warp(c);
    if (!npw) return FSP_EINVAL;
    if (npw != 32 && ((c.staging && c.staging != FSP_STAGING_STREAMED) || !inst->compact || c.tail_slices > 1))
        return FSP_EINVAL;
    const bool npw_free = c.nodes_per_thread == 0;
    c.nodes_per_thread = npw;
    // Default shape of a pool of a few thousand work items (32-node batches x
    // couple groups) for instances of at least four couple groups: split
    // staging (the setups in a prep kernel of their own, the scan in work
    // items of one couple group, two above 4,096 items), in the shapes the
    // autotuner picks at 200x20: 6 warps x 2 blocks per SM below 1,024 items
    // (4,096 nodes: 0.18 of the ALU peak against 0.16 with two 28-node sets
    // per warp), 12 warps x 1 up to 2,048 (8,192 nodes: 0.30 against 0.26
    // with global staging), 8 warps x 2 up to 8,192 (16,384 and 32,768
    // nodes: 0.43 and 0.55 against 0.38 and 0.49).
    if (!c.staging && !c.warps_per_block && !c.blocks_per_sm && !c.pairs_per_tile && !c.positions_per_tile &&
        c.tail_slices <= 1 && npw == 32 && inst->compact && G >= 4) {
        const int64_t items = (std::max<int64_t>(N, 1) + 31) / 32 * G;
        if (items >= 768 && items <= 8192) {
            fsp_launch_config t = c;
            t.staging = FSP_STAGING_SPLIT;
            t.warps_per_block = items < 1024 ? 6 : items <= 2048 ? 12 : 8;
            t.blocks_per_sm = t.warps_per_block == 12 ? 1 : 2;
            t.pairs_per_tile = items > 4096 ? 64 : 32;
            // only where a tile of 64 positions (or all of them) fits: the
            // tile chosen below is at least that large, else the pool keeps
            // the shape chosen further down
            t.positions_per_tile = std::min(inst->npad, 64) & ~3;
            size_t smem = 0;
            if (lanes_layout(inst, t, &smem) == FSP_OK) {
                c.staging = t.staging;
                c.warps_per_block = t.warps_per_block;
                c.blocks_per_sm = t.blocks_per_sm;
                c.pairs_per_tile = t.pairs_per_tile;
            }
        }
    }
    if (c.staging == FSP_STAGING_GLOBAL) {
        // Warps independent, records from L2/L1: every work item (a 32-node
        // batch and a slice of the couples) gets a warp of its own when the
        // pool is small.  Defaults: 4 warps per block, as many blocks per SM
        // as make 16 warps, and couple slices enough to give the grid's warps
        // an item each (at most G).
        if (!inst->compact || c.tail_slices > 1 || c.positions_per_tile) return FSP_EINVAL;
        if (!c.warps_per_block) c.warps_per_block = c.blocks_per_sm ? std::max(1, 16 / c.blocks_per_sm) : 4;
        if (!c.blocks_per_sm) c.blocks_per_sm = std::max(1, 16 / c.warps_per_block);
        if (c.warps_per_block * c.blocks_per_sm > 16) return FSP_EINVAL;
        int gper = lanes_groups_per_item(inst, c.pairs_per_tile);
        if (!c.pairs_per_tile) {
            const int64_t batches = (std::max<int64_t>(N, 1) + 31) / 32;
            const int64_t warps = (int64_t)d.num_sms * c.warps_per_block * c.blocks_per_sm;
            const int64_t S = std::min<int64_t>(G, std::max<int64_t>(1, (warps + batches - 1) / batches));
            gper = (int)((G + S - 1) / S);
        }
        c.pairs_per_tile = gper >= G ? inst->P : gper * 32;
        c.tail_slices = 1;
        c.positions_per_tile = 0;
        size_t smem = 0;
        return lanes_layout(inst, c, &smem);
    }
    // pairs per work item: only streamed staging splits a batch by couples
    const int req_g = lanes_groups_per_item(inst, c.pairs_per_tile);
    auto resolved_ppt = [&](int gper) { return gper >= G ? inst->P : gper * 32; };
    // blocks per SM: chosen with the warps when neither is given, else 1
    const bool bps_free = !c.blocks_per_sm && !c.warps_per_block;
    if (!c.blocks_per_sm) c.blocks_per_sm = 1;
    const int npad = inst->npad;
    auto fits = [&](int W, int staging, int pos) {
        fsp_launch_config t = c;
        t.warps_per_block = W;
        t.staging = staging;
        t.positions_per_tile = pos;
        size_t smem = 0;
        return lanes_layout(inst, t, &smem) == FSP_OK;
    };
    // tiled modes: streamed (block-wide tile pipeline), split (prep + scan
    // kernels) or warp (a tile pipeline per warp)
    const int tiled = (c.staging == FSP_STAGING_SPLIT || c.staging == FSP_STAGING_WARP) ? c.staging
                                                                                        : FSP_STAGING_STREAMED;
    // record tile for W warps: the largest multiple of 4 up to min(npad, 96)
    // that fits (larger tiles leave less L1 to the setup's tables: at 200x20,
    // 8 warps x 2 blocks, 96 positions 0.99 ms, 128 positions 1.05 ms for
    // 209,716 nodes), else the largest that fits at all; 0 if none
    auto best_chunk = [&](int W) {
        for (int ch = std::min(npad, 96) & ~3; ch >= 4; ch -= 4)
            if (fits(W, tiled, ch)) return ch;
        for (int ch = npad; ch > 96; ch -= 4)
            if (fits(W, tiled, ch)) return ch;
        return 0;
    };
    // resident staging only on request: holding every record in shared memory
    // leaves too little L1 for the setup's tables (measured slower at 20x20
    // and 200x20), so the default streams the records
    if (c.staging == FSP_STAGING_RESIDENT) {
        int bW = 0;
        for (int W = 16; W >= 1; --W) {
            if (c.warps_per_block && c.warps_per_block != W) continue;
            if (fits(W, FSP_STAGING_RESIDENT, 0)) {
                bW = W;
                break;
            }
        }
        if (bW && req_g == G && c.tail_slices <= 1) {
            c.warps_per_block = bW;
            c.staging = FSP_STAGING_RESIDENT;
            c.positions_per_tile = 0;
            c.blocks_per_sm = 1;
            c.pairs_per_tile = inst->P;
            c.tail_slices = 1;
            return FSP_OK;
        }
        return FSP_EINVAL;
    }
    c.staging = tiled;
    // couple slices: streamed and split staging; tail slices: streamed only
    if (tiled == FSP_STAGING_WARP && req_g != G) return FSP_EINVAL;
    if (tiled != FSP_STAGING_STREAMED && c.tail_slices > 1) return FSP_EINVAL;
    // Launch model for the defaults: a wave of work items (block batches of
    // 32 W nodes, times S couple slices of gper groups each) takes about
    // max(warps per SM, 16) x (setup + gper / G of a full scan), the setup
    // costing about a fifth of a full scan; slicing by couples pays for its
    // repeated setup only when the batches leave SMs idle.  One block per SM
    // runs about 1.2x slower per warp than two (at 200x20: 14 warps x 1 block
    // 1.30 ms, 8 warps x 2 blocks 1.08 ms), whose barriers and setups fall
    // out of phase.
    // Streamed staging with whole batches may slice the last partial wave's
    // batches (tail_slices, on request or from the tuner; the model below
    // takes it into account when requested).
    const bool tail_ok = tiled == FSP_STAGING_STREAMED && c.tail_slices > 1;
    auto tail_for = [&](int64_t batches, int64_t slots) -> int {
        const int64_t r = batches % slots;
        if (batches <= slots || r == 0) return 1;
        return std::min(G, c.tail_slices);
    };
    auto model_time = [&](int W, int gper) {
        const int64_t slots = (int64_t)d.num_sms * c.blocks_per_sm;
        const int64_t batches = (std::max<int64_t>(N, 1) + (int64_t)npw * W - 1) / ((int64_t)npw * W);
        const double occ = std::max(W * c.blocks_per_sm, 16) * (c.blocks_per_sm == 1 ? 1.2 : 1.0);
        if (gper < G) {
            const double items = (double)batches * std::ceil((double)G / gper);
            return std::ceil(items / (double)slots) * occ * (0.2 + (double)gper / G);
        }
        const int st = tail_ok ? tail_for(batches, slots) : 1;
        const int64_t full_waves = st > 1 ? batches / slots : (batches + slots - 1) / slots;
        const double tail = st > 1 ? 0.2 + std::ceil((double)G / st) / G : 0.0;
        return ((double)full_waves * 1.2 + tail) * occ;
    };
    auto best_gper = [&](int W, double *t) {
        int bg = req_g;
        double bt = model_time(W, req_g);
        if (!c.pairs_per_tile && tiled == FSP_STAGING_STREAMED && c.tail_slices <= 1)
            for (int g = G - 1; g >= 1; --g) {
                const double tg = model_time(W, g);
                if (tg < bt * (1.0 - 1e-9)) {
                    bt = tg;
                    bg = g;
                }
            }
        if (t) *t = bt;
        return bg;
    };
    if (!c.warps_per_block) {
        double best = -1.0;
        int bW = 0, bB = c.blocks_per_sm;
        const int bps_lo = c.blocks_per_sm, bps_hi = bps_free ? 2 : c.blocks_per_sm;
        for (int bps = bps_hi; bps >= bps_lo; --bps) {
            c.blocks_per_sm = bps;
            for (int W = 16 / bps; W >= 1; --W) {
                // even warp counts above 2 (odd ones measured slower: 7 x 2
                // blocks 1.29 ms, 8 x 2 1.08 ms at 200x20)
                if (W > 2 && (W & 1)) continue;
                const int ch = c.positions_per_tile ? c.positions_per_tile : best_chunk(W);
                if (ch < 4 || !fits(W, tiled, ch)) continue;
                if (!c.positions_per_tile && ch < std::min(npad, 64)) continue;
                double t = 0.0;
                best_gper(W, &t);
                const double score = 1.0 / t;
                // on a tie the smaller block wins: its items spread over more SMs
                if (score >= best * (1.0 - 1e-9)) {
                    best = score;
                    bW = W;
                    bB = bps;
                }
            }
        }
        if (best < 0) return FSP_EINVAL;
        c.warps_per_block = bW;
        c.blocks_per_sm = bB;
    }
    const int gper = best_gper(c.warps_per_block, nullptr);
    c.pairs_per_tile = resolved_ppt(gper);
    if (gper < G) {
        if (c.tail_slices > 1) return FSP_EINVAL;  // already split throughout
        c.tail_slices = 1;
    } else if (tiled != FSP_STAGING_STREAMED) {
        c.tail_slices = 1;
    } else if (c.tail_slices == 0) {
        // none by default: slicing the last wave measured 5-15% faster for
        // some pool sizes and up to 10% slower for others (at 200x20, 262,144
        // nodes: 1.08 ms whole, 1.20 ms in two slices -- the last wave holds
        // the deepest nodes, whose setups the slices repeat), so the tuner
        // decides
        c.tail_slices = 1;
    }
    if (!c.positions_per_tile) c.positions_per_tile = best_chunk(c.warps_per_block);
    if (c.positions_per_tile < 4) return FSP_EINVAL;
    // Pools of under two and a half waves of 32-node block batches take 28
    // nodes per warp by default (long scans of many couple groups): at 200x20
    // the autotuner picks 28 from 16,384 to 131,072 nodes (131,072: 0.77 of the
    // ALU peak against 0.69 with 32; the batches fill the waves better) and 32
    // at 262,144 (3.4 waves).
    if (npw_free && tiled == FSP_STAGING_STREAMED && inst->compact && G >= 4 && npad >= 64 &&
        c.tail_slices <= 1) {
        const int64_t slots = (int64_t)d.num_sms * c.blocks_per_sm;
        const int64_t b32 = (std::max<int64_t>(N, 1) + 32 * c.warps_per_block - 1) / (32 * c.warps_per_block);
        if (b32 * 2 < slots * 5) {
            fsp_launch_config t = c;
            t.nodes_per_thread = 28;
            size_t smem = 0;
            if (lanes_layout(inst, t, &smem) == FSP_OK) c.nodes_per_thread = 28;
        }
    }
    return fits(c.warps_per_block, tiled, c.positions_per_tile) ? FSP_OK : FSP_EINVAL;
}

}  // namespace

int max_smem_per_block(int device) { return device_limits(device).smem_optin; }
int max_smem_per_sm(int device) { return device_limits(device).smem_sm; }
int num_sms(int device) { return device_limits(device).num_sms; }

fsp_status check_device(const fsp_instance *inst) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    return dev == inst->device ? FSP_OK : FSP_EINVAL;
}

fsp_status take_device_status(const fsp_instance *inst) {
    if (!inst->host_status) return FSP_OK;
    volatile int32_t *hs = inst->host_status;
    const int32_t v = *hs;
    if (v != 0) {
        *hs = 0;
        return (fsp_status)v;
    }
    return FSP_OK;
}

fsp_status resolve_config(const fsp_instance *inst, int64_t N, const fsp_launch_config *req,
                          fsp_launch_config *out, size_t *smem_bytes) {
    const DeviceLimits d = device_limits(inst->device);
    if (d.num_sms <= 0 || d.smem_optin <= 0) return FSP_ECUDA;
    fsp_launch_config c = {};
    if (req) c = *req;
    if (c.kernel < 0 || c.kernel > 2) return FSP_EINVAL;
    const bool unset = c.kernel == 0 && !c.nodes_per_thread && !c.blocks_per_sm && !c.pairs_per_tile &&
                       !c.warps_per_block && !c.positions_per_tile && !c.staging && !c.tail_slices;
    if (unset) {
        std::lock_guard<std::mutex> g(inst->mu);
        for (auto &e : inst->tuned)
            if (e.first == N) c = e.second;
    }
    // per-job release times are computed by the couple-lanes setup only
    const bool per_job = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) != 0;
    if (per_job && c.kernel == FSP_KERNEL_LOCKSTEP) return FSP_EINVAL;
    if (c.kernel == 0) c.kernel = (inst->P >= 32 || per_job) ? FSP_KERNEL_LANES : FSP_KERNEL_LOCKSTEP;
    fsp_status st = c.kernel == FSP_KERNEL_LANES ? resolve_lanes(inst, N, d, c) : resolve_lockstep(inst, N, d, c);
    if (st != FSP_OK) return st;
    if (c.kernel == FSP_KERNEL_LANES) {
        st = lanes_layout(inst, c, smem_bytes);
        if (st != FSP_OK) return st;
    } else {
        *smem_bytes = layout_for(inst, c.nodes_per_thread, c.pairs_per_tile).total;
    }
    *out = c;
    return FSP_OK;
}

namespace {

template <int K, bool WIDE>
cudaError_t launch_variant(const BoundArgs &a, int grid, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        attr_err = cudaFuncSetAttribute(fsp_bound_kernel<K, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    });
    if (attr_err != cudaSuccess) return attr_err;
    fsp_bound_kernel<K, WIDE><<<grid, kThreads, smem, s>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

fsp_status launch_lockstep(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                           int32_t *out_lb, void *stream, const fsp_launch_config &c) {
    const DeviceLimits d = device_limits(inst->device);
    const int K = c.nodes_per_thread;
    BoundArgs a;
    a.rec = static_cast<const unsigned char *>(inst->t.rec);
    a.pairs = inst->t.pairs;
    a.p = inst->t.p;
    a.head = inst->t.head;
    a.tail = inst->t.tail;
    a.ptm = inst->t.ptm;
    a.nodes = nodes;
    a.depths = depths;
    a.out = out_lb;
    a.status = inst->dev_status;
    a.N = N;
    a.num_node_tiles = (N + (int64_t)K * kThreads - 1) / ((int64_t)K * kThreads);
    a.n = inst->n;
    a.m = inst->m;
    a.P = inst->P;
    a.npad = inst->npad;
    a.ppt = c.pairs_per_tile;
    a.ntiles = (inst->P + c.pairs_per_tile - 1) / c.pairs_per_tile;
    a.rec_bytes = (uint32_t)inst->rec_bytes;
    const Layout L = layout_for(inst, K, c.pairs_per_tile);
    a.off_tiles = L.off_tiles;
    a.tile_stride = L.tile_stride;
    a.off_A = L.off_A;
    a.off_flags = L.off_flags;
    a.wait_limit = 4000000000LL;  // about two seconds at 2 GHz
    const int64_t slots = (int64_t)d.num_sms * c.blocks_per_sm;
    const int grid = (int)std::min<int64_t>(a.num_node_tiles, slots);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool wide = !inst->compact;
    switch (K * 2 + (wide ? 1 : 0)) {
        case 16: e = launch_variant<8, false>(a, grid, L.total, s); break;
        case 17: e = launch_variant<8, true>(a, grid, L.total, s); break;
        case 8: e = launch_variant<4, false>(a, grid, L.total, s); break;
        case 9: e = launch_variant<4, true>(a, grid, L.total, s); break;
        case 4: e = launch_variant<2, false>(a, grid, L.total, s); break;
        case 5: e = launch_variant<2, true>(a, grid, L.total, s); break;
        case 2: e = launch_variant<1, false>(a, grid, L.total, s); break;
        default: e = launch_variant<1, true>(a, grid, L.total, s); break;
    }
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}

}  // namespace

fsp_status launch_bound(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                        int32_t *out_lb, void *stream, const fsp_launch_config *cfg) {
    fsp_launch_config c;
    size_t smem = 0;
    fsp_status st = resolve_config(inst, N, cfg, &c, &smem);
    if (st != FSP_OK) return st;
    if (c.kernel == FSP_KERNEL_LANES) return launch_lanes(inst, nodes, depths, N, out_lb, stream, c);
    return launch_lockstep(inst, nodes, depths, N, out_lb, stream, c);
}

}  // namespace fspgb

using namespace fspgb;

extern "C" fsp_status fsp_bound_pool_ex(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                                        int64_t N, int32_t *out_lb, void *cuda_stream,
                                        const fsp_launch_config *cfg) {
    if (!inst || N < 0) return FSP_EINVAL;
    if (N > 0 && (!nodes || !depths || !out_lb)) return FSP_EINVAL;
    fsp_status st = take_device_status(inst);
    if (st != FSP_OK) return st;
    st = check_device(inst);
    if (st != FSP_OK) return st;
    if (N == 0) return FSP_OK;
    return launch_bound(inst, nodes, depths, N, out_lb, cuda_stream, cfg);
}

extern "C" fsp_status fsp_bound_pool(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                                     int64_t N, int32_t *out_lb, void *cuda_stream) {
    return fsp_bound_pool_ex(inst, nodes, depths, N, out_lb, cuda_stream, nullptr);
}

extern "C" fsp_status fsp_bound_pool_host(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths,
                                          int64_t N, int32_t *out_lb, void *cuda_stream) {
    if (!inst || N < 0) return FSP_EINVAL;
    if (N > 0 && (!nodes || !depths || !out_lb)) return FSP_EINVAL;
    fsp_status st = take_device_status(inst);
    if (st != FSP_OK) return st;
    st = check_device(inst);
    if (st != FSP_OK) return st;
    if (N == 0) return FSP_OK;
    cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
    const int n = inst->n;

    // Staged through device memory in chunks: the copies go back to back on
    // a copy stream, each chunk's bounding waits only for its own copy, and
    // consecutive chunks are bounded on two streams, so one chunk's last wave
    // overlaps the next chunk's first.  Every chunk is bounded with the launch
    // shape tuned for the whole pool when the caller tuned one (the chunks'
    // own sizes have none), else with the default shape of the pool.
    fsp_launch_config shape = {};
    bool have_tuned = false;
    {
        std::lock_guard<std::mutex> g(inst->mu);
        for (auto &e : inst->tuned)
            if (e.first == N) {
                shape = e.second;
                have_tuned = true;
            }
    }
    if (!have_tuned) {
        size_t smem = 0;
        st = resolve_config(inst, N, nullptr, &shape, &smem);
        if (st != FSP_OK) return st;
    }
    // Chunk ends.  With the couple-lanes streamed shape, a first chunk of two
    // thirds of a wave of block batches (bounding starts after a short copy),
    // then whole waves, so that every launch but the last fills the grid; the
    // copies (about 2 ns per 200-job node at 207 GB/s here, against about
    // 4 ns of bounding) stay ahead.  At 200x20: 1.32 ms per 262,144-node
    // pool, against 1.56 ms for a 20/80 split and 1.64 ms for one chunk.
    // Pools under two waves, or other shapes: 20/80 from 32,768 nodes.
    constexpr int kMaxChunks = 8;
    int64_t ends[kMaxChunks + 1] = {0};
    int nchunks = 1;
    ends[1] = N;
    const int64_t wave = (shape.kernel == FSP_KERNEL_LANES && shape.staging == FSP_STAGING_STREAMED)
                             ? (int64_t)num_sms(inst->device) * std::max(1, shape.blocks_per_sm) * 32 *
                                   shape.warps_per_block
                             : 0;
    if (wave > 0 && N >= 2 * wave) {
        const int64_t first = wave * 2 / 3;
        // whole waves per chunk, enough of them to stay within kMaxChunks
        const int64_t rest_waves = (N - first + wave - 1) / wave;
        const int64_t step = (rest_waves + kMaxChunks - 2) / (kMaxChunks - 1) * wave;
        ends[1] = first;
        while (ends[nchunks] < N) {
            ends[nchunks + 1] = std::min(N, ends[nchunks] + step);
            ++nchunks;
        }
    } else if (N >= 32768) {
        nchunks = 2;
        ends[1] = N / 5;
        ends[2] = N;
    }
    std::lock_guard<std::mutex> host_lock(inst->host_mu);
    cudaStream_t &cpy = inst->host_streams[0], &comp2 = inst->host_streams[1];
    cudaEvent_t &ev_start = inst->host_events[0], &ev_done = inst->host_events[1];
    cudaEvent_t *ev_in = inst->host_events + 2;
    int16_t *d_nodes = nullptr;
    int32_t *d_depths = nullptr, *d_out = nullptr;
    const size_t nodes_bytes = sizeof(int16_t) * (size_t)N * n;
    cudaMemPool_t pool = nullptr;
    st = scratch_pool(inst->device, &pool);
    if (st != FSP_OK) return st;
    for (int i = 0; st == FSP_OK && i < 2; ++i)
        if (!inst->host_streams[i] && cudaStreamCreateWithFlags(&inst->host_streams[i], cudaStreamNonBlocking) != cudaSuccess)
            st = FSP_ECUDA;
    for (int i = 0; st == FSP_OK && i < 2 + kMaxChunks; ++i)
        if (!inst->host_events[i] && cudaEventCreateWithFlags(&inst->host_events[i], cudaEventDisableTiming) != cudaSuccess)
            st = FSP_ECUDA;
    if (st == FSP_OK &&
        (cudaMallocFromPoolAsync((void **)&d_nodes, nodes_bytes, pool, user) != cudaSuccess ||
         cudaMallocFromPoolAsync((void **)&d_depths, sizeof(int32_t) * (size_t)N, pool, user) != cudaSuccess ||
         cudaMallocFromPoolAsync((void **)&d_out, sizeof(int32_t) * (size_t)N, pool, user) != cudaSuccess)) {
        cudaGetLastError();
        st = FSP_ENOMEM;
    }
    if (st == FSP_OK) {
        cudaEventRecord(ev_start, user);  // the staging memory is ready on the caller's stream
        cudaStreamWaitEvent(cpy, ev_start, 0);
        cudaStreamWaitEvent(comp2, ev_start, 0);
        for (int64_t c = 0; c < nchunks && st == FSP_OK; ++c) {
            const int64_t lo = ends[c], hi = ends[c + 1];
            if (lo >= hi) break;
            const size_t rows = (size_t)(hi - lo);
            if (cudaMemcpyAsync(d_nodes + lo * n, nodes + lo * n, sizeof(int16_t) * rows * n, cudaMemcpyHostToDevice,
                                cpy) != cudaSuccess ||
                cudaMemcpyAsync(d_depths + lo, depths + lo, sizeof(int32_t) * rows, cudaMemcpyHostToDevice, cpy) !=
                    cudaSuccess ||
                cudaEventRecord(ev_in[c], cpy) != cudaSuccess) {
                st = FSP_ECUDA;
                break;
            }
            cudaStream_t s = (c & 1) ? comp2 : user;
            cudaStreamWaitEvent(s, ev_in[c], 0);
            st = launch_bound(inst, d_nodes + lo * n, d_depths + lo, hi - lo, d_out + lo, s, &shape);
            if (st != FSP_OK) break;
            if (cudaMemcpyAsync(out_lb + lo, d_out + lo, sizeof(int32_t) * rows, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                st = FSP_ECUDA;
        }
        // the caller's stream waits for both other streams (copies and chunks)
        cudaEventRecord(ev_done, comp2);
        cudaStreamWaitEvent(user, ev_done, 0);
        cudaEventRecord(ev_done, cpy);
        cudaStreamWaitEvent(user, ev_done, 0);
    }
    if (d_nodes) cudaFreeAsync(d_nodes, user);
    if (d_depths) cudaFreeAsync(d_depths, user);
    if (d_out) cudaFreeAsync(d_out, user);
    if (cudaStreamSynchronize(user) != cudaSuccess && st == FSP_OK) st = FSP_ECUDA;
    if (st == FSP_OK) st = take_device_status(inst);
    return st;
}

// ---------------------------------------------------------------------------
// Self-check of the device-side bounded waits.  Every wait of the bounding
// kernels (tile copies, prepared-state copies, the per-warp rings) gives up
// after a clock64 limit, reports FSP_ETIMEDOUT in the instance's status word
// and returns, so a lost completion never hangs the GPU.  This kernel runs
// the same wait on an mbarrier phase that nothing ever completes.
namespace fspgb {

__global__ void fsp_wait_probe(int32_t *status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit);  // no thread ever arrives
    if (!__syncthreads_and(ok) && threadIdx.x == 0) report_status(status, (int32_t)FSP_ETIMEDOUT);
}

}  // namespace fspgb

extern "C" fsp_status fsp_check_wait_timeout(const fsp_instance *inst, int64_t limit_cycles) {
    if (!inst || limit_cycles < 1 || limit_cycles > (int64_t)1 << 32) return FSP_EINVAL;
    fsp_status st = fspgb::check_device(inst);
    if (st != FSP_OK) return st;
    st = fspgb::take_device_status(inst);
    if (st != FSP_OK) return st;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FSP_ECUDA;
    fspgb::note_launches(1);
    fspgb::fsp_wait_probe<<<1, 64, 0, s>>>(inst->dev_status, (long long)limit_cycles);
    const bool launched = cudaGetLastError() == cudaSuccess;
    const bool done = cudaStreamSynchronize(s) == cudaSuccess;
    cudaStreamDestroy(s);
    if (!launched || !done) return FSP_ECUDA;
    return fspgb::take_device_status(inst);
}
