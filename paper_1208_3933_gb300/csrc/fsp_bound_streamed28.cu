// fsp_bound_streamed28.cu -- the streamed couple-lanes bound with one or two
// sets of 28 nodes per warp (sm_103a).  The host side (layout, launch shape,
// depth order) is in fsp_bound_lanes.cu; this file holds the kernel and its
// launcher so that the library's translation units compile in parallel.
#include <cuda_runtime.h>

#include <mutex>

#include "fsp_internal.h"
#include "fsp_lanes_device.cuh"
#include "fsp_ptx.cuh"

namespace fspgb {

// The streamed kernel with NS node sets of 28 per warp (NS = 1 or 2, compact
// records): a block batch is 28 NS W nodes; each flag word yields its 28
// predicates from four byte-wise conversions (bits 7, 15, 23 and 31 unused),
// and with two sets every record read serves 56 nodes.  A warp sets up its
// sets one after the other (lane = node, lanes 7, 15, 23 and 31 idle), and
// the couple values of each group are reduced over the lanes at once, so no
// per-node maxima are carried across groups.
template <int MP, int NS>
__global__ void __launch_bounds__(512, 1) fsp_lanes_streamed28(const LanesArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint8_t *sgp = smem + 16;
    int2 *hcache = reinterpret_cast<int2 *>(smem + a.off_cache);
    int2 *tcache = hcache + a.m * 32;
    const int nfw = flag_words(a.n);
    uint32_t *F0 = reinterpret_cast<uint32_t *>(smem + a.off_flags) + (size_t)warp * NS * nfw;
    uint32_t *F1 = F0 + (NS - 1) * nfw;
    int32_t *AQ0 = reinterpret_cast<int32_t *>(smem + a.off_aq) + (size_t)warp * NS * 32 * a.aq_stride;
    int32_t *AQ1 = AQ0 + (NS - 1) * 32 * a.aq_stride;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    for (int i = threadIdx.x; i < a.G * 64; i += blockDim.x) sgp[i] = a.gpairs[i];
    load_sorted_heads(a, hcache, tcache);
    __syncthreads();

    TilePipe tp{bar, smem + a.off_tables, a.tile_stride, a.ntiles <= 2};
    auto tile_issue = [&](uint32_t fill, int t) {
        const int g = t / a.nchunks, ch = t - g * a.nchunks;
        const int pos = min(a.chunk, a.npad - ch * a.chunk);
        const unsigned char *src = a.grec + ((size_t)g * a.npad + (size_t)ch * a.chunk) * 32 * a.rec_bytes;
        tp.issue(fill, src, (uint32_t)pos * 32u * a.rec_bytes);
    };
    // work items as in fsp_lanes_streamed, block batches of 28 NS W nodes
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
    // lane -> node of each set: lanes 7, 15, 23, 31 hold no node
    const bool real = (kSet28 >> lane) & 1u;
    const int r28 = set28_slot(lane);

    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int sl = slice_of(it);
        const int64_t bt = sl < 0 ? it : full + (int64_t)((uint32_t)(it - full) / S);
        const int64_t base = bt * (int64_t)(28 * NS * W) + warp * 28 * NS;
        const int64_t x0 = real ? node_at(a, base + r28) : a.N;
        const int64_t x1 = (NS == 2 && real) ? node_at(a, base + 28 + r28) : a.N;
        bool valid0 = false, valid1 = false;
        int bterm0 = 0, bterm1 = 0;
#pragma unroll 1
        for (int set = 0; set < NS; ++set) {
            int bt_ = 0;
            const bool v = lanes_setup<MP>(a, set ? x1 : x0, lane, set ? F1 : F0,
                                           (set ? AQ1 : AQ0) + lane * a.aq_stride, bt_, hcache, tcache);
            if (set) {
                valid1 = v;
                bterm1 = bt_;
            } else {
                valid0 = v;
                bterm0 = bt_;
            }
        }
        int M0 = 0, M1 = 0;
        int u[28 * NS];
#pragma unroll
        for (int b = 0; b < 28 * NS; ++b) u[b] = 0;
        int kk = 0, ll = 1;
        const int t1 = sl < 0 ? a.ntiles : min(a.G, (sl + 1) * gper) * a.nchunks;
        for (int t = first_tile(sl); t < t1; ++t) {
            const int g = t / a.nchunks, ch = t - g * a.nchunks;
            if (!tp.resident && threadIdx.x == 0) {
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
                for (int b = 0; b < 28 * NS; ++b) u[b] = 0;
                kk = sgp[2 * (g * 32 + lane)];
                ll = sgp[2 * (g * 32 + lane) + 1];
            }
            const int npos = min(a.chunk, a.npad - ch * a.chunk);
            scan_compact28<NS>(reinterpret_cast<const uint2 *>(tb) + lane, npos, F0, F1, u);
            if (ch == a.nchunks - 1) {
                M0 = max(M0, set28_group_max<0>(AQ0, a.aq_stride, a.m, kk, ll, u, lane));
                if constexpr (NS == 2) M1 = max(M1, set28_group_max<28>(AQ1, a.aq_stride, a.m, kk, ll, u, lane));
            }
            if (!tp.resident) {
                __syncthreads();
                ++tp.fill;
            }
        }
#pragma unroll
        for (int set = 0; set < NS; ++set) {
            const int64_t x = set ? x1 : x0;
            const bool valid = set ? valid1 : valid0;
            const int best = max(set ? M1 : M0, set ? bterm1 : bterm0);
            if (x < a.N) {
                if (sl < 0)
                    a.out[x] = valid ? best : FSP_LB_INVALID;
                else if (!valid)
                    a.out[x] = FSP_LB_INVALID;  // every slice finds the row invalid
                else
                    atomicMax(a.out + x, best);  // out was zeroed; bounds are >= 0
            }
        }
        __syncwarp();  // the flag and row arrays are rewritten by the next batch
    }
}

namespace {

template <int MP>
cudaError_t launch_streamed28_variant(const LanesArgs &a, int ns, int grid, int threads, size_t smem, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = set_smem_attr(fsp_lanes_streamed28<MP, 1>);
        if (attr_err == cudaSuccess) attr_err = set_smem_attr(fsp_lanes_streamed28<MP, 2>);
    });
    if (attr_err != cudaSuccess) return attr_err;
    note_launches(1);
    if (ns == 2)
        fsp_lanes_streamed28<MP, 2><<<grid, threads, smem, s>>>(a);
    else
        fsp_lanes_streamed28<MP, 1><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_streamed28_mp(const LanesArgs &a, int mp, int ns, int grid, int threads, size_t smem,
                                 cudaStream_t s) {
    switch (mp) {
        case 8: return launch_streamed28_variant<8>(a, ns, grid, threads, smem, s);
        case 12: return launch_streamed28_variant<12>(a, ns, grid, threads, smem, s);
        case 16: return launch_streamed28_variant<16>(a, ns, grid, threads, smem, s);
        case 20: return launch_streamed28_variant<20>(a, ns, grid, threads, smem, s);
        case 24: return launch_streamed28_variant<24>(a, ns, grid, threads, smem, s);
        default: return launch_streamed28_variant<32>(a, ns, grid, threads, smem, s);
    }
}

}  // namespace fspgb
