// fsp_order.cu -- the depth order of a pool, and the stream-ordered scratch
// pool of the bounding launches.
//
// A warp bounds 32 nodes with one lane per node, and the setup's loops over a
// node's prefix run as long as the warp's deepest node.  Bounding the nodes
// of a large pool in order of depth (a counting sort over the n + 3 depth
// values, invalid depths in the end bins) gives every warp nodes of one or two
// depths, so no lane idles through another lane's longer prefix.  The order
// is a permutation of slot -> node; bounds are still written at the node's
// own index.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "fsp_internal.h"

namespace fspgb {
namespace {

constexpr int kOrderThreads = 256;
constexpr int kOrderBlocks = 48;  // blocks of the histogram and scatter passes

__device__ __forceinline__ int depth_bin(int d, int n) { return min(max(d, -1), n + 1) + 1; }  // [0, n + 2]

// Block k owns nodes [k * per, (k + 1) * per): its histogram goes to
// hist[bin * blocks + k] (no global atomics).
__global__ void __launch_bounds__(kOrderThreads) order_hist(const int32_t *depths, int64_t N, int n, int64_t per,
                                                            int32_t *hist) {
    extern __shared__ int32_t h[];
    const int nb = n + 3;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t x0 = (int64_t)blockIdx.x * per, x1 = min(N, x0 + per);
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) atomicAdd(&h[depth_bin(__ldg(depths + x), n)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[(int64_t)i * gridDim.x + blockIdx.x] = h[i];
}

// Block k writes its nodes at its offsets, counting within a bin in shared
// memory (the order among equal depths is arbitrary).  Block k's first slot
// in bin b lies after every node of a smaller bin and after bin b's nodes in
// blocks before k; each block takes these offsets from the histogram itself
// (hist is nb x blocks, a few thousand entries read from L2): thread t sums a
// contiguous segment of bins, the segment sums are scanned across the block
// with warp shuffles, and each thread then walks its segment.
__global__ void __launch_bounds__(kOrderThreads) order_scatter(const int32_t *depths, int64_t N, int n, int64_t per,
                                                               const int32_t *hist, int32_t *order) {
    extern __shared__ int32_t cur[];  // [nb] slots, then [nb] bin totals
    __shared__ int32_t wsum[kOrderThreads / 32];
    const int nb = n + 3, K = gridDim.x, k = blockIdx.x;
    int32_t *tot = cur + nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = (nb + kOrderThreads - 1) / kOrderThreads;
    const int b0 = min(nb, (int)threadIdx.x * seg), b1 = min(nb, b0 + seg);
    int sum = 0;
    for (int b = b0; b < b1; ++b) {
        const int32_t *hb = hist + (int64_t)b * K;
        int t = 0, before = 0;
        for (int kk = 0; kk < K; ++kk) {
            const int h = __ldg(hb + kk);
            t += h;
            before += kk < k ? h : 0;
        }
        cur[b] = before;
        tot[b] = t;
        sum += t;
    }
    int incl = sum;  // inclusive scan of the segment sums across the warp
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int run = incl - sum;  // exclusive within the warp, plus the warps before
    for (int w = 0; w < warp; ++w) run += wsum[w];
    for (int b = b0; b < b1; ++b) {
        cur[b] += run;
        run += tot[b];
    }
    __syncthreads();
    const int64_t x0 = (int64_t)k * per, x1 = min(N, x0 + per);
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x)
        order[atomicAdd(&cur[depth_bin(__ldg(depths + x), n)], 1)] = (int32_t)x;
}

std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

}  // namespace

fsp_status scratch_pool(int dev, cudaMemPool_t *out) {
    if (dev < 0 || dev >= 64) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return FSP_ECUDA;
        // keep the memory between calls, so steady-state calls map nothing
        uint64_t keep = UINT64_MAX;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return FSP_ECUDA;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return FSP_OK;
}

fsp_status depth_order(const fsp_instance *inst, const int32_t *depths, int64_t N, cudaStream_t s,
                       int32_t **order) {
    *order = nullptr;
    // small pools, or prefixes too short for their lengths to matter: identity
    if (N < kDepthOrderMin || N > INT32_MAX || inst->n < kDepthOrderMinJobs) return FSP_OK;
    cudaMemPool_t pool = nullptr;
    fsp_status st = scratch_pool(inst->device, &pool);
    if (st != FSP_OK) return st;
    const int nb = inst->n + 3;
    const int blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>(kOrderBlocks, (N + kOrderThreads - 1) / kOrderThreads));
    const int64_t per = (N + blocks - 1) / blocks;
    const int total = nb * blocks;
    int32_t *buf = nullptr;
    if (cudaMallocFromPoolAsync((void **)&buf, sizeof(int32_t) * ((size_t)N + total), pool, s) != cudaSuccess) {
        cudaGetLastError();
        return FSP_ENOMEM;
    }
    int32_t *hist = buf + N;
    const size_t hsmem = sizeof(int32_t) * nb;
    note_launches(2);
    order_hist<<<blocks, kOrderThreads, hsmem, s>>>(depths, N, inst->n, per, hist);
    order_scatter<<<blocks, kOrderThreads, 2 * hsmem, s>>>(depths, N, inst->n, per, hist, buf);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFreeAsync(buf, s);
        return FSP_ECUDA;
    }
    *order = buf;
    return FSP_OK;
}

}  // namespace fspgb
