// fsp_noalloc.cu -- a batched bound that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a bound:
// a process whose GPU memory is already owned by another allocator (a
// framework's caching allocator holding the whole device), a serving loop
// that must not take cudaMalloc's implicit device synchronisation, or code
// running where allocation is not permitted.  fsp_bound_batch_noalloc gives
// them the batched bound of fsp_batch_create + fsp_batch_launch without any
// allocation.  The plan (one argument block per pool and the prefix sums of
// the pools' work items, at most FSP_NOALLOC_MAX_POOLS pools) travels to the
// device inside the kernel's parameter block, so no host buffer is copied
// and nothing on the host has to outlive the call.  The only device scratch,
// the work counter the warps claim items from, lives in the file-scope array
// below.
//
// The array is one per device and shared by every call: a call re-zeroes the
// counter, so calls whose work overlaps on the GPU race with each other.  The
// first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; do that first call
// outside any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "fsp_internal.h"
#include "fsp_batch_scan.cuh"
#include "fsp_lanes_device.cuh"

namespace fspgb {
namespace {

constexpr int kNoallocMaxPools = FSP_NOALLOC_MAX_POOLS;

// The plan of one call, passed by value as the kernel's parameter block
// (about 14 KB, within the 32,764 bytes a kernel's parameters may take).
struct NoallocPlan {
    LanesArgs pools[kNoallocMaxPools];
    int64_t offs[kNoallocMaxPools + 1];  // work-item prefix sums of the pools
};
static_assert(sizeof(NoallocPlan) + 64 <= 32764, "plan exceeds the kernel parameter space");

// Device scratch of the entry point: the work counter (one int32 at offset 0).
constexpr size_t kScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Work item `claim` of the plan belongs to the pool whose [offs[p], offs[p+1])
// range holds it (pools are ordered longest items first on the host).
__device__ __forceinline__ int pool_of(const int64_t *offs, int count, int64_t claim) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= claim)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int MP>
__global__ void __launch_bounds__(512, 1)
    fsp_lanes_batch_noalloc(const __grid_constant__ NoallocPlan plan, int32_t *counter, int count, int64_t nitems,
                            int32_t n_max, int32_t aq_stride, uint32_t off_aq) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *F = reinterpret_cast<uint32_t *>(smem) + (size_t)warp * n_max;
    int32_t *AQ = reinterpret_cast<int32_t *>(smem + off_aq) + (size_t)warp * 32 * aq_stride;
    for (;;) {
        int claim = 0;
        if (lane == 0) claim = atomicAdd(counter, 1);
        claim = __shfl_sync(kFull, claim, 0);
        if ((int64_t)claim >= nitems) break;
        const int pi = pool_of(plan.offs, count, claim);
        const LanesArgs &a = plan.pools[pi];
        const int64_t x = ((int64_t)claim - plan.offs[pi]) * 32 + lane;
        int bterm = 0;
        const bool valid = lanes_setup<MP>(a, x, lane, F, AQ + lane * aq_stride, bterm);
        int lb[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) lb[b] = 0;
        for (int g = 0; g < a.G; ++g) {
            const int kk = __ldg(a.gpairs + 2 * (g * 32 + lane)), ll = __ldg(a.gpairs + 2 * (g * 32 + lane) + 1);
            int u[32];
#pragma unroll
            for (int b = 0; b < 32; ++b) u[b] = 0;
            const uint2 *R = reinterpret_cast<const uint2 *>(a.grec) + (size_t)g * a.npad * 32 + lane;
            scan_compact_global(R, a.npad, F, u);
            couple_epilogue<false>(AQ, aq_stride, a.m, kk, ll, u, lb);
        }
        const int best = transpose_max(lb, lane);
        if (x < a.N) a.out[x] = valid ? max(best, bterm) : FSP_LB_INVALID;
        __syncwarp();
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_addr_mu;
unsigned char *g_addr[64] = {};

fsp_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= 64) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FSP_ECUDA;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return FSP_OK;
}

// The kernel's dynamic shared-memory limit is raised to the device's opt-in
// maximum once per device and variant, so concurrent calls never change it
// under each other; each launch passes its own size.
template <int MP>
cudaError_t launch_noalloc(int dev, const NoallocPlan &plan, int32_t *counter, int count, int64_t nitems, int n_max,
                           int stride, uint32_t off_aq, int grid, int threads, size_t smem, cudaStream_t s) {
    static std::once_flag once[64];
    static cudaError_t attr_err[64] = {};
    std::call_once(once[dev], [dev] {
        attr_err[dev] = cudaFuncSetAttribute(fsp_lanes_batch_noalloc<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             max_smem_per_block(dev));
    });
    if (attr_err[dev] != cudaSuccess) return attr_err[dev];
    fsp_lanes_batch_noalloc<MP><<<grid, threads, smem, s>>>(plan, counter, count, nitems, n_max, stride, off_aq);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fspgb

using namespace fspgb;

extern "C" fsp_status fsp_bound_batch_noalloc(const fsp_pool_desc *pools, int32_t count, void *cuda_stream) {
    if (count < 0 || (count > 0 && !pools)) return FSP_EINVAL;
    if (count > kNoallocMaxPools) return FSP_EINVAL;  // more pools than the scratch array holds
    if (count == 0) return FSP_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FSP_ECUDA;
    int n_max = 1, m_max = 2, mp = 8;
    for (int32_t i = 0; i < count; ++i) {
        const fsp_pool_desc &p = pools[i];
        if (!p.inst || p.N < 0 || (p.N > 0 && (!p.nodes || !p.depths || !p.out_lb))) return FSP_EINVAL;
        if (p.inst->device != dev || !p.inst->compact) return FSP_EINVAL;
        n_max = std::max(n_max, p.inst->n);
        m_max = std::max(m_max, p.inst->m);
        mp = std::max(mp, p.inst->mpad);
    }
    n_max = flag_words(n_max);  // flag words per warp
    unsigned char *scratch = nullptr;
    fsp_status st = scratch_address(dev, &scratch);
    if (st != FSP_OK) return st;

    // The plan is built on the host without allocating: pools ordered by the
    // cost of one work item, longest first (an insertion sort, stable, on at
    // most 64 entries), then their item prefix sums.  It is handed to the
    // kernel by value; the launch copies it, so the one static plan buffer
    // (14 KB, kept off the caller's stack) is free again when the launch
    // returns, and a mutex keeps two threads' calls from filling it at once.
    int order[kNoallocMaxPools];
    auto cost = [&](int i) { return (int64_t)pools[i].inst->G * pools[i].inst->npad; };
    for (int i = 0; i < count; ++i) {
        int j = i;
        for (; j > 0 && cost(order[j - 1]) < cost(i); --j) order[j] = order[j - 1];
        order[j] = i;
    }
    const int stride = (m_max + (m_max + 1) / 2) | 1;
    static NoallocPlan plan;
    static std::mutex plan_mu;
    std::lock_guard<std::mutex> plan_lock(plan_mu);
    std::memset(&plan, 0, sizeof plan);
    plan.offs[0] = 0;
    for (int r = 0; r < count; ++r) {
        const fsp_pool_desc &p = pools[order[r]];
        const fsp_instance *inst = p.inst;
        LanesArgs &a = plan.pools[r];
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
        a.aq_stride = stride;
        a.release = (inst->flags & FSP_INSTANCE_RELEASE_PER_JOB) ? 1 : 0;
        a.q32 = inst->compact ? 0 : 1;
        plan.offs[r + 1] = plan.offs[r] + (p.N + 31) / 32;
    }
    const int64_t nitems = plan.offs[count];
    if (nitems > INT32_MAX) return FSP_EINVAL;
    if (nitems == 0) return FSP_OK;

    // shared memory: flags [warps][n_max] words, rows [warps][32][stride] ints
    const int optin = max_smem_per_block(dev);
    int W = 16;
    uint32_t off_aq = 0;
    size_t smem = 0;
    for (; W >= 1; --W) {
        off_aq = (uint32_t)(((size_t)W * n_max * 4 + 127) / 128 * 128);
        smem = ((size_t)off_aq + (size_t)W * 32 * stride * 4 + 127) / 128 * 128;
        if (smem <= (size_t)optin) break;
    }
    if (W < 1) return FSP_EINVAL;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nitems + W - 1) / W, num_sms(dev)));

    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int32_t *counter = reinterpret_cast<int32_t *>(scratch);
    if (cudaMemsetAsync(counter, 0, sizeof(int32_t), s) != cudaSuccess) return FSP_ECUDA;
    cudaError_t e;
    switch (mp) {
#define FSP_NOALLOC_CASE(MPV)                                                                                  \
    case MPV:                                                                                                   \
        e = launch_noalloc<MPV>(dev, plan, counter, count, nitems, n_max, stride, off_aq, grid, 32 * W, smem, s); \
        break;
        FSP_NOALLOC_CASE(8)
        FSP_NOALLOC_CASE(12)
        FSP_NOALLOC_CASE(16)
        FSP_NOALLOC_CASE(20)
        FSP_NOALLOC_CASE(24)
#undef FSP_NOALLOC_CASE
        default: e = launch_noalloc<32>(dev, plan, counter, count, nitems, n_max, stride, off_aq, grid, 32 * W, smem, s); break;
    }
    return e == cudaSuccess ? FSP_OK : FSP_ECUDA;
}
