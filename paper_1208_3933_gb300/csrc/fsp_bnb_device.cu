// fsp_bnb_device.cu -- depth-first branch-and-bound with branching and
// elimination on the device.
//
// The paper keeps selection, branching and elimination on the CPU and ships
// each pool of children to the GPU for bounding (Section III-A).  Here the
// open nodes live in a device stack and never leave the device; one round
//   1. pops up to `expand` nodes from the top of the stack (a parent whose
//      bound reached the incumbent is dropped: elimination),
//   2. branches each parent into one child per unscheduled job (forward
//      branching, Section II-B: the job is appended to the prefix), children
//      of a parent in job order,
//   3. bounds all children as one pool (the couple-lanes kernels),
//   4. takes the best leaf (a leaf's bound is its makespan) as the new
//      incumbent when it improves, drops children whose bound reaches the
//      incumbent, and pushes the survivors back where the parents were, the
//      children of the topmost parent on top and, within a parent, in
//      decreasing (bound, job) order so that the smallest is popped first.
// The round's sizes (stack size, parents popped, children generated) live in
// device state that the round kernels read, so a depth-first search enqueues
// rounds back to back and the host reads the state once per group of rounds
// (stack growth, node limit, termination) -- no host round trip per pool.
// Best-first selection and searches whose children would need a large
// bounding launch read the state once per round instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "fsp_internal.h"

namespace fspgb {
namespace {

constexpr int kScanThreads = 1024;

// Round state kept on the device.
struct DevState {
    int32_t best;          // incumbent makespan, or ub0 + 1 before any
    int32_t found;         // an incumbent exists
    int32_t total;         // children generated this round
    int32_t survivors;     // children pushed this round
    unsigned long long round_key;  // (makespan << 32) | child of this round's best leaf
    long long S;           // open nodes on the stack
    long long top0;        // first parent popped this round (S - k)
    long long count;       // nodes bounded so far
    int32_t k;             // parents popped this round
    int32_t pad;
};

// Block-wide exclusive scan of `count(i)` over i in [0, k): out[i] and the
// total in out[k].  One block of kScanThreads threads.
template <typename CountF>
__device__ void block_exclusive_scan(int k, CountF count, int32_t *out) {
    __shared__ int32_t part[kScanThreads];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < k; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int v = i < k ? count(i) : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < kScanThreads; off <<= 1) {
            const int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < k) out[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry += part[kScanThreads - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = carry;
}

// (1)+(2a) children per popped parent: n - d for a parent still below the
// incumbent, else 0; offsets of each parent's children.
// The round pops k = min(K, S) parents from the top of the stack.
__global__ void __launch_bounds__(kScanThreads) bnb_count_children(const int32_t *sdep, const int32_t *slb, int K,
                                                                     int n, DevState *st, int32_t *offs) {
    const int32_t best = st->best;
    const int64_t S = st->S;
    const int k = (int)(S < K ? S : K);
    const int64_t top0 = S - k;
    block_exclusive_scan(
        k, [&](int i) { return slb[top0 + i] < best ? n - sdep[top0 + i] : 0; }, offs);
    if (threadIdx.x == 0) {
        st->k = k;
        st->top0 = top0;
        st->total = offs[k];
        st->round_key = ~0ull;
    }
}

// (2b) one warp per parent writes its children: the parent's prefix plus one
// unscheduled job, in job order.
__global__ void bnb_make_children(const int16_t *srows, const int32_t *sdep, int n, const DevState *st,
                                  const int32_t *offs, int16_t *crows, int32_t *cdep, int32_t *cparent) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= st->k) return;
    const int64_t top0 = st->top0;
    const int c0 = offs[p], cnt = offs[p + 1] - c0;
    if (cnt == 0) return;
    const int d = sdep[top0 + p];
    const int16_t *prow = srows + (top0 + p) * (int64_t)n;
    // scheduled-job bitmap of the prefix, built by the warp in shared memory
    extern __shared__ uint32_t sched[];
    const int nw = (n + 31) >> 5;
    uint32_t *bm = sched + (threadIdx.x >> 5) * nw;
    for (int w = lane; w < nw; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int i = lane; i < d; i += 32) {
        const int j = prow[i];
        atomicOr(&bm[j >> 5], 1u << (j & 31));
    }
    __syncwarp();
    // the r-th unscheduled job (in job order) becomes child c0 + r
    int r = 0;
    for (int w = 0; w < nw; ++w) {
        const uint32_t un = ~bm[w] & (w == nw - 1 && (n & 31) ? ((1u << (n & 31)) - 1u) : 0xffffffffu);
        const int j = w * 32 + lane;
        const bool mine = (un >> lane) & 1u;
        const int rank = r + __popc(un & ((1u << lane) - 1u));
        if (mine) {
            const int c = c0 + rank;
            int16_t *crow = crows + (int64_t)c * n;
            for (int i = 0; i < d; ++i) crow[i] = prow[i];
            crow[d] = (int16_t)j;
            for (int i = d + 1; i < n; ++i) crow[i] = 0;
            cdep[c] = d + 1;
            cparent[c] = p;
        }
        r += __popc(un);
    }
}

// (4a) leaves update the round's best; other children survive while their
// bound is below the incumbent.
__device__ __forceinline__ void filter_child(int c, const int32_t *clb, const int32_t *cdep, int n, int32_t best,
                                             DevState *st, int32_t *keep) {
    const int32_t lb = clb[c];
    int kv = 0;
    if (lb >= 0 && lb < best) {
        if (cdep[c] == n)
            atomicMin(&st->round_key, ((unsigned long long)(uint32_t)lb << 32) | (uint32_t)c);
        else
            kv = 1;
    }
    keep[c] = kv;
}

__global__ void bnb_filter(const int32_t *clb, const int32_t *cdep, int n, DevState *st, int32_t *keep) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st->total) return;
    filter_child(c, clb, cdep, n, st->best, st, keep);
}

// (4b) the incumbent from this round's best leaf.
__global__ void bnb_incumbent(const int16_t *crows, int n, DevState *st, int16_t *best_row) {
    const unsigned long long key = st->round_key;
    if (key == ~0ull) return;
    const int32_t ms = (int32_t)(key >> 32);
    if (ms >= st->best) return;
    const int c = (int)(key & 0xffffffffu);
    for (int i = threadIdx.x; i < n; i += blockDim.x) best_row[i] = crows[(int64_t)c * n + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        st->best = ms;
        st->found = 1;
    }
}

// (4c) survivors per parent and their offsets in the stack; the new stack
// size (the survivors replace the popped parents) and the node count.
__global__ void __launch_bounds__(kScanThreads) bnb_count_survivors(const int32_t *offs, const int32_t *keep,
                                                                      DevState *st, int32_t *soffs) {
    const int k = st->k;
    block_exclusive_scan(
        k,
        [&](int p) {
            int s = 0;
            for (int c = offs[p]; c < offs[p + 1]; ++c) s += keep[c];
            return s;
        },
        soffs);
    if (threadIdx.x == 0) {
        st->survivors = soffs[k];
        st->S = st->top0 + soffs[k];
        st->count += st->total;
    }
}

// (4d) push: survivor c of parent p goes to top0 + soffs[p] + (number of
// surviving siblings with a larger (bound, job)).
__device__ __forceinline__ void push_child(int c, const int16_t *crows, const int32_t *cdep, const int32_t *clb,
                                           const int32_t *cparent, const int32_t *offs, const int32_t *keep,
                                           const int32_t *soffs, int n, int64_t top0, int16_t *srows,
                                           int32_t *sdep, int32_t *slb) {
    const int p = cparent[c];
    const int32_t lb = clb[c];
    const int d = cdep[c];
    const int job = crows[(int64_t)c * n + d - 1];
    int r = 0;
    for (int s = offs[p]; s < offs[p + 1]; ++s) {
        if (s == c || !keep[s]) continue;
        const int32_t lbs = clb[s];
        const int jobs = crows[(int64_t)s * n + d - 1];
        r += (lbs > lb) || (lbs == lb && jobs > job);
    }
    const int64_t dst = top0 + soffs[p] + r;
    for (int i = 0; i < n; ++i) srows[dst * n + i] = crows[(int64_t)c * n + i];
    sdep[dst] = d;
    slb[dst] = lb;
}

__global__ void bnb_push(const int16_t *crows, const int32_t *cdep, const int32_t *clb, const int32_t *cparent,
                         const int32_t *offs, const int32_t *keep, const int32_t *soffs, int n, const DevState *st,
                         int16_t *srows, int32_t *sdep, int32_t *slb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st->total || !keep[c]) return;
    push_child(c, crows, cdep, clb, cparent, offs, keep, soffs, n, st->top0, srows, sdep, slb);
}

// (4a)-(4d) in one block, for rounds of at most a few thousand children:
// the same filter, incumbent, survivor count and push as the four kernels
// above, separated by block barriers instead of launches.
__global__ void __launch_bounds__(kScanThreads) bnb_round_tail(const int16_t *crows, const int32_t *cdep,
                                                                 const int32_t *clb, const int32_t *cparent,
                                                                 const int32_t *offs, int n, DevState *st,
                                                                 int32_t *keep, int32_t *soffs, int16_t *best_row,
                                                                 int16_t *srows, int32_t *sdep, int32_t *slb) {
    __shared__ int s_leaf;
    __shared__ int32_t s_ms;
    const int total = st->total, k = st->k;
    const int64_t top0 = st->top0;
    const int32_t best = st->best;
    for (int c = threadIdx.x; c < total; c += blockDim.x) filter_child(c, clb, cdep, n, best, st, keep);
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long key = st->round_key;
        s_leaf = -1;
        if (key != ~0ull && (int32_t)(key >> 32) < best) {
            s_leaf = (int)(key & 0xffffffffu);
            s_ms = (int32_t)(key >> 32);
        }
    }
    __syncthreads();
    if (s_leaf >= 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) best_row[i] = crows[(int64_t)s_leaf * n + i];
        if (threadIdx.x == 0) {
            st->best = s_ms;
            st->found = 1;
        }
    }
    block_exclusive_scan(
        k,
        [&](int p) {
            int v = 0;
            for (int c = offs[p]; c < offs[p + 1]; ++c) v += keep[c];
            return v;
        },
        soffs);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->survivors = soffs[k];
        st->S = top0 + soffs[k];
        st->count += total;
    }
    for (int c = threadIdx.x; c < total; c += blockDim.x)
        if (keep[c]) push_child(c, crows, cdep, clb, cparent, offs, keep, soffs, n, top0, srows, sdep, slb);
}

// ---- best-first selection: bring the k open nodes of smallest bound to the
// top of the stack (positions [S - k, S)), so that the round expands them;
// among equal bounds the deeper node first (the usual tie-break, which dives
// to leaves instead of widening a plateau of equal bounds), and among equal
// keys the node higher on the stack (the most recently pushed, as depth-first
// order would take it).  The key (lb - lo) * (n + 1) + (n - d) is binned
// relative to the root's bound (bounds never decrease along a branch):
// bin = min(key >> shift, nbins - 1).  Every step is deterministic: the
// threshold bin's share is taken by stack position through per-tile counts
// and scans, and the swap lists are built in stack order, so a search
// expands the same nodes on every run.
constexpr int kBestBins = 4096;
constexpr int kTile = 256;  // stack entries per block step of the selection passes

struct BestState {
    int32_t tb;        // threshold bin: every node in a lower bin is selected
    int32_t need_tb;   // how many nodes of bin tb are selected (the highest on the stack)
    int32_t n_out;     // selected nodes below the top region
    int32_t n_in;      // unselected nodes inside the top region
};

// Block of kTile threads: how many threads of higher (after) or lower
// (before) index in the block have f set.
__device__ __forceinline__ int block_count_after(bool f, int32_t *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    int c = lane == 31 ? 0 : __popc(bal >> (lane + 1));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    for (int v = w + 1; v < kTile / 32; ++v) c += wsum[v];
    __syncthreads();
    return c;
}

__device__ __forceinline__ int block_count_before(bool f, int32_t *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    int c = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    for (int v = 0; v < w; ++v) c += wsum[v];
    __syncthreads();
    return c;
}

__device__ __forceinline__ int best_bin(int32_t lb, int32_t d, int n, int32_t lo, int shift) {
    const int64_t key = (int64_t)(lb < lo ? 0 : lb - lo) * (n + 1) + (n - d);
    const int64_t b = key >> shift;
    return (int)(b < kBestBins - 1 ? b : kBestBins - 1);
}

__global__ void bnb_best_hist(const int32_t *slb, const int32_t *sdep, int64_t S, int n, int32_t lo, int shift,
                              int32_t *hist) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[best_bin(slb[i], sdep[i], n, lo, shift)], 1);
}

// one block: the first bin at which the cumulative count reaches k
__global__ void __launch_bounds__(kScanThreads) bnb_best_threshold(int32_t *hist, int k, BestState *bs) {
    block_exclusive_scan(kBestBins, [&](int i) { return hist[i]; }, hist);
    __syncthreads();
    for (int i = threadIdx.x; i < kBestBins; i += blockDim.x) {
        const int before = hist[i], upto = i + 1 < kBestBins ? hist[i + 1] : hist[kBestBins];
        if (before < k && upto >= k) {
            bs->tb = i;
            bs->need_tb = k - before;
        }
    }
}

// bin-tb nodes per tile of kTile stack entries
__global__ void __launch_bounds__(kTile) bnb_best_tile_count(const int32_t *slb, const int32_t *sdep, int64_t S,
                                                            int n, int32_t lo, int shift, const BestState *bs,
                                                            int32_t *tcount) {
    const int tb = bs->tb;
    for (int64_t t = blockIdx.x; t * kTile < S; t += gridDim.x) {
        const int64_t i = t * kTile + threadIdx.x;
        const int c = __syncthreads_count(i < S && best_bin(slb[i], sdep[i], n, lo, shift) == tb);
        if (threadIdx.x == 0) tcount[t] = c;
    }
}

// one block: tabove[T - 1 - t] = bin-tb nodes in the tiles above tile t
__global__ void __launch_bounds__(kScanThreads) bnb_best_tile_above(const int32_t *tcount, int T, int32_t *tabove) {
    block_exclusive_scan(T, [&](int r) { return tcount[T - 1 - r]; }, tabove);
}

// Selection of every node: bins below tb, and the need_tb nodes of bin tb
// highest on the stack; per tile, the selected nodes below the top region
// and the unselected ones inside it.
__global__ void __launch_bounds__(kTile) bnb_best_mark(const int32_t *slb, const int32_t *sdep, int64_t S, int n,
                                                      int k, int32_t lo, int shift, const BestState *bs,
                                                      const int32_t *tabove, int T, uint8_t *sel_flag,
                                                      int32_t *out_cnt, int32_t *in_cnt) {
    __shared__ int32_t wsum[kTile / 32];
    const int tb = bs->tb, need = bs->need_tb;
    const int64_t top0 = S - k;
    for (int64_t t = blockIdx.x; t * kTile < S; t += gridDim.x) {
        const int64_t i = t * kTile + threadIdx.x;
        const int b = i < S ? best_bin(slb[i], sdep[i], n, lo, shift) : kBestBins;
        const int rank = tabove[T - 1 - t] + block_count_after(b == tb, wsum);
        const bool sel = b < tb || (b == tb && rank < need);
        if (i < S) sel_flag[i] = sel ? 1 : 0;
        const int no = __syncthreads_count(sel && i < top0);
        const int ni = __syncthreads_count(i < S && !sel && i >= top0);
        if (threadIdx.x == 0) {
            out_cnt[t] = no;
            in_cnt[t] = ni;
        }
    }
}

// one block: list offsets per tile (exclusive scans) and the list lengths
__global__ void __launch_bounds__(kScanThreads) bnb_best_list_offsets(const int32_t *out_cnt, const int32_t *in_cnt,
                                                                      int T, int32_t *out_off, int32_t *in_off,
                                                                      BestState *bs) {
    block_exclusive_scan(T, [&](int t) { return out_cnt[t]; }, out_off);
    __syncthreads();
    block_exclusive_scan(T, [&](int t) { return in_cnt[t]; }, in_off);
    __syncthreads();
    if (threadIdx.x == 0) {
        bs->n_out = out_off[T];
        bs->n_in = in_off[T];
    }
}

// both swap lists in stack order
__global__ void __launch_bounds__(kTile) bnb_best_lists(int64_t S, int k, const uint8_t *sel_flag,
                                                       const int32_t *out_off, const int32_t *in_off,
                                                       int64_t *out_list, int64_t *in_list) {
    __shared__ int32_t wsum[kTile / 32];
    const int64_t top0 = S - k;
    for (int64_t t = blockIdx.x; t * kTile < S; t += gridDim.x) {
        const int64_t i = t * kTile + threadIdx.x;
        const bool sel = i < S && sel_flag[i];
        const bool o = sel && i < top0, q = i < S && !sel && i >= top0;
        const int ro = block_count_before(o, wsum);
        const int rq = block_count_before(q, wsum);
        if (o) out_list[out_off[t] + ro] = i;
        if (q) in_list[in_off[t] + rq] = i;
    }
}

// swaps the t-th selected node below the top with the t-th unselected one in
// it (the two lists have the same length); one warp per pair
__global__ void bnb_best_swap(int16_t *srows, int32_t *sdep, int32_t *slb, int n, const BestState *bs,
                              const int64_t *out_list, const int64_t *in_list) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= bs->n_out) return;
    const int64_t a = out_list[t], b = in_list[t];
    for (int i = lane; i < n; i += 32) {
        const int16_t x = srows[a * n + i];
        srows[a * n + i] = srows[b * n + i];
        srows[b * n + i] = x;
    }
    if (lane == 0) {
        const int32_t d = sdep[a], l = slb[a];
        sdep[a] = sdep[b];
        slb[a] = slb[b];
        sdep[b] = d;
        slb[b] = l;
    }
}

struct DevBuffers {
    int16_t *srows = nullptr, *crows = nullptr, *best_row = nullptr;
    int32_t *sdep = nullptr, *slb = nullptr, *cdep = nullptr, *clb = nullptr, *cparent = nullptr;
    int32_t *offs = nullptr, *keep = nullptr, *soffs = nullptr;
    DevState *st = nullptr;
    int32_t *hist = nullptr;                    // best-first: bins
    BestState *bs = nullptr;                    // best-first: threshold and list lengths
    int64_t *out_list = nullptr, *in_list = nullptr;  // best-first: swap pairs (expand each)
    int32_t *tiles = nullptr;                   // best-first: six per-tile arrays of tiles_cap + 1
    uint8_t *sel_flag = nullptr;                // best-first: selection of every stack entry
    int64_t cap = 0, tiles_cap = 0;
    cudaGraphExec_t round_exec = nullptr;       // one depth-first round, captured
    const int16_t *round_rows = nullptr;        // the stack the captured round writes
    int round_kernels = 0;                      // kernels in the captured round
    void release() {
        if (round_exec) cudaGraphExecDestroy(round_exec);
        round_exec = nullptr;
        for (void *p : {(void *)srows, (void *)crows, (void *)best_row, (void *)sdep, (void *)slb, (void *)cdep,
                        (void *)clb, (void *)cparent, (void *)offs, (void *)keep, (void *)soffs, (void *)st,
                        (void *)hist, (void *)bs, (void *)out_list, (void *)in_list, (void *)tiles,
                        (void *)sel_flag})
            if (p) cudaFree(p);
    }
};

// Best-first scratch for a stack of b.cap entries (contents not kept).
fsp_status grow_best(DevBuffers &b) {
    const int64_t T = (b.cap + kTile - 1) / kTile;
    if (T <= b.tiles_cap) return FSP_OK;
    if (b.tiles) cudaFree(b.tiles);
    if (b.sel_flag) cudaFree(b.sel_flag);
    b.tiles = nullptr;
    b.sel_flag = nullptr;
    b.tiles_cap = 0;
    if (cudaMalloc((void **)&b.tiles, sizeof(int32_t) * 6 * (size_t)(T + 1)) != cudaSuccess ||
        cudaMalloc((void **)&b.sel_flag, (size_t)b.cap) != cudaSuccess)
        return FSP_ENOMEM;
    b.tiles_cap = T;
    return FSP_OK;
}

// Grows the stack to hold `need` nodes, keeping its first `keep_nodes`.
fsp_status grow_stack(DevBuffers &b, int n, int64_t need, int64_t keep_nodes) {
    if (need <= b.cap) return FSP_OK;
    const int64_t cap = std::max<int64_t>(need, b.cap * 2);
    int16_t *r = nullptr;
    int32_t *d = nullptr, *l = nullptr;
    if (cudaMalloc((void **)&r, sizeof(int16_t) * cap * n) != cudaSuccess ||
        cudaMalloc((void **)&d, sizeof(int32_t) * cap) != cudaSuccess ||
        cudaMalloc((void **)&l, sizeof(int32_t) * cap) != cudaSuccess) {
        if (r) cudaFree(r);
        if (d) cudaFree(d);
        return FSP_ENOMEM;
    }
    if (keep_nodes > 0 &&
        (cudaMemcpy(r, b.srows, sizeof(int16_t) * keep_nodes * n, cudaMemcpyDeviceToDevice) != cudaSuccess ||
         cudaMemcpy(d, b.sdep, sizeof(int32_t) * keep_nodes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
         cudaMemcpy(l, b.slb, sizeof(int32_t) * keep_nodes, cudaMemcpyDeviceToDevice) != cudaSuccess)) {
        cudaFree(r);
        cudaFree(d);
        cudaFree(l);
        return FSP_ECUDA;
    }
    if (b.srows) cudaFree(b.srows);
    if (b.sdep) cudaFree(b.sdep);
    if (b.slb) cudaFree(b.slb);
    b.srows = r;
    b.sdep = d;
    b.slb = l;
    b.cap = cap;
    return FSP_OK;
}

}  // namespace
}  // namespace fspgb

using namespace fspgb;

extern "C" fsp_status fsp_branch_and_bound_device(const fsp_instance *inst, int32_t ub0, int32_t expand,
                                                  int32_t selection, int64_t node_limit, int16_t *best_perm,
                                                  int32_t *best_makespan, int64_t *nodes_bounded) {
    if (!inst || expand < 0 || expand > 65536 || node_limit < 0) return FSP_EINVAL;
    if (selection != FSP_SELECT_DEPTH_FIRST && selection != FSP_SELECT_BEST_FIRST) return FSP_EINVAL;
    const bool best_first = selection == FSP_SELECT_BEST_FIRST;
    fsp_status st = check_device(inst);
    if (st != FSP_OK) return st;
    st = take_device_status(inst);
    if (st != FSP_OK) return st;
    const int n = inst->n;
    const int K = expand ? expand : 256;
    const int64_t max_children = (int64_t)K * n;
    if (max_children > INT32_MAX) return FSP_EINVAL;

    DevBuffers b;
    cudaStream_t s = nullptr;
    DevState *hst = nullptr;
    auto fail = [&](fsp_status e) {
        if (s) cudaStreamSynchronize(s);
        b.release();
        if (hst) cudaFreeHost(hst);
        if (s) cudaStreamDestroy(s);
        return e;
    };
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(FSP_ECUDA);
    if (cudaMallocHost((void **)&hst, sizeof(DevState)) != cudaSuccess) return fail(FSP_ENOMEM);
    if (cudaMalloc((void **)&b.crows, sizeof(int16_t) * max_children * n) != cudaSuccess ||
        cudaMalloc((void **)&b.best_row, sizeof(int16_t) * n) != cudaSuccess ||
        cudaMalloc((void **)&b.cdep, sizeof(int32_t) * max_children) != cudaSuccess ||
        cudaMalloc((void **)&b.clb, sizeof(int32_t) * max_children) != cudaSuccess ||
        cudaMalloc((void **)&b.cparent, sizeof(int32_t) * max_children) != cudaSuccess ||
        cudaMalloc((void **)&b.keep, sizeof(int32_t) * max_children) != cudaSuccess ||
        cudaMalloc((void **)&b.offs, sizeof(int32_t) * (K + 1)) != cudaSuccess ||
        cudaMalloc((void **)&b.soffs, sizeof(int32_t) * (K + 1)) != cudaSuccess ||
        cudaMalloc((void **)&b.st, sizeof(DevState)) != cudaSuccess)
        return fail(FSP_ENOMEM);
    if (best_first && (cudaMalloc((void **)&b.hist, sizeof(int32_t) * (kBestBins + 1)) != cudaSuccess ||
                       cudaMalloc((void **)&b.bs, sizeof(BestState)) != cudaSuccess ||
                       cudaMalloc((void **)&b.out_list, sizeof(int64_t) * K) != cudaSuccess ||
                       cudaMalloc((void **)&b.in_list, sizeof(int64_t) * K) != cudaSuccess))
        return fail(FSP_ENOMEM);
    st = grow_stack(b, n, std::max<int64_t>(4096, max_children), 0);
    if (st != FSP_OK) return fail(st);

    // the root: empty prefix, bounded like any node
    int64_t count = 0;
    int32_t root_lb = 0;  // bounds never decrease along a branch: the floor of every bin
    {
        if (cudaMemsetAsync(b.srows, 0, sizeof(int16_t) * n, s) != cudaSuccess ||
            cudaMemsetAsync(b.sdep, 0, sizeof(int32_t), s) != cudaSuccess)
            return fail(FSP_ECUDA);
        st = launch_bound(inst, b.srows, b.sdep, 1, b.slb, s, nullptr);
        if (st != FSP_OK) return fail(st);
        count = 1;
        if (cudaMemcpyAsync(&root_lb, b.slb, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(FSP_ECUDA);
        DevState init = {};
        init.best = (int32_t)std::min<int64_t>((int64_t)ub0 + 1, INT32_MAX);
        init.found = 0;
        init.round_key = ~0ull;
        init.S = 1;
        init.count = 1;
        *hst = init;
        if (cudaMemcpyAsync(b.st, hst, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(FSP_ECUDA);
    }
    // A depth-first search whose rounds bound at most kAsyncMaxChildren
    // children enqueues kRoundsPerSync rounds at a time, each bounding every
    // child slot (slots past the round's children hold stale rows, bounded
    // and ignored); otherwise the host reads the round's child count and
    // bounds exactly those.
    constexpr int64_t kAsyncMaxChildren = 16384;
    constexpr int kRoundsPerSync = 16;
    const bool async_rounds = !best_first && max_children <= kAsyncMaxChildren;
    if (cudaMemsetAsync(b.cdep, 0xff, sizeof(int32_t) * max_children, s) != cudaSuccess) return fail(FSP_ECUDA);
    int64_t S = 1;  // the root is open (and counted as bounded)
    const int make_warps = 8;
    const size_t make_smem = (size_t)make_warps * ((n + 31) / 32) * 4;
    while (S > 0) {
        if (node_limit && count >= node_limit) {
            cudaStreamSynchronize(s);
            if (nodes_bounded) *nodes_bounded = count;
            b.release();
            cudaFreeHost(hst);
            cudaStreamDestroy(s);
            return FSP_ETIMEDOUT;
        }
        // A round pops at most K nodes, so a stack of S nodes cannot empty
        // within S / K rounds: the group never runs past the search's end.
        const int group = async_rounds ? (int)std::max<int64_t>(1, std::min<int64_t>(kRoundsPerSync, S / K)) : 1;
        // room for every child of this group's rounds
        st = grow_stack(b, n, S + (int64_t)group * max_children, S);
        if (st != FSP_OK) return fail(st);
        // the kernels of one round over nb child slots; with nb < 0 the
        // children are counted first, and a round without children ends
        // there (*ended: the stack lost its k popped parents)
        bool ended = false;
        auto enqueue_round = [&](int64_t nb) -> fsp_status {
            note_launches(2);
            bnb_count_children<<<1, kScanThreads, 0, s>>>(b.sdep, b.slb, K, n, b.st, b.offs);
            bnb_make_children<<<(K + make_warps - 1) / make_warps, 32 * make_warps, make_smem, s>>>(
                b.srows, b.sdep, n, b.st, b.offs, b.crows, b.cdep, b.cparent);
            if (cudaGetLastError() != cudaSuccess) return FSP_ECUDA;
            if (nb < 0) {  // the counted children (read back now)
                if (cudaMemcpyAsync(hst, b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return FSP_ECUDA;
                nb = hst->total;
                if (nb == 0) {
                    // nothing to bound or push: the new stack size is top0
                    hst->S = hst->top0;
                    ended = true;
                    return cudaMemcpyAsync(&b.st->S, &hst->S, sizeof(hst->S), cudaMemcpyHostToDevice, s) ==
                                   cudaSuccess
                               ? FSP_OK
                               : FSP_ECUDA;
                }
            }
            if (nb > 0) {
                const fsp_status bs = launch_bound(inst, b.crows, b.cdep, nb, b.clb, s, nullptr);
                if (bs != FSP_OK) return bs;
            }
            if (async_rounds) {  // at most kAsyncMaxChildren children: one block
                note_launches(1);
                bnb_round_tail<<<1, kScanThreads, 0, s>>>(b.crows, b.cdep, b.clb, b.cparent, b.offs, n, b.st,
                                                          b.keep, b.soffs, b.best_row, b.srows, b.sdep, b.slb);
                return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ECUDA;
            }
            const int tb = 256, gb = (int)((std::max<int64_t>(nb, 1) + tb - 1) / tb);
            note_launches(4);
            bnb_filter<<<gb, tb, 0, s>>>(b.clb, b.cdep, n, b.st, b.keep);
            bnb_incumbent<<<1, 128, 0, s>>>(b.crows, n, b.st, b.best_row);
            bnb_count_survivors<<<1, kScanThreads, 0, s>>>(b.offs, b.keep, b.st, b.soffs);
            bnb_push<<<gb, tb, 0, s>>>(b.crows, b.cdep, b.clb, b.cparent, b.offs, b.keep, b.soffs, n, b.st,
                                       b.srows, b.sdep, b.slb);
            return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ECUDA;
        };
        if (async_rounds && group > 1) {
            // Groups of depth-first rounds replay one captured round, each
            // bounding every child slot; it is captured again when the stack
            // has moved (the first round of a search runs uncaptured, so the
            // kernels' one-time attributes are set outside any capture).
            if (!b.round_exec || b.round_rows != b.srows) {
                cudaMemPool_t pool = nullptr;  // created outside the capture, if the bound needs scratch
                st = scratch_pool(inst->device, &pool);
                if (st != FSP_OK) return fail(st);
                if (b.round_exec) cudaGraphExecDestroy(b.round_exec);
                b.round_exec = nullptr;
                cudaGraph_t g = nullptr;
                const int64_t before = fsp_kernel_launches();
                if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return fail(FSP_ECUDA);
                const fsp_status rs = enqueue_round(max_children);
                const cudaError_t ec = cudaStreamEndCapture(s, &g);
                b.round_kernels = (int)(fsp_kernel_launches() - before);
                note_launches(-b.round_kernels);  // counted when replayed
                if (rs != FSP_OK || ec != cudaSuccess || cudaGraphInstantiate(&b.round_exec, g, 0) != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return fail(rs != FSP_OK ? rs : FSP_ECUDA);
                }
                cudaGraphDestroy(g);
                b.round_rows = b.srows;
            }
            for (int r = 0; r < group; ++r) {
                note_launches(b.round_kernels);
                if (cudaGraphLaunch(b.round_exec, s) != cudaSuccess) return fail(FSP_ECUDA);
            }
        } else {
            const int k = (int)std::min<int64_t>(K, S);  // one round: S is current
            if (best_first && k < S) {
                // bins of the keys from the root bound to the incumbent; coarser
                // when the range is wide
                int shift = 0;
                const int64_t span = (int64_t)std::max(hst->best - root_lb, 1) * (n + 1);
                while ((span >> shift) >= kBestBins) ++shift;
                const int g = (int)std::min<int64_t>((S + 255) / 256, 1024);
                const int64_t T64 = (S + kTile - 1) / kTile;
                if (T64 > INT32_MAX - 1) return fail(FSP_ENOMEM);
                const int T = (int)T64, gt = (int)std::min<int64_t>(T64, 4096);
                st = grow_best(b);
                if (st != FSP_OK) return fail(st);
                const size_t ts = (size_t)b.tiles_cap + 1;
                int32_t *tcount = b.tiles, *tabove = b.tiles + ts, *out_cnt = b.tiles + 2 * ts,
                        *in_cnt = b.tiles + 3 * ts, *out_off = b.tiles + 4 * ts, *in_off = b.tiles + 5 * ts;
                note_launches(8);
                if (cudaMemsetAsync(b.hist, 0, sizeof(int32_t) * (kBestBins + 1), s) != cudaSuccess)
                    return fail(FSP_ECUDA);
                bnb_best_hist<<<g, 256, 0, s>>>(b.slb, b.sdep, S, n, root_lb, shift, b.hist);
                bnb_best_threshold<<<1, kScanThreads, 0, s>>>(b.hist, k, b.bs);
                bnb_best_tile_count<<<gt, kTile, 0, s>>>(b.slb, b.sdep, S, n, root_lb, shift, b.bs, tcount);
                bnb_best_tile_above<<<1, kScanThreads, 0, s>>>(tcount, T, tabove);
                bnb_best_mark<<<gt, kTile, 0, s>>>(b.slb, b.sdep, S, n, k, root_lb, shift, b.bs, tabove, T,
                                                   b.sel_flag, out_cnt, in_cnt);
                bnb_best_list_offsets<<<1, kScanThreads, 0, s>>>(out_cnt, in_cnt, T, out_off, in_off, b.bs);
                bnb_best_lists<<<gt, kTile, 0, s>>>(S, k, b.sel_flag, out_off, in_off, b.out_list, b.in_list);
                bnb_best_swap<<<(k + 7) / 8, 256, 0, s>>>(b.srows, b.sdep, b.slb, n, b.bs, b.out_list, b.in_list);
            }
            // child slots to bound: the popped parents' (a depth-first round
            // pops exactly k), or the counted children
            st = enqueue_round(async_rounds ? (int64_t)k * n : -1);
            if (st != FSP_OK) return fail(st);
            if (ended) {  // the state on the host is current
                S = hst->S;
                continue;
            }
        }
        if (cudaMemcpyAsync(hst, b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(FSP_ECUDA);
        st = take_device_status(inst);
        if (st != FSP_OK) return fail(st);
        S = hst->S;
        count = hst->count;
    }
    const bool found = hst->found != 0;
    const int32_t best = hst->best;
    if (found && best_perm &&
        cudaMemcpy(best_perm, b.best_row, sizeof(int16_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FSP_ECUDA);
    if (nodes_bounded) *nodes_bounded = count;
    b.release();
    cudaFreeHost(hst);
    cudaStreamDestroy(s);
    if (!found) return FSP_ENOTFOUND;
    if (best_makespan) *best_makespan = best;
    return FSP_OK;
}
