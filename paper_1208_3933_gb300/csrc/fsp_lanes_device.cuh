// fsp_lanes_device.cuh -- device building blocks of the couple-lanes
// bounding kernels (fsp_bound_lanes.cu: one pool; fsp_batch.cu: many pools of
// many instances in one persistent launch).  See fsp_bound_lanes.cu for the
// method and the data layout.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "fsp_internal.h"
#include "fsp_plan.h"
#include "fsp_ptx.cuh"

namespace fspgb {



constexpr unsigned kFull = 0xffffffffu;

// The node bounded in slot i of a launch (slots past N map to themselves).
__device__ __forceinline__ int64_t node_at(const LanesArgs &a, int64_t i) {
    return (a.order && i < a.N) ? (int64_t)__ldg(a.order + i) : i;
}

// 32x32 bit-matrix transpose across a warp: on entry lane L holds row L
// (bit b = M[L][b]); on exit lane b holds column b (bit L = M[L][b]).  Five
// butterfly stages, each swapping the off-diagonal halves of every block.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    uint32_t mask = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t y = __shfl_xor_sync(kFull, x, j);
        x = (lane & j) ? ((x & ~mask) | ((y >> j) & mask)) : ((x & mask) | ((y & mask) << j));
        mask ^= mask << (j >> 1);
    }
    return x;
}

// The latency q_l of a node row (after the m values A_k): int16 for
// instances with compact records (every tail is below 2^15 there), int32
// otherwise.
__device__ __forceinline__ void store_q(int32_t *row, int m, int l, int v, bool q32) {
    if (q32)
        row[m + l] = v;
    else
        reinterpret_cast<int16_t *>(row + m)[l] = (int16_t)v;
}

__device__ __forceinline__ int load_q(const int32_t *row, int m, int l, bool q32) {
    return q32 ? row[m + l] : (int)reinterpret_cast<const int16_t *>(row + m)[l];
}

// NV bit-matrix transposes at once (as warp_transpose32, one matrix per
// value): the five shuffle stages are interleaved across the values, so a
// stage's NV shuffles are in flight together instead of one chain at a time.
template <int NV>
__device__ __forceinline__ void warp_transpose32_n(uint32_t (&x)[NV], int lane) {
    uint32_t mask = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        uint32_t y[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) y[v] = __shfl_xor_sync(kFull, x[v], j);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            x[v] = (lane & j) ? ((x[v] & ~mask) | ((y[v] >> j) & mask)) : ((x[v] & mask) | ((y[v] & mask) << j));
        mask ^= mask << (j >> 1);
    }
}

// Where the setup reads the processing-time rows (lanes_setup's PS).
constexpr int kPtabNone = 0, kPtabByte = 1;

// Machines of the minima search handled together (MP is a multiple of 4).
constexpr int kMinimaChunk = 4;
// Nodes with at most this many unscheduled jobs take their minima by walking
// those jobs (instances of at most kWalkMaxMP padded machines).
constexpr int kWalkMinima = 32;
constexpr int kWalkMaxMP = 20;

// Copies the first 32 entries of every machine's head- and tail-sorted job
// lists into shared memory ([m][32] each; entries past n read (0,0)).
__device__ __forceinline__ void load_sorted_heads(const LanesArgs &a, int2 *hcache, int2 *tcache) {
    for (int i = threadIdx.x; i < a.m * 32; i += blockDim.x) {
        const int k = i >> 5, pos = i & 31;
        hcache[i] = pos < a.n ? a.hsort[(size_t)k * a.n + pos] : make_int2(0, 0);
        tcache[i] = pos < a.n ? a.tsort[(size_t)k * a.n + pos] : make_int2(0, 0);
    }
}

// Setup of node x (lane = node) for the warp's 32 nodes: the flag words F[j]
// (bit b: job j unscheduled in the warp's node b; F holds 32 * ceil(n / 32)
// words, which first hold the lanes' membership bitmaps), the lane's row
// (A_k = r_k + S_k as int32, then q_l, see store_q) and the one-machine term
// max_{l>=1} (A_l + q_l).  Returns whether the row is valid.  PS says where
// the processing-time rows are read: kPtabNone from pp in global memory,
// kPtabByte from ptab, the block's shared-memory copy of pp as bytes
// ([n][mpad] uint8, compact instances only: every p < 256), a quarter of the
// shared-memory traffic of an int32 copy for one byte extract per value.
template <int MP, int PS = kPtabNone>
__device__ __forceinline__ bool lanes_setup(const LanesArgs &a, int64_t x, int lane, uint32_t *F, int32_t *myrow,
                                            int &bterm, const int2 *hcache = nullptr,
                                            const int2 *tcache = nullptr, const void *ptab = nullptr) {
    const int n = a.n, m = a.m, nw = (n + 31) >> 5;
    // job j's row of processing times (kPtabByte: words of four bytes)
    auto prow = [&](int j) {
        if constexpr (PS == kPtabByte)
            return static_cast<const uint32_t *>(ptab) + (size_t)j * (a.mpad >> 2);
        else
            return reinterpret_cast<const int4 *>(a.pp + (size_t)j * a.mpad);
    };
    // machines 4q .. 4q+3 of a row; columns past the instance's own padding
    // read as zeros (no branch)
    auto pld = [&](auto r, int q) {
        const bool in = 4 * q < a.mpad;
        if constexpr (PS == kPtabByte) {
            const uint32_t w = in ? r[q] : 0u;
            return make_int4((int)__byte_perm(w, 0u, 0x4440u), (int)__byte_perm(w, 0u, 0x4441u),
                             (int)__byte_perm(w, 0u, 0x4442u), (int)__byte_perm(w, 0u, 0x4443u));
        } else {
            return in ? __ldg(r + q) : make_int4(0, 0, 0, 0);
        }
    };
    bool valid = false;
    int d = 0;
    if (x < a.N) {
        d = __ldg(a.depths + x);
        valid = (d >= 0 && d <= n);
    }
    // (1) one pass over the prefix.  Membership: each lane marks its node's
    // jobs in a private bitmap (word w of lane L at F[32 w + L], so the 32
    // lanes never share a word) with an atomic OR whose result is not read,
    // so the marks form no chain of dependent shared-memory reads; a job
    // outside [0,n) invalidates the row, and so does a job marked twice,
    // found afterwards as fewer marked bits than the depth.  Recurrence:
    // C(sigma,k) by the flow-shop recurrence and the prefix column sums, one
    // step max(c + p, C_k + p) = a single fused add-max.  An invalid row
    // still runs the loop on clamped jobs; its result is discarded.
    for (int w = 0; w < nw; ++w) F[w * 32 + lane] = 0u;
    int C[MP], Ps[MP];
#pragma unroll
    for (int k = 0; k < MP; ++k) {
        C[k] = 0;
        Ps[k] = 0;
    }
    const int16_t *row = a.nodes + x * (int64_t)n;
    const int dv = valid ? d : 0;
    // the lines of the prefix are requested from DRAM at once; the pass
    // below then waits on L2, not on one DRAM round trip per four jobs
    prefetch_l2_range(row, 2 * dv);
    bool bad = false;
    // membership of job j (clamped into range: an invalid row is discarded)
    auto mark = [&](int j) {
        const bool inr = (unsigned)j < (unsigned)n;
        const int jj = inr ? j : 0;
        bad |= !inr;
        atomicOr(F + (jj >> 5) * 32 + lane, 1u << (jj & 31));
        return jj;
    };
    // four consecutive jobs: machine k of job t needs job t's machine k-1 and
    // job t-1's machine k, so the four recurrences run as a wavefront (23
    // dependent steps for 20 machines instead of 80) and their processing
    // times are loaded together
    auto take4 = [&](int j0, int j1, int j2, int j3) {
        const auto p0 = prow(mark(j0));
        const auto p1 = prow(mark(j1));
        const auto p2 = prow(mark(j2));
        const auto p3 = prow(mark(j3));
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
        for (int q = 0; q < MP / 4; ++q) {
            const int4 v0 = pld(p0, q), v1 = pld(p1, q), v2 = pld(p2, q), v3 = pld(p3, q);
            const int q0[4] = {v0.x, v0.y, v0.z, v0.w}, q1[4] = {v1.x, v1.y, v1.z, v1.w};
            const int q2[4] = {v2.x, v2.y, v2.z, v2.w}, q3[4] = {v3.x, v3.y, v3.z, v3.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * q + e;
                c0 = __viaddmax_s32(c0, q0[e], C[k] + q0[e]);
                c1 = __viaddmax_s32(c1, q1[e], c0 + q1[e]);
                c2 = __viaddmax_s32(c2, q2[e], c1 + q2[e]);
                c3 = __viaddmax_s32(c3, q3[e], c2 + q3[e]);
                C[k] = c3;
                Ps[k] += (q0[e] + q1[e]) + (q2[e] + q3[e]);
            }
        }
    };
    auto take = [&](int j) {
        const auto pj = prow(mark(j));
        int c = 0;
#pragma unroll
        for (int q = 0; q < MP / 4; ++q) {
            const int4 v = pld(pj, q);
            const int pv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * q + e;
                c = __viaddmax_s32(c, pv[e], C[k] + pv[e]);
                C[k] = c;
                Ps[k] += pv[e];
            }
        }
    };
    int i = 0;
    if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(a.nodes) & 7) == 0) {  // 8-byte aligned rows: four jobs per load
        // the next four jobs are loaded while these four are taken
        const int2 *row4 = reinterpret_cast<const int2 *>(row);
        int2 v = i + 4 <= dv ? __ldg(row4) : make_int2(0, 0);
#pragma unroll 1
        for (; i + 4 <= dv; i += 4) {
            const int2 nv = i + 8 <= dv ? __ldg(row4 + (i >> 2) + 1) : make_int2(0, 0);
            take4((int)(int16_t)(v.x & 0xFFFF), v.x >> 16, (int)(int16_t)(v.y & 0xFFFF), v.y >> 16);
            v = nv;
        }
    }
#pragma unroll 1
    for (; i < dv; ++i) take(__ldg(row + i));
    __syncwarp();
    {  // a job marked twice leaves fewer marked bits than the depth
        int cnt = 0;
        for (int w = 0; w < nw; ++w) cnt += __popc(F[w * 32 + lane]);
        bad |= cnt != dv;
    }
    valid = valid && !bad;
    // S_k = ptot_k - prefix sum of machine k, kept in the lane's row until
    // A_k = r_k + S_k replaces it
#pragma unroll
    for (int k = 0; k < MP; ++k)
        if (k < m) myrow[k] = __ldg(a.ptot + k) - Ps[k];
    // Per-job release times (when the instance asks for them): RM of
    // Section II-D read as the earliest start of every unscheduled job j on
    // every machine k after the prefix, est_j0 = C_0 and
    // est_jk = max(est_j,k-1 + p_j,k-1, C_k) (one fused add-max), and
    // r_k = min over U of est_jk (r_k = C_k once U is empty).  The lane walks
    // its node's unscheduled jobs in its own membership bitmap.
    const bool per_job = a.release != 0;
    int R[MP];
    if (per_job) {
#pragma unroll
        for (int k = 0; k < MP; ++k) R[k] = C[k];
        if (valid && d < n) {
#pragma unroll
            for (int k = 0; k < MP; ++k) R[k] = INT_MAX;
            for (int w = 0; w < nw; ++w) {
                uint32_t un = ~F[w * 32 + lane];
                if (w == nw - 1 && (n & 31)) un &= (1u << (n & 31)) - 1u;
                while (un) {
                    const int j = w * 32 + __ffs(un) - 1;
                    un &= un - 1u;
                    const auto pj = prow(j);
                    int est = C[0], prev = 0;
#pragma unroll
                    for (int q = 0; q < MP / 4; ++q) {
                        const int4 v = pld(pj, q);
                        const int pv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int k = 4 * q + e;
                            if (k > 0) est = __viaddmax_s32(est, prev, C[k]);
                            R[k] = min(R[k], est);
                            prev = pv[e];
                        }
                    }
                }
            }
        }
    }
    // Deep nodes (at most kWalkMinima unscheduled jobs): the release and
    // latency minima are taken by walking the node's own unscheduled jobs in
    // its bitmap, min over U of sum_{h<k} p_jh and of sum_{h>k} p_jh, for
    // every machine at once.  The sorted lists below would find them only
    // after many rounds, when nearly every listed job is scheduled.  The
    // minima kept in registers limit this to instances of at most kWalkMaxMP
    // (padded) machines.
    const bool walk = MP <= kWalkMaxMP && valid && d < n && n - d <= kWalkMinima;
    int MH[MP <= kWalkMaxMP ? MP : 1], MQ[MP <= kWalkMaxMP ? MP : 1];
    if constexpr (MP <= kWalkMaxMP) {
#pragma unroll
        for (int k = 0; k < MP; ++k) {
            MH[k] = INT_MAX;
            MQ[k] = INT_MAX;
        }
        if (walk) {
            for (int w = 0; w < nw; ++w) {
                uint32_t un = ~F[w * 32 + lane];
                if (w == nw - 1 && (n & 31)) un &= (1u << (n & 31)) - 1u;
                while (un) {
                    const int j = w * 32 + __ffs(un) - 1;
                    un &= un - 1u;
                    const auto pj = prow(j);
                    int pv[MP];
#pragma unroll
                    for (int q = 0; q < MP / 4; ++q) {
                        const int4 v = pld(pj, q);
                        pv[4 * q] = v.x;
                        pv[4 * q + 1] = v.y;
                        pv[4 * q + 2] = v.z;
                        pv[4 * q + 3] = v.w;
                    }
                    int rowsum = 0;
#pragma unroll
                    for (int k = 0; k < MP; ++k) rowsum += pv[k];  // padding columns are zero
                    int head = 0;
#pragma unroll
                    for (int k = 0; k < MP; ++k) {
                        MH[k] = min(MH[k], head);
                        MQ[k] = min(MQ[k], rowsum - head - pv[k]);
                        head += pv[k];
                    }
                }
            }
        }
    }
    // (2) the flag words: transposing lane L's bitmap word w gives lane i the
    // bits over nodes of job 32 w + i; F[j] bit b = job j unscheduled in the
    // warp's node b (valid nodes only)
    const uint32_t vmask = __ballot_sync(kFull, valid);
    for (int w = 0; w < nw; ++w) {
        const uint32_t t = warp_transpose32(F[w * 32 + lane], lane);
        F[w * 32 + lane] = ~t & vmask;
    }
    __syncwarp();
    // (3) A_k = max(C_k, min_U head) + S_k (per-job release times: r_k + S_k),
    // q_l = min_U tail.
    // Each machine's (job, head) and (job, tail) lists are sorted by sum, so
    // a minimum over U is the sum of the first listed job that is unscheduled
    // in the node.  A round examines 32 list entries per machine, one per
    // lane: the transposed flag words give every node the lanes that hit, and
    // the first hit's sum is shuffled in.  Round 0 covers the 32 cheapest
    // entries (from the shared-memory copy when given); nodes whose entries
    // were all scheduled go on round by round.
    const bool settled = !valid || d == n || walk;  // nothing to search for
    const bool q32 = a.q32 != 0;
    uint32_t open_h = 0, open_t = 0;  // machines still searching (bit k)
    const bool in = lane < n;
    constexpr int CH = kMinimaChunk;
    // A warp whose nodes all have their minima already (walked, complete or
    // invalid) skips the list search: round 0 would only confirm them.
    const bool all_settled = __all_sync(kFull, settled);
    if (all_settled) {
#pragma unroll
        for (int k = 0; k < MP; ++k) {
            if (k < m) {
                int mh = 0, ql = 0;
                if constexpr (MP <= kWalkMaxMP) {
                    if (walk) {
                        mh = MH[k];
                        ql = MQ[k];
                    }
                }
                myrow[k] = (per_job ? R[k] : max(C[k], mh)) + myrow[k];
                store_q(myrow, m, k, ql, q32);
            }
        }
    }
    // Machines are taken kMinimaChunk at a time: their list entries and flag
    // words are loaded together and their transposes interleaved.
#pragma unroll
    for (int k0 = 0; k0 < MP; k0 += CH) {
        if (!all_settled && k0 < m) {
            int2 eh[CH], et[CH];
            uint32_t w[2 * CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = k0 + c;
                // heads are 0 on machine 0 and not needed with per-job release
                // times; tails are 0 on machine m-1
                const bool want_h = in && k < m && k > 0 && !per_job, want_t = in && k < m - 1;
                eh[c] = make_int2(0, 0);
                et[c] = make_int2(0, 0);
                if (want_h) eh[c] = hcache ? hcache[k * 32 + lane] : __ldg(a.hsort + (size_t)k * n + lane);
                if (want_t) et[c] = tcache ? tcache[k * 32 + lane] : __ldg(a.tsort + (size_t)k * n + lane);
                w[2 * c] = want_h ? F[eh[c].x] : 0u;
                w[2 * c + 1] = want_t ? F[et[c].x] : 0u;
            }
            warp_transpose32_n<2 * CH>(w, lane);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = k0 + c;
                const bool want_h = k < m && k > 0 && !per_job, want_t = k < m - 1;
                const int fh = __ffs(w[2 * c]) - 1, ft = __ffs(w[2 * c + 1]) - 1;
                const int vh = __shfl_sync(kFull, eh[c].y, fh < 0 ? 0 : fh);
                const int vt = __shfl_sync(kFull, et[c].y, ft < 0 ? 0 : ft);
                if (k < m) {
                    int mh = (!settled && fh >= 0) ? vh : 0;
                    int ql = (!settled && ft >= 0) ? vt : 0;
                    if constexpr (MP <= kWalkMaxMP) {
                        if (walk) {
                            mh = MH[k];
                            ql = MQ[k];
                        }
                    }
                    if (want_h && !settled && fh < 0)
                        open_h |= 1u << k;  // A_k once a later round finds the minimum
                    else
                        myrow[k] = (per_job ? R[k] : max(C[k], mh)) + myrow[k];
                    if (want_t && !settled && ft < 0) open_t |= 1u << k;
                    store_q(myrow, m, k, ql, q32);
                }
            }
        }
    }
    // later rounds: list entries [base, base + 32) of every machine some node
    // still searches, the machines taken as in round 0
    for (int base = 32; base < n; base += 32) {
        const uint32_t any_h = __reduce_or_sync(kFull, open_h), any_t = __reduce_or_sync(kFull, open_t);
        if ((any_h | any_t) == 0u) break;
        const int pos = base + lane;
        const bool inr = pos < n;
#pragma unroll
        for (int k0 = 0; k0 < MP; k0 += CH) {
            if (k0 < m && (((any_h | any_t) >> k0) & ((1u << CH) - 1u))) {
                int2 eh[CH], et[CH];
                uint32_t w[2 * CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int k = k0 + c;
                    const bool lh = inr && k < m && ((any_h >> k) & 1u), lt = inr && k < m && ((any_t >> k) & 1u);
                    eh[c] = make_int2(0, 0);
                    et[c] = make_int2(0, 0);
                    if (lh) eh[c] = __ldg(a.hsort + (size_t)k * n + pos);
                    if (lt) et[c] = __ldg(a.tsort + (size_t)k * n + pos);
                    w[2 * c] = lh ? F[eh[c].x] : 0u;
                    w[2 * c + 1] = lt ? F[et[c].x] : 0u;
                }
                warp_transpose32_n<2 * CH>(w, lane);
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int k = k0 + c;
                    const int fh = __ffs(w[2 * c]) - 1, ft = __ffs(w[2 * c + 1]) - 1;
                    const int vh = __shfl_sync(kFull, eh[c].y, fh < 0 ? 0 : fh);
                    const int vt = __shfl_sync(kFull, et[c].y, ft < 0 ? 0 : ft);
                    if (k < m) {
                        if (((open_h >> k) & 1u) && fh >= 0) {
                            myrow[k] = max(C[k], vh) + myrow[k];
                            open_h &= ~(1u << k);
                        }
                        if (((open_t >> k) & 1u) && ft >= 0) {
                            store_q(myrow, m, k, vt, q32);
                            open_t &= ~(1u << k);
                        }
                    }
                }
            }
        }
    }
    bterm = 0;
    for (int l = 1; l < m; ++l) bterm = max(bterm, myrow[l] + load_q(myrow, m, l, q32));
    __syncwarp();
    return valid;
}

// Copies pp ([n][mpad] int32, mpad a multiple of 4, every entry < 256) into
// the block's shared-memory table as bytes, four machines to a word (machine
// 4q + e in byte e of word q); every thread of the block takes part, the
// caller synchronises before the table is read.
__device__ __forceinline__ void load_ptab(const LanesArgs &a, void *ptab) {
    const int4 *src = reinterpret_cast<const int4 *>(a.pp);
    uint32_t *dst = static_cast<uint32_t *>(ptab);
    const int nq = a.n * a.mpad / 4;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        const int4 v = __ldg(src + i);
        dst[i] = (uint32_t)v.x | ((uint32_t)v.y << 8) | ((uint32_t)v.z << 16) | ((uint32_t)v.w << 24);
    }
}

// One slack update of the 32 nodes for a couple-lanes record r (the
// two-word encoding of fsp_internal.h): r.x is 1024 s + j, r.y is
// 1024 delta; then u_b = max(u_b + 1024 delta, 1024 s + j) for every node b
// whose flag bit for job j is set, one fused integer add-max.  The slack is
// thus kept as 1024 u plus the job bits of the last record that won a max:
// a sum only ever adds 1024 delta, which keeps those low bits, and a max of
// two such values decides as their integer parts do (or ties on them), so
// u_b >> 10 follows the integer recurrence exactly.
__device__ __forceinline__ void lanes_step(uint2 r, const uint32_t *F, int (&u)[32]) {
    const uint32_t fw = F[r.x & 1023u];
    const int sv = (int)r.x, dv = (int)r.y;
#pragma unroll
    for (int b = 0; b < 32; ++b)
        if ((fw >> b) & 1u) u[b] = __viaddmax_s32(u[b], dv, sv);
}

// One couple group's scan over positions [0, npos) of a record tile (lane =
// couple): scaled slack for two-word records, plain int32 for 128-bit ones.
// npos is a multiple of 4 (couple rows are padded to 4 entries and tiles hold
// multiples of 4 positions), so the loop takes four positions a round with
// no remainder.
__device__ __forceinline__ void scan_compact(const uint2 *R, int npos, const uint32_t *F, int (&u)[32]) {
#pragma unroll 1
    for (int i = 0; i < npos; i += 4) {
        const uint2 r0 = R[i * 32], r1 = R[(i + 1) * 32], r2 = R[(i + 2) * 32], r3 = R[(i + 3) * 32];
        lanes_step(r0, F, u);
        lanes_step(r1, F, u);
        lanes_step(r2, F, u);
        lanes_step(r3, F, u);
    }
}

__device__ __forceinline__ void scan_wide(const int4 *R, int npos, const uint32_t *F, int (&u)[32]) {
#pragma unroll 1
    for (int i = 0; i < npos; ++i) {
        const int4 r = R[i * 32];
        const uint32_t fw = F[r.x];
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if ((fw >> b) & 1u) u[b] = max(u[b] + r.z, r.y);
    }
}

// A lane's couple values A_k + q_l + u_b folded into lb.  Q32 marks 128-bit
// records: their rows hold q as int32 (store_q) and their slack is plain;
// compact records keep q as int16 and the slack scaled by 1024 (lanes_step).
template <bool Q32>
__device__ __forceinline__ void couple_epilogue(const int32_t *AQ, int stride, int m, int kk, int ll,
                                                const int (&u)[32], int (&lb)[32]) {
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const int32_t *rb = AQ + b * stride;
        const int base = rb[kk] + load_q(rb, m, ll, Q32);
        lb[b] = max(lb[b], base + (Q32 ? u[b] : (u[b] >> 10)));
    }
}

// transpose-max: afterwards lane b holds max over the warp's lanes of lb[b]
__device__ __forceinline__ int transpose_max(int (&lb)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const int send = upper ? lb[i] : lb[i + w];
            const int keep = upper ? lb[i + w] : lb[i];
            lb[i] = max(keep, __shfl_xor_sync(kFull, send, w));
        }
    }
    return lb[0];
}



// Two node sets per warp, 28 nodes each (flag bits 7, 15, 23 and 31 unused):
// the 28 predicates of a flag word come from the low seven bits of its four
// bytes, which the hardware turns into predicates a byte at a time, and one
// record and one job index serve 56 nodes.  Bit b (b & 7 != 7) of a set's
// flag word is its node set28_slot(b) in 0..27.
constexpr uint32_t kSet28 = 0x7f7f7f7fu;
__host__ __device__ constexpr int set28_slot(int b) { return b - (b >> 3); }

// lanes_step for NS sets of 28 (1 or 2): F0 and F1 are their flag words (F1
// unread for one set), u[0..27] and u[28..55] their slacks.
template <int NS>
__device__ __forceinline__ void lanes_step28(uint2 r, const uint32_t *F0, const uint32_t *F1, int (&u)[28 * NS]) {
    const uint32_t j = r.x & 1023u;
    const int sv = (int)r.x, dv = (int)r.y;
#pragma unroll
    for (int set = 0; set < NS; ++set) {
        const uint32_t f = (set ? F1 : F0)[j];
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if ((kSet28 >> b) & 1u)
                if ((f >> b) & 1u) u[28 * set + set28_slot(b)] = __viaddmax_s32(u[28 * set + set28_slot(b)], dv, sv);
    }
}

// npos is a multiple of 4, as in scan_compact.
template <int NS>
__device__ __forceinline__ void scan_compact28(const uint2 *R, int npos, const uint32_t *F0, const uint32_t *F1,
                                               int (&u)[28 * NS]) {
#pragma unroll 1
    for (int i = 0; i < npos; i += 4) {
        const uint2 r0 = R[i * 32], r1 = R[(i + 1) * 32], r2 = R[(i + 2) * 32], r3 = R[(i + 3) * 32];
        lanes_step28<NS>(r0, F0, F1, u);
        lanes_step28<NS>(r1, F0, F1, u);
        lanes_step28<NS>(r2, F0, F1, u);
        lanes_step28<NS>(r3, F0, F1, u);
    }
}

// One couple group's values A_k + q_l + u of the 28-node set whose slacks
// start at u[OFF], reduced over the warp's lanes (couples): lane b receives
// the maximum for the set's node in bit b (0 in the unused lanes).  Compact
// records only (int16 latencies, slack scaled by 1024).
template <int OFF, int NU>
__device__ __forceinline__ int set28_group_max(const int32_t *AQ, int stride, int m, int kk, int ll,
                                               const int (&u)[NU], int lane) {
    int v[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        if ((kSet28 >> b) & 1u) {
            const int32_t *rb = AQ + b * stride;
            v[b] = rb[kk] + load_q(rb, m, ll, false) + (u[OFF + set28_slot(b)] >> 10);
        } else {
            v[b] = 0;
        }
    }
    return transpose_max(v, lane);
}

}  // namespace fspgb
