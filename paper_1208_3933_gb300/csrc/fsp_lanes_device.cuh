// fsp_lanes_device.cuh -- device building blocks of the couple-lanes
// bounding kernels (fsp_bound_lanes.cu: one pool; fsp_batch.cu: many pools of
// many instances in one persistent launch).  See fsp_bound_lanes.cu for the
// method and the data layout.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fsp_internal.h"
#include "fsp_plan.h"

namespace fspgb {



constexpr unsigned kFull = 0xffffffffu;

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

// Minimum over the unscheduled jobs of one machine's head (or tail) sums for
// the warp's 32 nodes (lane = node): `sorted` lists (job, sum) by ascending
// sum, so the answer is the sum of the first listed job whose flag bit is
// set.  32 list entries are examined per step, one per lane; the transposed
// flag words give every node the lanes that hit, and the first hit's sum is
// shuffled in.  Nodes already `settled` get 0.
__device__ __forceinline__ int first_unscheduled(const int2 *__restrict__ sorted, const uint32_t *F, int n, int lane,
                                                 bool settled) {
    int result = 0;
    bool done = settled;
    for (int base = 0; base < n && __any_sync(kFull, !done); base += 32) {
        const int pos = base + lane;
        int2 e = make_int2(0, 0);
        uint32_t w = 0;
        if (pos < n) {
            e = __ldg(sorted + pos);
            w = F[e.x];
        }
        const uint32_t hits = warp_transpose32(w, lane);
        const int first = __ffs(hits) - 1;
        const int val = __shfl_sync(kFull, e.y, first < 0 ? 0 : first);
        if (!done && first >= 0) {
            result = val;
            done = true;
        }
    }
    return result;
}

// Setup of node x (lane = node) for the warp's 32 nodes: the flag words F[j]
// (bit b: job j unscheduled in the warp's node b), the lane's row
// (A_k = r_k + S_k as int32, q_l as int16) and the one-machine term
// max_{l>=1} (A_l + q_l).  Returns whether the row is valid.
template <int MP>
__device__ __forceinline__ bool lanes_setup(const LanesArgs &a, int64_t x, int lane, uint32_t *F, int32_t *myrow,
                                            int &bterm) {
    const int n = a.n, m = a.m;
    bool valid = false;
    int d = 0;
    if (x < a.N) {
        d = __ldg(a.depths + x);
        valid = (d >= 0 && d <= n);
    }
    const uint32_t vmask = __ballot_sync(kFull, valid);
    for (int j = lane; j < n; j += 32) F[j] = vmask;
    __syncwarp();
    const int16_t *row = a.nodes + x * (int64_t)n;
    // (1) clear the prefix jobs' flag bits; a job outside [0,n) or seen twice
    // invalidates the row (no branch on the loop's critical path)
    {
        const int dv = valid ? d : 0;
        bool bad = false;
#pragma unroll 4
        for (int i = 0; i < dv; ++i) {
            const int j = __ldg(row + i);
            const bool inr = (unsigned)j < (unsigned)n;
            const uint32_t old = atomicAnd(&F[inr ? j : 0], inr ? ~(1u << lane) : kFull);
            bad |= !inr || !((old >> lane) & 1u);
        }
        valid = valid && !bad;
    }
    // (2) C(sigma,k) by the flow-shop recurrence, and the prefix column sums;
    // one step is max(c + p, C_k + p), a single fused add-max
    int C[MP], Ps[MP];
#pragma unroll
    for (int k = 0; k < MP; ++k) {
        C[k] = 0;
        Ps[k] = 0;
    }
    if (valid) {
#pragma unroll 4
        for (int i = 0; i < d; ++i) {
            const int j = __ldg(row + i);
            const int4 *pj = reinterpret_cast<const int4 *>(a.pp + (size_t)j * a.mpad);
            int c = 0;
#pragma unroll
            for (int q = 0; q < MP / 4; ++q) {
                if (4 * q >= a.mpad) break;
                const int4 v = __ldg(pj + q);
                const int pv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = 4 * q + e;
                    c = __viaddmax_s32(c, pv[e], C[k] + pv[e]);
                    C[k] = c;
                    Ps[k] += pv[e];
                }
            }
        }
    }
    __syncwarp();
    // (3) A_k = max(C_k, min_U head) + (ptot_k - prefix sum), q_l = min_U tail
    const bool settled = !valid || d == n;  // nothing to search for
    int16_t *qrow = reinterpret_cast<int16_t *>(myrow + m);
    bterm = 0;
#pragma unroll
    for (int k = 0; k < MP; ++k) {
        if (k < m) {
            const int mh = k > 0 ? first_unscheduled(a.hsort + (size_t)k * n, F, n, lane, settled) : 0;
            const int Ak = max(C[k], mh) + (__ldg(a.ptot + k) - Ps[k]);
            const int ql = k < m - 1 ? first_unscheduled(a.tsort + (size_t)k * n, F, n, lane, settled) : 0;
            myrow[k] = Ak;
            qrow[k] = (int16_t)ql;
            if (k >= 1) bterm = max(bterm, Ak + ql);
        }
    }
    __syncwarp();
    return valid;
}

// One couple group's scan over positions [0, npos) of a record tile (lane =
// couple): fp32 slack for 32-bit records, int32 for 128-bit records.
__device__ __forceinline__ void scan_compact(const uint32_t *R, int npos, const uint32_t *F, float (&u)[32]) {
#pragma unroll 2
    for (int i = 0; i < npos; ++i) {
        const uint32_t r = R[i * 32];
        const uint32_t fw = F[r & 1023u];
        // exact int -> float for 0 <= v < 2^23 via the exponent of 2^23
        const float sf = __int_as_float(0x4B000000 | ((r >> 10) & 8191u)) - 8388608.0f;
        const float df = __int_as_float(0x4B000000 | (uint32_t)(((int)r >> 23) + 256)) - 8388864.0f;
#pragma unroll
        for (int b = 0; b < 32; ++b)
            if ((fw >> b) & 1u) u[b] = fmaxf(u[b] + df, sf);
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

template <typename U>
__device__ __forceinline__ void couple_epilogue(const int32_t *AQ, int stride, int m, int kk, int ll, const U (&u)[32],
                                                int (&lb)[32]) {
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const int32_t *rb = AQ + b * stride;
        const int base = rb[kk] + reinterpret_cast<const int16_t *>(rb + m)[ll];
        lb[b] = max(lb[b], base + (int)u[b]);
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



}  // namespace fspgb
