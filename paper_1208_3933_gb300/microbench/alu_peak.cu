// alu_peak.cu -- integer-pipe throughput probe for the roofline of the
// bounding kernel (an integer scan: no tensor-core or HBM bound applies).
//
// Every thread runs 8 independent chains for `iters` iterations of one
// instruction pattern, unrolled over 8 distinct operand pairs.  The host side
// converts the measured time into operations per SM per clock, using the SM
// clock read inside the kernel (clock64 against %globaltimer).
//   pattern 0: u = max(u + d_i, s_i)        (the bounding recurrence: add + max)
//   pattern 1: u = u + d_i                  (add)
//   pattern 2: u = (u ^ d_i) & s_i | d_i    (logic)
//   pattern 3: u = u * 3 + d_i              (integer multiply-add)
//   pattern 4: f = fmaxf(f + a_i, b_i)      (fp32 add + max)
#include <cuda_runtime.h>
#include <cstdint>

namespace {

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

template <int PAT>
__global__ void __launch_bounds__(256) alu_kernel(int iters, const int *seed, int *sink, long long *clk,
                                                  unsigned long long *ns) {
    int d[8], s[8], u[8];
    float fa[8], fb[8], fu[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        d[i] = seed[i] + threadIdx.x;
        s[i] = seed[8 + i] ^ blockIdx.x;
        u[i] = seed[16 + i] + i;
        fa[i] = (float)d[i];
        fb[i] = (float)s[i];
        fu[i] = (float)u[i];
    }
    __syncthreads();
    const long long c0 = clock64();
    const uint64_t t0 = gtimer();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int di = d[(i + k) & 7], si = s[(i + k) & 7];
                if (PAT == 0) u[i] = max(u[i] + di, si);
                if (PAT == 1) u[i] = u[i] + di;
                if (PAT == 2) u[i] = ((u[i] ^ di) & si) | di;
                if (PAT == 3) u[i] = u[i] * 3 + di;
                if (PAT == 4) fu[i] = fmaxf(fu[i] + fa[(i + k) & 7], fb[(i + k) & 7]);
            }
        }
    }
    __syncthreads();
    const long long c1 = clock64();
    const uint64_t t1 = gtimer();
    int acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += u[i] + (int)fu[i];
    if (acc == 0x7fffffff) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        clk[blockIdx.x] = c1 - c0;
        ns[blockIdx.x] = t1 - t0;
    }
}

}  // namespace

// Runs pattern `pat` on `blocks` x 256 threads; returns the elapsed event time
// in *ms, the mean SM clock in MHz in *mhz, and the operations per thread in
// *ops_per_thread (instructions of the pattern, 2 for add+max).
extern "C" int fsp_microbench_alu(int pat, int blocks, int iters, float *ms, float *mhz, double *ops_per_thread) {
    int *seed = nullptr, *sink = nullptr;
    long long *clk = nullptr;
    unsigned long long *ns = nullptr;
    int hs[24];
    for (int i = 0; i < 24; ++i) hs[i] = (i * 7919) % 97 + 1;
    if (cudaMalloc(&seed, sizeof(hs)) || cudaMalloc(&sink, sizeof(int) * blocks * 256) ||
        cudaMalloc(&clk, sizeof(long long) * blocks) || cudaMalloc(&ns, sizeof(unsigned long long) * blocks))
        return -2;
    cudaMemcpy(seed, hs, sizeof(hs), cudaMemcpyHostToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        switch (pat) {
            case 0: alu_kernel<0><<<blocks, 256>>>(iters, seed, sink, clk, ns); break;
            case 1: alu_kernel<1><<<blocks, 256>>>(iters, seed, sink, clk, ns); break;
            case 2: alu_kernel<2><<<blocks, 256>>>(iters, seed, sink, clk, ns); break;
            case 3: alu_kernel<3><<<blocks, 256>>>(iters, seed, sink, clk, ns); break;
            default: alu_kernel<4><<<blocks, 256>>>(iters, seed, sink, clk, ns); break;
        }
    };
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : -3;
    cudaEventElapsedTime(ms, e0, e1);
    long long *hc = new long long[blocks];
    unsigned long long *hn = new unsigned long long[blocks];
    cudaMemcpy(hc, clk, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    cudaMemcpy(hn, ns, sizeof(unsigned long long) * blocks, cudaMemcpyDeviceToHost);
    double sc = 0, sn = 0;
    for (int b = 0; b < blocks; ++b) {
        sc += (double)hc[b];
        sn += (double)hn[b];
    }
    *mhz = (float)(sn > 0 ? sc / sn * 1e3 : 0.0);
    const double per = (pat == 0 || pat == 4) ? 2.0 : (pat == 2 ? 2.0 : 1.0);
    *ops_per_thread = per * 64.0 * (double)iters;
    delete[] hc;
    delete[] hn;
    cudaFree(seed);
    cudaFree(sink);
    cudaFree(clk);
    cudaFree(ns);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
