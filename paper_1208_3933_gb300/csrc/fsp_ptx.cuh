// fsp_ptx.cuh -- inline-PTX helpers shared by the bounding kernels:
// mbarrier init / expect-tx / bounded wait, the bulk (non-tensor)
// global->shared copy that stages Johnson-record tiles, and an L2 prefetch
// of a byte range (sm_90+ PTX, built for sm_103a).
#pragma once

#include <cstdint>

namespace fspgb {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity, giving up after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// One bulk (non-tensor) global->shared copy completing on an mbarrier.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Asks the memory system to bring the bytes [p, p + bytes) into L2 (a hint:
// nothing is loaded into registers).  Every address requested lies inside
// the range, so only lines that hold some of its bytes are touched.
__device__ __forceinline__ void prefetch_l2_range(const void *p, int bytes) {
    if (bytes <= 0) return;
    const char *c = static_cast<const char *>(p);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c));
    for (int o = 128 - (int)(reinterpret_cast<uintptr_t>(c) & 127); o < bytes; o += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// Writes a device-side error code to the instance's host-mapped status word.
__device__ __forceinline__ void report_status(int32_t *status, int32_t code) {
    if (status) {
        *reinterpret_cast<volatile int32_t *>(status) = code;
        __threadfence_system();
    }
}

// Double-buffered tile pipeline over a cyclic sequence of `ntiles` tiles:
// fill f goes to buffer f & 1 and completes phase f >> 1 of that buffer's
// mbarrier.  With ntiles <= 2 every tile has its own buffer and is staged
// once ("resident").  Thread 0 issues; `pending` tracks its copies in flight
// so a block that gives up can let them land before exiting.
struct TilePipe {
    uint64_t *bar;
    unsigned char *buf;
    uint32_t stride;
    bool resident;
    uint32_t fill = 0;
    uint32_t pending = 0, pend_par = 0;

    __device__ void issue(uint32_t f, const unsigned char *src, uint32_t bytes) {
        const uint32_t bi = f & 1;
        mbar_arrive_expect_tx(&bar[bi], bytes);
        bulk_g2s(buf + bi * stride, src, bytes, &bar[bi]);
        pending |= 1u << bi;
        pend_par = (pend_par & ~(1u << bi)) | (((f >> 1) & 1u) << bi);
    }

    // Buffer holding the tile consumed now (tile index t in resident mode).
    __device__ uint32_t current(int t) const { return resident ? (uint32_t)t : (fill & 1); }

    // Bounded wait for the tile consumed now; every thread calls it, and the
    // result is agreed across the block.
    __device__ bool wait(int t, long long limit) {
        const uint32_t bi = current(t);
        const uint32_t parity = resident ? 0u : ((fill >> 1) & 1u);
        const bool ok = mbar_wait_bounded(&bar[bi], parity, limit);
        const bool all = __syncthreads_and(ok) != 0;
        if (all) pending &= ~(1u << bi);
        return all;
    }

    // After a failed wait: thread 0 lets its issued copies land (bounded).
    __device__ void drain(long long limit) {
        for (uint32_t bi = 0; bi < 2; ++bi)
            if ((pending >> bi) & 1u) mbar_wait_bounded(&bar[bi], (pend_par >> bi) & 1u, limit);
    }
};

}  // namespace fspgb
