// fsp_instance.cpp -- builds and uploads the per-instance tables of
// Section II-D (PTM, LM, JM, MM and the head/tail sums behind RM and QM).
// The paper computes the lags and Johnson orders "once at the beginning of
// the algorithm"; so does fsp_instance_create, in O(P n log n) host work.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include "fsp_internal.h"

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Johnson's rule on couple (k,l) with lags (Johnson 1954, generalised with
// lags by Lageweg, Lenstra and Rinnooy Kan; Section II-C): with
// a_j = p_jk + lag_j and b_j = p_jl + lag_j, first the jobs with
// p_jk <= p_jl by ascending a_j, then the others by descending b_j.  Ties
// are broken by job index so the table is reproducible.
void johnson_order(int n, int m, const int32_t *p, int k, int l, std::vector<int64_t> &lag,
                   std::vector<int32_t> &order) {
    struct Item {
        int grp;
        int64_t key;
        int32_t job;
    };
    std::vector<Item> it(n);
    for (int j = 0; j < n; ++j) {
        int64_t lg = 0;
        for (int h = k + 1; h < l; ++h) lg += p[j * m + h];
        lag[j] = lg;
        const int64_t a = p[j * m + k] + lg, b = p[j * m + l] + lg;
        if (p[j * m + k] <= p[j * m + l])
            it[j] = {0, a, j};
        else
            it[j] = {1, -b, j};
    }
    std::sort(it.begin(), it.end(), [](const Item &x, const Item &y) {
        if (x.grp != y.grp) return x.grp < y.grp;
        if (x.key != y.key) return x.key < y.key;
        return x.job < y.job;
    });
    for (int i = 0; i < n; ++i) order[i] = it[i].job;
}

}  // namespace

extern "C" fsp_status fsp_instance_create(const int32_t *p, int32_t n, int32_t m, fsp_instance **out) {
    return fsp_instance_create_ex(p, n, m, 0u, out);
}

extern "C" fsp_status fsp_instance_create_ex(const int32_t *p, int32_t n, int32_t m, uint32_t flags,
                                             fsp_instance **out) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    if (!p || n < 1 || n > FSP_MAX_JOBS || m < 2 || m > FSP_MAX_MACHINES) return FSP_EINVAL;
    if (flags & ~(uint32_t)FSP_INSTANCE_RELEASE_PER_JOB) return FSP_EINVAL;
    int64_t total = 0;
    int32_t maxp = 0;
    for (int64_t i = 0; i < (int64_t)n * m; ++i) {
        if (p[i] < 0) return FSP_EINVAL;
        total += p[i];
        maxp = std::max(maxp, p[i]);
    }
    if (total >= (int64_t(1) << 30)) return FSP_EINVAL;

    fsp_instance *inst = new (std::nothrow) fsp_instance();
    if (!inst) return FSP_ENOMEM;
    inst->n = n;
    inst->m = m;
    inst->flags = flags;
    inst->P = m * (m - 1) / 2;
    inst->npad = (int32_t)align_up((size_t)n, fspgb::kRecAlign);
    inst->p.assign(p, p + (size_t)n * m);

    // Couples ordered by the second machine l, then k: the kernel computes the
    // latency of machine l (QM) once, at the first couple of each l.
    const int P = inst->P, npad = inst->npad;
    inst->pairs.resize(2 * (size_t)P);
    {
        int c = 0;
        for (int l = 1; l < m; ++l)
            for (int k = 0; k < l; ++k, ++c) {
                inst->pairs[2 * c] = (uint8_t)k;
                inst->pairs[2 * c + 1] = (uint8_t)l;
            }
    }

    // Record format: compact when every field fits its bit field.
    // s = lag_j + p_jl = sum_{k<h<=l} p_jh is largest for (k,l) = (0,m-1).
    int64_t maxs = 0;
    for (int j = 0; j < n; ++j) {
        int64_t row = 0;
        for (int h = 1; h < m; ++h) row += p[j * m + h];
        maxs = std::max(maxs, row);
    }
    inst->compact = (n <= 1024 && maxs < 8192 && maxp < 256) ? 1 : 0;
    inst->rec_bytes = inst->compact ? 4 : 16;
    inst->grec_bytes = inst->compact ? 8 : 16;

    std::vector<uint32_t> rec_c;
    std::vector<int32_t> rec_w;
    if (inst->compact)
        rec_c.assign((size_t)P * npad, 0u);
    else
        rec_w.assign((size_t)P * npad * 4, 0);
    std::vector<int64_t> lag(n);
    std::vector<int32_t> order(n);
    for (int c = 0; c < P; ++c) {
        const int k = inst->pairs[2 * c], l = inst->pairs[2 * c + 1];
        johnson_order(n, m, p, k, l, lag, order);
        for (int i = 0; i < n; ++i) {
            const int j = order[i];
            const int32_t delta = p[j * m + l] - p[j * m + k];
            const int32_t s = (int32_t)(lag[j] + p[j * m + l]);
            if (inst->compact) {
                rec_c[(size_t)c * npad + i] = (uint32_t)j | ((uint32_t)s << 10) | ((uint32_t)delta << 23);
            } else {
                int32_t *r = &rec_w[((size_t)c * npad + i) * 4];
                r[0] = j;
                r[1] = s;
                r[2] = delta;
                r[3] = 0;
            }
        }
    }

    // Couple-lanes layout: couple c in group c/32, lane c%32, position-major.
    inst->G = (P + 31) / 32;
    const int G = inst->G;
    std::vector<uint32_t> grec_c;  // two words per record
    std::vector<int32_t> grec_w;
    // empty couples and padding positions hold the no-op record s = 0, delta = 0
    if (inst->compact)
        grec_c.assign((size_t)G * npad * 32 * 2, 0u);
    else
        grec_w.assign((size_t)G * npad * 32 * 4, 0);
    for (int c = 0; c < P; ++c) {
        const int g = c / 32, lane = c % 32;
        for (int i = 0; i < npad; ++i) {
            const size_t dst = ((size_t)g * npad + i) * 32 + lane;
            if (inst->compact) {
                // couple-lanes encoding: word 0 = 1024 s + j, word 1 =
                // 1024 delta (two's complement), both used by the scan as they are
                const uint32_t r = rec_c[(size_t)c * npad + i];
                const uint32_t j = r & 1023u, sv = (r >> 10) & 8191u;
                const int32_t dv = (int32_t)r >> 23;
                grec_c[2 * dst] = (sv << 10) | j;
                grec_c[2 * dst + 1] = (uint32_t)(dv * 1024);
            }
            else
                for (int f = 0; f < 4; ++f) grec_w[dst * 4 + f] = rec_w[((size_t)c * npad + i) * 4 + f];
        }
    }
    std::vector<uint8_t> gpairs((size_t)G * 32 * 2, 0);
    for (int slot = 0; slot < G * 32; ++slot) {
        gpairs[2 * slot] = slot < P ? inst->pairs[2 * slot] : 0;
        gpairs[2 * slot + 1] = slot < P ? inst->pairs[2 * slot + 1] : 1;
    }

    std::vector<int32_t> head((size_t)m * n), tail((size_t)m * n), ptm((size_t)m * n);
    for (int j = 0; j < n; ++j) {
        int64_t acc = 0;
        for (int k = 0; k < m; ++k) {
            head[(size_t)k * n + j] = (int32_t)acc;
            acc += p[j * m + k];
        }
        acc = 0;
        for (int l = m - 1; l >= 0; --l) {
            tail[(size_t)l * n + j] = (int32_t)acc;
            acc += p[j * m + l];
        }
        for (int k = 0; k < m; ++k) ptm[(size_t)k * n + j] = p[j * m + k];
    }

    // Jobs sorted by head (resp. tail) per machine: the minimum over the
    // unscheduled jobs is the first unscheduled entry of the sorted list.
    std::vector<int32_t> hsort((size_t)m * n * 2), tsort((size_t)m * n * 2), ptot(m, 0);
    {
        std::vector<int32_t> idx(n);
        for (int k = 0; k < m; ++k) {
            for (int j = 0; j < n; ++j) idx[j] = j;
            std::sort(idx.begin(), idx.end(), [&](int a, int b) {
                const int32_t x = head[(size_t)k * n + a], y = head[(size_t)k * n + b];
                return x != y ? x < y : a < b;
            });
            for (int i = 0; i < n; ++i) {
                hsort[((size_t)k * n + i) * 2] = idx[i];
                hsort[((size_t)k * n + i) * 2 + 1] = head[(size_t)k * n + idx[i]];
            }
            for (int j = 0; j < n; ++j) idx[j] = j;
            std::sort(idx.begin(), idx.end(), [&](int a, int b) {
                const int32_t x = tail[(size_t)k * n + a], y = tail[(size_t)k * n + b];
                return x != y ? x < y : a < b;
            });
            for (int i = 0; i < n; ++i) {
                tsort[((size_t)k * n + i) * 2] = idx[i];
                tsort[((size_t)k * n + i) * 2 + 1] = tail[(size_t)k * n + idx[i]];
            }
            int64_t tot = 0;
            for (int j = 0; j < n; ++j) tot += p[j * m + k];
            ptot[k] = (int32_t)tot;
        }
    }

    inst->mpad = m <= 8 ? 8 : m <= 12 ? 12 : m <= 16 ? 16 : m <= 20 ? 20 : m <= 24 ? 24 : 32;
    const int mpad = inst->mpad;
    std::vector<int32_t> pp((size_t)n * mpad, 0);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < m; ++k) pp[(size_t)j * mpad + k] = p[j * m + k];

    // One device block, every array 256-byte aligned.
    const size_t rec_sz = (size_t)P * npad * inst->rec_bytes;
    const size_t off_rec = 0;
    const size_t off_pairs = align_up(off_rec + rec_sz, 256);
    const size_t off_p = align_up(off_pairs + 2 * (size_t)P, 256);
    const size_t off_head = align_up(off_p + sizeof(int32_t) * n * m, 256);
    const size_t off_tail = align_up(off_head + sizeof(int32_t) * n * m, 256);
    const size_t off_ptm = align_up(off_tail + sizeof(int32_t) * n * m, 256);
    const size_t grec_sz = (size_t)G * npad * 32 * inst->grec_bytes;
    const size_t off_grec = align_up(off_ptm + sizeof(int32_t) * n * m, 256);
    const size_t off_gpairs = align_up(off_grec + grec_sz, 256);
    const size_t off_hsort = align_up(off_gpairs + gpairs.size(), 256);
    const size_t off_tsort = align_up(off_hsort + sizeof(int32_t) * hsort.size(), 256);
    const size_t off_ptot = align_up(off_tsort + sizeof(int32_t) * tsort.size(), 256);
    const size_t off_pp = align_up(off_ptot + sizeof(int32_t) * m, 256);
    const size_t bytes = align_up(off_pp + sizeof(int32_t) * pp.size(), 256);

    fsp_status st = FSP_OK;
    unsigned char *blk = nullptr;
    if (cudaGetDevice(&inst->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&inst->num_sms, cudaDevAttrMultiProcessorCount, inst->device) != cudaSuccess) {
        st = FSP_ECUDA;
    } else if (cudaMalloc((void **)&blk, bytes) != cudaSuccess) {
        st = FSP_ENOMEM;
    } else {
        const void *src_rec = inst->compact ? (const void *)rec_c.data() : (const void *)rec_w.data();
        if (cudaMemcpy(blk + off_rec, src_rec, rec_sz, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_pairs, inst->pairs.data(), 2 * (size_t)P, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_p, p, sizeof(int32_t) * n * m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_head, head.data(), sizeof(int32_t) * n * m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_tail, tail.data(), sizeof(int32_t) * n * m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_ptm, ptm.data(), sizeof(int32_t) * n * m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_grec, inst->compact ? (const void *)grec_c.data() : (const void *)grec_w.data(),
                       grec_sz, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_gpairs, gpairs.data(), gpairs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_hsort, hsort.data(), sizeof(int32_t) * hsort.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(blk + off_tsort, tsort.data(), sizeof(int32_t) * tsort.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(blk + off_ptot, ptot.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(blk + off_pp, pp.data(), sizeof(int32_t) * pp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            st = FSP_ECUDA;
        }
    }
    // Device-side errors (a bounded wait that ran out) land in a pinned,
    // mapped word the host reads without synchronising.
    int32_t *hs = nullptr;
    if (st == FSP_OK) {
        if (cudaHostAlloc((void **)&hs, 256, cudaHostAllocMapped) != cudaSuccess) {
            st = FSP_ENOMEM;
            hs = nullptr;
        } else {
            *hs = 0;
            if (cudaHostGetDevicePointer((void **)&inst->dev_status, hs, 0) != cudaSuccess) st = FSP_ECUDA;
        }
    }
    if (st != FSP_OK) {
        if (hs) cudaFreeHost(hs);
        if (blk) cudaFree(blk);
        delete inst;
        return st;
    }
    inst->host_status = hs;
    inst->dev_block = blk;
    inst->dev_bytes = bytes;
    inst->t.rec = blk + off_rec;
    inst->t.pairs = (const uint8_t *)(blk + off_pairs);
    inst->t.p = (const int32_t *)(blk + off_p);
    inst->t.head = (const int32_t *)(blk + off_head);
    inst->t.tail = (const int32_t *)(blk + off_tail);
    inst->t.ptm = (const int32_t *)(blk + off_ptm);
    inst->t.grec = blk + off_grec;
    inst->t.gpairs = (const uint8_t *)(blk + off_gpairs);
    inst->t.hsort = (const int32_t *)(blk + off_hsort);
    inst->t.tsort = (const int32_t *)(blk + off_tsort);
    inst->t.ptot = (const int32_t *)(blk + off_ptot);
    inst->t.pp = (const int32_t *)(blk + off_pp);
    *out = inst;
    return FSP_OK;
}

extern "C" void fsp_instance_destroy(fsp_instance *inst) {
    if (!inst) return;
    for (cudaStream_t s : inst->host_streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : inst->host_events)
        if (e) cudaEventDestroy(e);
    if (inst->dev_block) cudaFree(inst->dev_block);
    if (inst->host_status) cudaFreeHost(inst->host_status);
    delete inst;
}

extern "C" fsp_status fsp_instance_query(const fsp_instance *inst, fsp_instance_info *info) {
    if (!inst || !info) return FSP_EINVAL;
    info->n = inst->n;
    info->m = inst->m;
    info->pairs = inst->P;
    info->compact = inst->compact;
    info->device_bytes = (int64_t)inst->dev_bytes;
    info->device = inst->device;
    info->flags = (int32_t)inst->flags;
    return FSP_OK;
}

extern "C" const char *fsp_status_string(fsp_status s) {
    switch (s) {
        case FSP_OK: return "ok";
        case FSP_EINVAL: return "invalid argument";
        case FSP_ENOMEM: return "out of memory";
        case FSP_ECUDA: return "CUDA error";
        case FSP_EBADNODE: return "invalid node";
        case FSP_ETIMEDOUT: return "timed out";
        case FSP_ENOTFOUND: return "no schedule within the upper bound";
        case FSP_EBUSY: return "busy or shut down";
    }
    return "unknown status";
}

namespace {
std::atomic<int64_t> g_launches{0};
}  // namespace

void fspgb::note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

extern "C" int64_t fsp_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char *fsp_version(void) { return "0.1.0"; }
