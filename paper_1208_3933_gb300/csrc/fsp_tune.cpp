// fsp_tune.cpp -- launch-shape autotuner for the bounding kernels.
//
// The paper observes that the best pool/launch configuration depends on the
// instance and "has to be determined at runtime by testing different pool
// sizes" (Section VI); here the instance and pool size are given, and the
// tuner times every launch shape of both kernels that fits the device on the
// caller's pool, keeps the fastest for (instance, N) in the instance, and can
// persist it in a plain-text cache file keyed by (device, n, m, records, N).
// Every candidate's bounds are compared with the first candidate's: the
// shapes must agree bit for bit, or the tuner fails with FSP_ECUDA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fsp_internal.h"

namespace {

std::string cache_key(const fsp_instance *inst, int64_t N) {
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, inst->device);
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s sm%d n%d m%d c%d N%lld", name.c_str(), prop.multiProcessorCount, inst->n,
                  inst->m, inst->compact, (long long)N);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, fsp_launch_config *cfg) {
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        const size_t kl = key.size();
        if (std::strncmp(line, key.c_str(), kl) != 0 || line[kl] != ' ') continue;
        fsp_launch_config c = {};
        if (std::sscanf(line + kl, " => %d %d %d %d %d %d %d %d", &c.kernel, &c.nodes_per_thread, &c.blocks_per_sm,
                        &c.pairs_per_tile, &c.warps_per_block, &c.positions_per_tile, &c.staging,
                        &c.tail_slices) >= 7) {
            *cfg = c;  // the last entry for a key wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const fsp_launch_config &c, float ms) {
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s => %d %d %d %d %d %d %d %d  # %.4f ms\n", key.c_str(), c.kernel, c.nodes_per_thread,
                 c.blocks_per_sm, c.pairs_per_tile, c.warps_per_block, c.positions_per_tile, c.staging,
                 c.tail_slices, ms);
    std::fclose(f);
}

void remember(const fsp_instance *inst, int64_t N, const fsp_launch_config &c) {
    std::lock_guard<std::mutex> g(inst->mu);
    for (auto &e : inst->tuned)
        if (e.first == N) {
            e.second = c;
            return;
        }
    inst->tuned.emplace_back(N, c);
}

std::vector<fsp_launch_config> candidates(const fsp_instance *inst, int64_t N) {
    std::vector<fsp_launch_config> out;
    const int sms = fspgb::num_sms(inst->device);
    auto add = [&](fsp_launch_config c) {
        fsp_launch_config r;
        size_t smem = 0;
        if (fspgb::resolve_config(inst, N, &c, &r, &smem) != FSP_OK) return;
        for (auto &o : out)
            if (std::memcmp(&o, &r, sizeof r) == 0) return;
        out.push_back(r);
    };
    for (int W : {16, 15, 14, 13, 12, 10, 8, 6, 4, 2, 1}) {
        fsp_launch_config c = {};
        c.kernel = FSP_KERNEL_LANES;
        c.warps_per_block = W;
        c.staging = FSP_STAGING_RESIDENT;
        add(c);
        for (int staging : {FSP_STAGING_STREAMED, FSP_STAGING_SPLIT, FSP_STAGING_WARP})
            for (int pos : {0, 256, 128, 96, 64}) {
                c.staging = staging;
                c.positions_per_tile = pos;
                c.pairs_per_tile = 0;
                c.tail_slices = 0;
                add(c);
                if (W <= 8) {
                    fsp_launch_config c2 = c;
                    c2.blocks_per_sm = 2;
                    add(c2);
                }
                // one or two node sets of 28 per warp (streamed staging, compact records)
                if (staging == FSP_STAGING_STREAMED && inst->compact)
                    for (int npw : {28, 56}) {
                        fsp_launch_config c2 = c;
                        c2.nodes_per_thread = npw;
                        add(c2);
                        if (W <= 8) {
                            c2.blocks_per_sm = 2;
                            add(c2);
                        }
                    }
                // pools of more than one wave: the last partial wave's batches
                // split by couples as well
                if (staging == FSP_STAGING_STREAMED && pos == 0 && N > 32 * W * (int64_t)sms)
                    for (int ts : {2, 3}) {
                        fsp_launch_config c3 = c;
                        c3.tail_slices = ts;
                        add(c3);
                        if (W <= 8) {
                            c3.blocks_per_sm = 2;
                            add(c3);
                        }
                    }
                // pools of under two waves of block batches: work items of
                // fewer couples (streamed and split staging) as well
                if ((staging == FSP_STAGING_STREAMED || staging == FSP_STAGING_SPLIT) && pos == 0 &&
                    N < 2 * 32 * W * (int64_t)sms)
                    for (int ppt : {32, 64, 96}) {
                        if (ppt >= inst->P) break;
                        c.pairs_per_tile = ppt;
                        c.tail_slices = 0;
                        add(c);
                        if (W <= 8) {
                            fsp_launch_config c2 = c;
                            c2.blocks_per_sm = 2;
                            add(c2);
                        }
                    }
            }
    }
    // small pools: streamed staging with node tiles of 1-4 warps and several
    // blocks per SM, couple slices of one or two groups
    if (N < 2 * 32 * 16 * (int64_t)sms)
        for (int W : {1, 2, 4})
            for (int bps : {4, 8})
                for (int pos : {64, 32})
                    for (int ppt : {32, 64}) {
                        if (W * bps > 16 || ppt >= inst->P) continue;
                        fsp_launch_config c = {};
                        c.kernel = FSP_KERNEL_LANES;
                        c.staging = FSP_STAGING_STREAMED;
                        c.warps_per_block = W;
                        c.blocks_per_sm = bps;
                        c.positions_per_tile = pos;
                        c.pairs_per_tile = ppt;
                        add(c);
                    }
    // global staging (warps independent, records from L2/L1): node tiles of
    // 1-16 warps, couple slices chosen from the pool size or fixed
    for (int W : {16, 8, 4, 2, 1})
        for (int ppt : {0, 32, 64, 96, 1 << 30}) {
            if (ppt && ppt < (1 << 30) && ppt >= inst->P) continue;
            fsp_launch_config c = {};
            c.kernel = FSP_KERNEL_LANES;
            c.staging = FSP_STAGING_GLOBAL;
            c.warps_per_block = W;
            c.pairs_per_tile = ppt == (1 << 30) ? inst->P : ppt;
            add(c);
        }
    for (int K : {8, 4, 2, 1})
        for (int bps : {1, 2}) {
            fsp_launch_config c = {};
            c.kernel = FSP_KERNEL_LOCKSTEP;
            c.nodes_per_thread = K;
            c.blocks_per_sm = bps;
            add(c);
        }
    return out;
}

}  // namespace

extern "C" fsp_status fsp_autotune(const fsp_instance *inst, const int16_t *nodes, const int32_t *depths, int64_t N,
                                   int32_t *out_lb, void *cuda_stream, const char *cache_path,
                                   fsp_launch_config *best, float *best_ms) {
    if (!inst || N < 1 || !nodes || !depths || !out_lb) return FSP_EINVAL;
    fsp_status st = fspgb::take_device_status(inst);
    if (st != FSP_OK) return st;
    st = fspgb::check_device(inst);
    if (st != FSP_OK) return st;
    const std::string key = cache_key(inst, N);
    fsp_launch_config hit;
    if (cache_lookup(cache_path, key, &hit)) {
        fsp_launch_config r;
        size_t smem = 0;
        if (fspgb::resolve_config(inst, N, &hit, &r, &smem) == FSP_OK) {
            remember(inst, N, r);
            if (best) *best = r;
            if (best_ms) *best_ms = -1.0f;
            return FSP_OK;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const std::vector<fsp_launch_config> cands = candidates(inst, N);
    if (cands.empty()) return FSP_EINVAL;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FSP_ECUDA;
    }
    std::vector<int32_t> ref((size_t)N), cur((size_t)N);
    float best_t = 1e30f;
    fsp_launch_config best_c = cands[0];
    st = FSP_OK;
    for (size_t ci = 0; ci < cands.size() && st == FSP_OK; ++ci) {
        const fsp_launch_config &c = cands[ci];
        st = fspgb::launch_bound(inst, nodes, depths, N, out_lb, s, &c);  // warm-up, and the bounds
        if (st != FSP_OK) break;
        if (cudaMemcpyAsync(ci == 0 ? ref.data() : cur.data(), out_lb, sizeof(int32_t) * N, cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = FSP_ECUDA;
            break;
        }
        if (ci > 0 && std::memcmp(ref.data(), cur.data(), sizeof(int32_t) * N) != 0) {
            st = FSP_ECUDA;  // two launch shapes disagree: never expected
            break;
        }
        // time enough repetitions to cover about 2 ms
        float once = 0.f;
        cudaEventRecord(e0, s);
        st = fspgb::launch_bound(inst, nodes, depths, N, out_lb, s, &c);
        cudaEventRecord(e1, s);
        if (st != FSP_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            st = st != FSP_OK ? st : FSP_ECUDA;
            break;
        }
        cudaEventElapsedTime(&once, e0, e1);
        const int reps = std::max(1, std::min(20, (int)(2.0f / std::max(once, 1e-3f))));
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == FSP_OK; ++r) st = fspgb::launch_bound(inst, nodes, depths, N, out_lb, s, &c);
        cudaEventRecord(e1, s);
        if (st != FSP_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            st = st != FSP_OK ? st : FSP_ECUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        t /= reps;
        if (t < best_t) {
            best_t = t;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == FSP_OK) st = fspgb::take_device_status(inst);
    if (st != FSP_OK) return st;
    remember(inst, N, best_c);
    cache_store(cache_path, key, best_c, best_t);
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return FSP_OK;
}

extern "C" fsp_status fsp_tuned_config(const fsp_instance *inst, int64_t N, fsp_launch_config *cfg) {
    if (!inst || !cfg || N < 0) return FSP_EINVAL;
    size_t smem = 0;
    return fspgb::resolve_config(inst, N, nullptr, cfg, &smem);
}
