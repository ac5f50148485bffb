// fsp_bnb.cpp -- depth-first branch-and-bound around the GPU bounding
// operator (Section II-A operators; Section II-B forward branching: child i
// of a node appends unscheduled job J_i to its prefix; Section III-A: the
// children of an expanded node form one pool bounded on the device, the
// bounds come back to the host for elimination and selection).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fsp_internal.h"

namespace {

struct Node {
    int32_t lb;
    int32_t d;
    std::vector<int16_t> row;
};

struct Child {
    int32_t lb;
    int32_t job;
};

}  // namespace

extern "C" fsp_status fsp_branch_and_bound(const fsp_instance *inst, int32_t ub0, int16_t *best_perm,
                                           int32_t *best_makespan, int64_t *nodes_bounded) {
    if (!inst) return FSP_EINVAL;
    fsp_status st = fspgb::check_device(inst);
    if (st != FSP_OK) return st;
    const int n = inst->n;

    // Device and pinned host buffers for one pool of at most n children.
    cudaStream_t s = nullptr;
    int16_t *d_rows = nullptr, *h_rows = nullptr;
    int32_t *d_dep = nullptr, *d_out = nullptr, *h_dep = nullptr, *h_out = nullptr;
    auto cleanup = [&]() {
        if (d_rows) cudaFree(d_rows);
        if (d_dep) cudaFree(d_dep);
        if (d_out) cudaFree(d_out);
        if (h_rows) cudaFreeHost(h_rows);
        if (h_dep) cudaFreeHost(h_dep);
        if (h_out) cudaFreeHost(h_out);
        if (s) cudaStreamDestroy(s);
    };
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cleanup();
        return FSP_ECUDA;
    }
    if (cudaMalloc((void **)&d_rows, sizeof(int16_t) * n * n) != cudaSuccess ||
        cudaMalloc((void **)&d_dep, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc((void **)&d_out, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMallocHost((void **)&h_rows, sizeof(int16_t) * n * n) != cudaSuccess ||
        cudaMallocHost((void **)&h_dep, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMallocHost((void **)&h_out, sizeof(int32_t) * n) != cudaSuccess) {
        cleanup();
        return FSP_ENOMEM;
    }

    // Bounds h_rows[0..cnt) on the device; results land in h_out.
    auto bound = [&](int cnt) -> fsp_status {
        if (cudaMemcpyAsync(d_rows, h_rows, sizeof(int16_t) * cnt * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_dep, h_dep, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return FSP_ECUDA;
        fsp_status r = fspgb::launch_bound(inst, d_rows, d_dep, cnt, d_out, s, nullptr);
        if (r != FSP_OK) return r;
        if (cudaMemcpyAsync(h_out, d_out, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FSP_ECUDA;
        r = fspgb::take_device_status(inst);
        if (r != FSP_OK) return r;
        for (int i = 0; i < cnt; ++i)
            if (h_out[i] == FSP_LB_INVALID) return FSP_EBADNODE;
        return FSP_OK;
    };

    int64_t UB = (int64_t)ub0 + 1;
    bool found = false;
    int64_t count = 0;
    std::vector<int16_t> best(n, 0);
    std::vector<Node> stack;
    stack.reserve((size_t)n * n / 2 + 2);

    // the root: empty prefix
    std::memset(h_rows, 0, sizeof(int16_t) * n);
    h_dep[0] = 0;
    st = bound(1);
    if (st != FSP_OK) {
        cleanup();
        return st;
    }
    ++count;
    stack.push_back(Node{h_out[0], 0, std::vector<int16_t>(n, 0)});

    std::vector<char> used(n);
    std::vector<Child> kids;
    kids.reserve(n);
    while (!stack.empty()) {
        Node nd = std::move(stack.back());
        stack.pop_back();
        if (nd.lb >= UB) continue;  // elimination
        if (nd.d == n) {            // a leaf: its bound is its makespan
            UB = nd.lb;
            found = true;
            best = nd.row;
            continue;
        }
        // branching: one child per unscheduled job, in job order
        std::fill(used.begin(), used.end(), 0);
        for (int i = 0; i < nd.d; ++i) used[nd.row[i]] = 1;
        int cnt = 0;
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            int16_t *r = h_rows + (size_t)cnt * n;
            std::memcpy(r, nd.row.data(), sizeof(int16_t) * nd.d);
            r[nd.d] = (int16_t)j;
            h_dep[cnt] = nd.d + 1;
            ++cnt;
        }
        st = bound(cnt);  // bounding: the children as one pool
        if (st != FSP_OK) {
            cleanup();
            return st;
        }
        count += cnt;
        kids.clear();
        for (int i = 0; i < cnt; ++i) kids.push_back(Child{h_out[i], h_rows[(size_t)i * n + nd.d]});
        std::sort(kids.begin(), kids.end(), [](const Child &x, const Child &y) {
            return x.lb != y.lb ? x.lb < y.lb : x.job < y.job;
        });
        // selection: depth first, smallest (LB, job) popped first
        for (int t = cnt - 1; t >= 0; --t) {
            if (kids[t].lb >= UB) continue;
            Node c{kids[t].lb, nd.d + 1, nd.row};
            c.row[nd.d] = (int16_t)kids[t].job;
            stack.push_back(std::move(c));
        }
    }
    cleanup();
    if (nodes_bounded) *nodes_bounded = count;
    if (!found) return FSP_ENOTFOUND;
    if (best_makespan) *best_makespan = (int32_t)UB;
    if (best_perm) std::memcpy(best_perm, best.data(), sizeof(int16_t) * n);
    return FSP_OK;
}

namespace {

// Best position for inserting `job` into the partial sequence seq (Taillard
// 1990: with e = completion times of every prefix and q = tails of every
// suffix, each of the L+1 positions is evaluated in O(m)).  Returns the
// partial makespan there; the first position wins ties.  e, q, f are work
// arrays of at least (L+1) m, (L+2) m and m entries.
int64_t best_insertion(const int32_t *p, int m, const std::vector<int> &seq, int job, std::vector<int64_t> &e,
                       std::vector<int64_t> &q, std::vector<int64_t> &f, int *best_pos) {
    const int L = (int)seq.size();
    for (int k = 0; k < m; ++k) e[k] = 0;
    for (int i = 1; i <= L; ++i)
        for (int k = 0; k < m; ++k) {
            const int64_t up = e[(size_t)(i - 1) * m + k], left = k ? e[(size_t)i * m + k - 1] : 0;
            e[(size_t)i * m + k] = std::max(up, left) + p[seq[i - 1] * m + k];
        }
    for (int k = 0; k < m; ++k) q[(size_t)L * m + k] = 0;
    for (int i = L - 1; i >= 0; --i)
        for (int k = m - 1; k >= 0; --k) {
            const int64_t down = q[(size_t)(i + 1) * m + k], right = k + 1 < m ? q[(size_t)i * m + k + 1] : 0;
            q[(size_t)i * m + k] = std::max(down, right) + p[seq[i] * m + k];
        }
    int pos_best = 0;
    int64_t best = -1;
    for (int pos = 0; pos <= L; ++pos) {
        int64_t mk = 0;
        for (int k = 0; k < m; ++k) {
            f[k] = std::max(e[(size_t)pos * m + k], k ? f[k - 1] : 0) + p[job * m + k];
            mk = std::max(mk, f[k] + q[(size_t)pos * m + k]);
        }
        if (best < 0 || mk < best) {
            best = mk;
            pos_best = pos;
        }
    }
    *best_pos = pos_best;
    return best;
}

int64_t makespan_of(const int32_t *p, int m, const std::vector<int> &seq) {
    std::vector<int64_t> C(m, 0);
    for (int j : seq) {
        int64_t prev = 0;
        for (int k = 0; k < m; ++k) {
            C[k] = std::max(C[k], prev) + p[j * m + k];
            prev = C[k];
        }
    }
    return C[m - 1];
}

std::vector<int> neh_sequence(const fsp_instance *inst) {
    const int n = inst->n, m = inst->m;
    const int32_t *p = inst->p.data();
    std::vector<int> order(n);
    std::vector<int64_t> tot(n, 0);
    for (int j = 0; j < n; ++j) {
        order[j] = j;
        for (int k = 0; k < m; ++k) tot[j] += p[j * m + k];
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tot[a] > tot[b]; });
    std::vector<int> seq;
    seq.reserve(n);
    std::vector<int64_t> e((size_t)(n + 1) * m), q((size_t)(n + 2) * m), f(m);
    for (int idx = 0; idx < n; ++idx) {
        int pos = 0;
        best_insertion(p, m, seq, order[idx], e, q, f, &pos);
        seq.insert(seq.begin() + pos, order[idx]);
    }
    return seq;
}

// splitmix64 (Steele, Lea, Flood 2014): the heuristic's seeded random stream.
struct SplitMix {
    uint64_t x;
    uint64_t next() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    int below(int k) { return (int)(next() % (uint64_t)k); }
    double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

}  // namespace

// NEH constructive heuristic (Nawaz, Enscore and Ham 1983) for ub0 -- not
// part of the paper's method.  O(n^2 m) with the head/tail insertion
// evaluation (Taillard 1990).
extern "C" fsp_status fsp_neh(const fsp_instance *inst, int16_t *perm, int32_t *makespan) {
    if (!inst || !makespan) return FSP_EINVAL;
    const std::vector<int> seq = neh_sequence(inst);
    *makespan = (int32_t)makespan_of(inst->p.data(), inst->m, seq);
    if (perm)
        for (int i = 0; i < inst->n; ++i) perm[i] = (int16_t)seq[i];
    return FSP_OK;
}

// Iterated greedy (Ruiz and Stuetzle 2007) for ub0 -- not part of the paper's
// method.  From the NEH sequence, each iteration removes `d` = 4 random jobs,
// reinserts each at its best position, then improves the sequence by
// removing and reinserting every job (in random order) at its best position
// until a whole pass gains nothing; the result replaces the current sequence
// when it is no worse, else with probability exp(-(new - current) / T), T =
// 0.4 * sum(p) / (10 n m).  The best sequence seen is returned; its makespan
// is recomputed from the sequence, so it is always a valid upper bound.
extern "C" fsp_status fsp_iterated_greedy(const fsp_instance *inst, int32_t iterations, uint64_t seed,
                                          int16_t *perm, int32_t *makespan) {
    if (!inst || !makespan || iterations < 0) return FSP_EINVAL;
    const int n = inst->n, m = inst->m;
    const int32_t *p = inst->p.data();
    std::vector<int> cur = neh_sequence(inst), best = cur;
    int64_t cur_v = makespan_of(p, m, cur), best_v = cur_v;
    std::vector<int64_t> e((size_t)(n + 1) * m), q((size_t)(n + 2) * m), f(m);
    SplitMix rng{seed};
    double psum = 0;
    for (int i = 0; i < n * m; ++i) psum += p[i];
    const double temp = 0.4 * psum / (10.0 * n * m);
    const int d = std::min(4, n - 1);
    std::vector<int> removed, shuffled(n);
    for (int it = 0; n > 1 && it < iterations; ++it) {
        std::vector<int> seq = cur;
        removed.clear();
        for (int r = 0; r < d; ++r) {
            const int at = rng.below((int)seq.size());
            removed.push_back(seq[at]);
            seq.erase(seq.begin() + at);
        }
        int pos = 0;
        int64_t v = 0;
        for (int j : removed) {
            v = best_insertion(p, m, seq, j, e, q, f, &pos);
            seq.insert(seq.begin() + pos, j);
        }
        // insertion local search
        for (bool improved = true; improved;) {
            improved = false;
            for (int i = 0; i < n; ++i) shuffled[i] = i;
            for (int i = n - 1; i > 0; --i) std::swap(shuffled[i], shuffled[rng.below(i + 1)]);
            for (int j : shuffled) {
                const int at = (int)(std::find(seq.begin(), seq.end(), j) - seq.begin());
                seq.erase(seq.begin() + at);
                const int64_t w = best_insertion(p, m, seq, j, e, q, f, &pos);
                seq.insert(seq.begin() + pos, j);
                if (w < v) {
                    v = w;
                    improved = true;
                }
            }
        }
        if (v <= cur_v) {
            cur = seq;
            cur_v = v;
            if (v < best_v) {
                best = seq;
                best_v = v;
            }
        } else if (rng.unit() < std::exp(-(double)(v - cur_v) / temp)) {
            cur = seq;
            cur_v = v;
        }
    }
    *makespan = (int32_t)makespan_of(p, m, best);
    if (perm)
        for (int i = 0; i < n; ++i) perm[i] = (int16_t)best[i];
    return FSP_OK;
}
