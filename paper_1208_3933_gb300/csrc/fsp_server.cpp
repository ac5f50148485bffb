// fsp_server.cpp -- a device-resident bounding server with continuous batching.
//
// Clients (any number of host threads, e.g. concurrent branch-and-bound
// searches) submit pools of sub-problems of already-created instances; the
// instances' tables stay resident on the device.  One dispatcher thread:
//   - admits queued requests in arrival order while their device footprint
//     (nodes + depths + bounds) fits in a fixed device arena (the HBM budget);
//     a request larger than the whole arena is refused at submission;
//   - gathers the admitted requests into a batch for a free slot (a CUDA
//     stream with its own plan buffers), copies their pools in, launches the
//     batched bounding kernel over all of them, copies the bounds out, and
//     marks the slot's completion with a host callback;
//   - keeps admitting while earlier batches are in flight, so requests that
//     arrive meanwhile run as the next batch on another slot and their work
//     overlaps on the device.
// Latency is measured from submission to the completion callback; p50/p99
// are reported by fsp_server_get_stats.  Every wait a client does is bounded
// by its own timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "fsp_internal.h"
#include "fsp_plan.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over the device arena (offsets only), coalescing on free.
class Arena {
   public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

enum ReqState { kQueued = 0, kAdmitted = 1, kDone = 2, kCancelled = 3 };

}  // namespace

struct fsp_request {
    fsp_server *srv = nullptr;
    const fsp_instance *inst = nullptr;
    const int16_t *nodes = nullptr;
    const int32_t *depths = nullptr;
    int32_t *out = nullptr;
    int64_t N = 0;
    size_t bytes = 0, off = 0;    // arena footprint (0: bounded in place)
    // page-locked client buffers are bounded in place: the kernel reads the
    // rows and depths and writes the bounds through these device-visible
    // addresses of the client's own memory, with no copy and no arena space
    bool in_place = false;
    const int16_t *dv_nodes = nullptr;
    const int32_t *dv_depths = nullptr;
    int32_t *dv_out = nullptr;
    Clock::time_point t_submit;
    int state = kQueued;          // guarded by the server mutex
    fsp_status result = FSP_OK;
    bool released = false;        // the client dropped its handle
    std::condition_variable cv;   // this request's completion (server mutex)
};

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    std::vector<fsp_request *> reqs;
    bool busy = false;  // cleared by the completion callback
    // plan buffers: pinned host staging and device copies
    fspgb::LanesArgs *h_args = nullptr, *d_args = nullptr;
    int2 *h_items = nullptr, *d_items = nullptr;
    int32_t *d_counter = nullptr;
    size_t args_cap = 0, items_cap = 0;
    fsp_server *srv = nullptr;
};

}  // namespace

struct fsp_server {
    fsp_server_config cfg{};
    int device = 0;
    unsigned char *arena_mem = nullptr;
    size_t arena_size = 0;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_dispatch;  // queue, slot completion, shutdown
    std::deque<fsp_request *> queue;
    std::vector<fsp_request *> live;      // every request not yet freed
    std::vector<Slot> slots;
    std::thread dispatcher;
    bool accepting = true, stopping = false;
    fsp_status fatal = FSP_OK;
    // statistics
    std::vector<double> lat_us;
    int64_t pools_done = 0, nodes_done = 0, batches = 0, pools_batched = 0;
    Clock::time_point t_first, t_last;
    bool any_done = false;
};

namespace {

void finish_request(fsp_server *srv, fsp_request *r, fsp_status result, Clock::time_point now);

// Runs on the CUDA callback thread once a slot's batch (bounds included) has
// completed: retires its requests at once -- each waiting client is woken by
// its own request's condition variable -- and frees the slot for the
// dispatcher.  Host work only: no CUDA call is made here.
void complete_slot_cb(void *p) {
    Slot *s = static_cast<Slot *>(p);
    fsp_server *srv = s->srv;
    std::lock_guard<std::mutex> g(srv->mu);
    const auto now = Clock::now();
    fsp_status st = FSP_OK;
    for (fsp_request *r : s->reqs) {
        const fsp_status t = fspgb::take_device_status(r->inst);
        if (t != FSP_OK) st = t;
    }
    for (fsp_request *r : s->reqs) finish_request(srv, r, st, now);
    s->reqs.clear();
    s->busy = false;
    srv->cv_dispatch.notify_all();
}

bool grow(Slot &s, size_t nargs, size_t nitems) {
    if (nargs > s.args_cap) {
        if (s.h_args) cudaFreeHost(s.h_args);
        if (s.d_args) cudaFree(s.d_args);
        s.h_args = nullptr;
        s.d_args = nullptr;
        const size_t cap = std::max<size_t>(nargs, 64);
        if (cudaMallocHost((void **)&s.h_args, sizeof(fspgb::LanesArgs) * cap) != cudaSuccess ||
            cudaMalloc((void **)&s.d_args, sizeof(fspgb::LanesArgs) * cap) != cudaSuccess) {
            s.args_cap = 0;
            return false;
        }
        s.args_cap = cap;
    }
    if (nitems > s.items_cap) {
        if (s.h_items) cudaFreeHost(s.h_items);
        if (s.d_items) cudaFree(s.d_items);
        s.h_items = nullptr;
        s.d_items = nullptr;
        const size_t cap = std::max<size_t>(nitems, 4096);
        if (cudaMallocHost((void **)&s.h_items, sizeof(int2) * cap) != cudaSuccess ||
            cudaMalloc((void **)&s.d_items, sizeof(int2) * cap) != cudaSuccess) {
            s.items_cap = 0;
            return false;
        }
        s.items_cap = cap;
    }
    return true;
}

// Enqueues one batch on slot s (dispatcher thread, server mutex NOT held).
fsp_status launch_batch(fsp_server *srv, Slot &s) {
    cudaStream_t st = s.stream;
    std::vector<fsp_pool_desc> pools;
    std::vector<fsp_request *> wide;
    for (fsp_request *r : s.reqs) {
        if (r->in_place) {
            fsp_pool_desc d{r->inst, r->dv_nodes, r->dv_depths, r->dv_out, r->N};
            if (r->inst->compact)
                pools.push_back(d);
            else
                wide.push_back(r);
            continue;
        }
        unsigned char *base = srv->arena_mem + r->off;
        const int n = r->inst->n;
        int16_t *d_nodes = reinterpret_cast<int16_t *>(base);
        int32_t *d_dep = reinterpret_cast<int32_t *>(base + align_up(sizeof(int16_t) * r->N * n, 256));
        int32_t *d_out =
            reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(d_dep) + align_up(sizeof(int32_t) * r->N, 256));
        if (r->N > 0 &&
            (cudaMemcpyAsync(d_nodes, r->nodes, sizeof(int16_t) * r->N * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
             cudaMemcpyAsync(d_dep, r->depths, sizeof(int32_t) * r->N, cudaMemcpyHostToDevice, st) != cudaSuccess))
            return FSP_ECUDA;
        fsp_pool_desc d{r->inst, d_nodes, d_dep, d_out, r->N};
        if (r->inst->compact)
            pools.push_back(d);
        else
            wide.push_back(r);
    }
    std::vector<fspgb::LanesArgs> args;
    std::vector<int2> items;
    fspgb::PlanParams pp;
    fsp_status rc = fspgb::build_plan(pools.data(), (int32_t)pools.size(), srv->cfg.warps_per_block, 0,
                                      srv->device, args, items, pp);
    if (rc != FSP_OK) return rc;
    if (!grow(s, args.size(), items.size())) return FSP_ENOMEM;
    if (!args.empty()) std::memcpy(s.h_args, args.data(), sizeof(fspgb::LanesArgs) * args.size());
    if (!items.empty()) std::memcpy(s.h_items, items.data(), sizeof(int2) * items.size());
    if ((!args.empty() && cudaMemcpyAsync(s.d_args, s.h_args, sizeof(fspgb::LanesArgs) * args.size(),
                                          cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (!items.empty() &&
         cudaMemcpyAsync(s.d_items, s.h_items, sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st) != cudaSuccess))
        return FSP_ECUDA;
    rc = fspgb::launch_plan(s.d_args, s.d_items, s.d_counter, pp, st);
    if (rc != FSP_OK) return rc;
    // instances with 128-bit records: one plain launch each
    for (fsp_request *r : wide) {
        unsigned char *base = srv->arena_mem + r->off;
        const int n = r->inst->n;
        const int16_t *d_nodes = reinterpret_cast<const int16_t *>(base);
        const int32_t *d_dep = reinterpret_cast<const int32_t *>(base + align_up(sizeof(int16_t) * r->N * n, 256));
        int32_t *d_out = const_cast<int32_t *>(d_dep) + align_up(sizeof(int32_t) * r->N, 256) / sizeof(int32_t);
        if (r->in_place) {
            d_nodes = r->dv_nodes;
            d_dep = r->dv_depths;
            d_out = r->dv_out;
        }
        if (r->N > 0) {
            rc = fspgb::launch_bound(r->inst, d_nodes, d_dep, r->N, d_out, st, nullptr);
            if (rc != FSP_OK) return rc;
        }
    }
    for (fsp_request *r : s.reqs) {
        if (r->N == 0 || r->in_place) continue;
        const unsigned char *base = srv->arena_mem + r->off;
        const int32_t *d_out = reinterpret_cast<const int32_t *>(
            base + align_up(sizeof(int16_t) * r->N * r->inst->n, 256) + align_up(sizeof(int32_t) * r->N, 256));
        if (cudaMemcpyAsync(r->out, d_out, sizeof(int32_t) * r->N, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return FSP_ECUDA;
    }
    if (cudaLaunchHostFunc(st, complete_slot_cb, &s) != cudaSuccess) return FSP_ECUDA;
    return FSP_OK;
}

void free_request(fsp_server *srv, fsp_request *r) {
    // server mutex held
    auto it = std::find(srv->live.begin(), srv->live.end(), r);
    if (it != srv->live.end()) {
        *it = srv->live.back();
        srv->live.pop_back();
    }
    delete r;
}

void finish_request(fsp_server *srv, fsp_request *r, fsp_status result, Clock::time_point now) {
    // server mutex held
    if (r->state == kAdmitted && r->bytes) srv->arena.release(r->off, r->bytes);
    r->state = kDone;
    r->result = result;
    if (result == FSP_OK) {
        srv->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
        srv->pools_done += 1;
        srv->nodes_done += r->N;
        if (!srv->any_done) srv->t_first = r->t_submit;
        srv->any_done = true;
        srv->t_last = now;
    }
    if (r->released)
        free_request(srv, r);
    else
        r->cv.notify_all();
}

void dispatcher_main(fsp_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        // completed slots are retired by their completion callback
        bool in_flight = false;
        for (Slot &s : srv->slots) in_flight |= s.busy;
        if (srv->stopping && srv->queue.empty() && !in_flight) break;
        // admit into a free slot
        Slot *free_slot = nullptr;
        for (Slot &s : srv->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        if (free_slot && !srv->queue.empty() && srv->fatal == FSP_OK) {
            std::vector<fsp_request *> take;
            while (!srv->queue.empty() && (int)take.size() < srv->cfg.max_batch_pools) {
                fsp_request *r = srv->queue.front();
                size_t off = 0;
                if (r->bytes && !srv->arena.alloc(r->bytes, &off)) break;  // in order: wait for memory
                r->off = off;
                r->state = kAdmitted;
                srv->queue.pop_front();
                take.push_back(r);
            }
            if (!take.empty()) {
                free_slot->reqs = take;
                free_slot->busy = true;
                lk.unlock();
                const fsp_status st = launch_batch(srv, *free_slot);
                lk.lock();
                srv->batches += 1;
                srv->pools_batched += (int64_t)take.size();
                if (st != FSP_OK) {
                    // nothing of this batch can be trusted; fail its requests
                    lk.unlock();
                    cudaStreamSynchronize(free_slot->stream);
                    lk.lock();
                    for (fsp_request *r : free_slot->reqs) finish_request(srv, r, st, Clock::now());
                    free_slot->reqs.clear();
                    free_slot->busy = false;
                    srv->fatal = st;
                }
                continue;
            }
        }
        srv->cv_dispatch.wait(lk);
    }
}

}  // namespace

extern "C" fsp_status fsp_server_create(const fsp_server_config *cfg, fsp_server **out) {
    if (!out) return FSP_EINVAL;
    *out = nullptr;
    fsp_server_config c = {};
    if (cfg) c = *cfg;
    if (c.hbm_budget_bytes < 0 || c.max_batch_pools < 0 || c.slots < 0 || c.slots > 8 || c.warps_per_block < 0 ||
        c.warps_per_block > 16)
        return FSP_EINVAL;
    if (!c.hbm_budget_bytes) c.hbm_budget_bytes = (int64_t)1 << 30;
    if (!c.max_batch_pools) c.max_batch_pools = 256;
    if (!c.slots) c.slots = 2;
    fsp_server *srv = new (std::nothrow) fsp_server();
    if (!srv) return FSP_ENOMEM;
    srv->cfg = c;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        delete srv;
        return FSP_ECUDA;
    }
    srv->arena_size = (size_t)c.hbm_budget_bytes;
    if (cudaMalloc((void **)&srv->arena_mem, srv->arena_size) != cudaSuccess) {
        delete srv;
        return FSP_ENOMEM;
    }
    srv->arena.reset(srv->arena_size);
    srv->slots.resize((size_t)c.slots);
    for (Slot &s : srv->slots) {
        s.srv = srv;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc((void **)&s.d_counter, 256) != cudaSuccess) {
            for (Slot &t : srv->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.d_counter) cudaFree(t.d_counter);
            }
            cudaFree(srv->arena_mem);
            delete srv;
            return FSP_ECUDA;
        }
    }
    srv->dispatcher = std::thread(dispatcher_main, srv);
    *out = srv;
    return FSP_OK;
}

extern "C" fsp_status fsp_server_submit(fsp_server *srv, const fsp_instance *inst, const int16_t *nodes,
                                        const int32_t *depths, int64_t N, int32_t *out_lb, fsp_request **req) {
    if (!req) return FSP_EINVAL;
    *req = nullptr;
    if (!srv || !inst || N < 0 || (N > 0 && (!nodes || !depths || !out_lb))) return FSP_EINVAL;
    if (inst->device != srv->device) return FSP_EINVAL;
    // page-locked (pinned or registered) buffers are read and written in place
    auto device_view = [](const void *h, void **d) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
            cudaGetLastError();  // not a CUDA-known pointer: clear the sticky-free error
            return false;
        }
        if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
        *d = a.devicePointer;
        return true;
    };
    void *dvn = nullptr, *dvd = nullptr, *dvo = nullptr;
    const bool in_place = N > 0 && device_view(nodes, &dvn) && device_view(depths, &dvd) && device_view(out_lb, &dvo);
    const size_t bytes =
        in_place ? 0 : align_up(sizeof(int16_t) * N * inst->n, 256) + 2 * align_up(sizeof(int32_t) * N, 256) + 256;
    if (bytes > srv->arena_size) return FSP_EBUSY;  // can never be admitted
    fsp_request *r = new (std::nothrow) fsp_request();
    if (!r) return FSP_ENOMEM;
    r->in_place = in_place;
    r->dv_nodes = static_cast<const int16_t *>(dvn);
    r->dv_depths = static_cast<const int32_t *>(dvd);
    r->dv_out = static_cast<int32_t *>(dvo);
    r->srv = srv;
    r->inst = inst;
    r->nodes = nodes;
    r->depths = depths;
    r->out = out_lb;
    r->N = N;
    r->bytes = bytes;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (!srv->accepting) {
            delete r;
            return FSP_EBUSY;
        }
        if (srv->fatal != FSP_OK) {
            delete r;
            return srv->fatal;
        }
        srv->queue.push_back(r);
        srv->live.push_back(r);
    }
    srv->cv_dispatch.notify_all();
    *req = r;
    return FSP_OK;
}

extern "C" fsp_status fsp_request_wait(fsp_request *r, int64_t timeout_us) {
    if (!r) return FSP_EINVAL;
    fsp_server *srv = r->srv;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return r->state == kDone || r->state == kCancelled; };
    if (timeout_us < 0) {
        r->cv.wait(lk, ready);
    } else if (!r->cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
        return FSP_ETIMEDOUT;
    }
    return r->state == kCancelled ? FSP_EBUSY : r->result;
}

extern "C" fsp_status fsp_request_cancel(fsp_request *r) {
    if (!r) return FSP_EINVAL;
    fsp_server *srv = r->srv;
    std::lock_guard<std::mutex> g(srv->mu);
    if (r->state != kQueued) return FSP_EBUSY;  // admitted work runs to completion
    auto it = std::find(srv->queue.begin(), srv->queue.end(), r);
    if (it != srv->queue.end()) srv->queue.erase(it);
    r->state = kCancelled;
    r->cv.notify_all();
    return FSP_OK;
}

extern "C" void fsp_request_release(fsp_request *r) {
    if (!r) return;
    fsp_server *srv = r->srv;
    std::lock_guard<std::mutex> g(srv->mu);
    if (r->state == kDone || r->state == kCancelled)
        free_request(srv, r);
    else
        r->released = true;  // freed by the dispatcher when it completes
}

extern "C" fsp_status fsp_server_get_stats(fsp_server *srv, fsp_server_stats *st) {
    if (!srv || !st) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    std::memset(st, 0, sizeof *st);
    st->pools_done = srv->pools_done;
    st->nodes_done = srv->nodes_done;
    st->batches = srv->batches;
    st->mean_pools_per_batch = srv->batches ? (double)srv->pools_batched / srv->batches : 0.0;
    st->queued = (int64_t)srv->queue.size();
    for (const Slot &s : srv->slots) st->in_flight += s.busy ? (int64_t)s.reqs.size() : 0;
    st->arena_bytes = (int64_t)srv->arena_size;
    st->arena_bytes_used = (int64_t)srv->arena.used();
    if (!srv->lat_us.empty()) {
        std::vector<double> v = srv->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = std::min(v.size() - 1, (size_t)std::ceil(q * v.size()) - (q * v.size() >= 1 ? 1 : 0));
            return v[i];
        };
        st->p50_us = pct(0.50);
        st->p99_us = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_us = sum / v.size();
    }
    if (srv->any_done) st->active_seconds = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
    return FSP_OK;
}

extern "C" fsp_status fsp_server_reset_stats(fsp_server *srv) {
    if (!srv) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    srv->lat_us.clear();
    srv->pools_done = srv->nodes_done = srv->batches = srv->pools_batched = 0;
    srv->any_done = false;
    return FSP_OK;
}

extern "C" fsp_status fsp_server_shutdown(fsp_server *srv) {
    if (!srv) return FSP_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    srv->accepting = false;
    return FSP_OK;
}

extern "C" void fsp_server_destroy(fsp_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->accepting = false;
        srv->stopping = true;
    }
    srv->cv_dispatch.notify_all();
    if (srv->dispatcher.joinable()) srv->dispatcher.join();
    for (Slot &s : srv->slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.d_counter) cudaFree(s.d_counter);
        if (s.h_args) cudaFreeHost(s.h_args);
        if (s.d_args) cudaFree(s.d_args);
        if (s.h_items) cudaFreeHost(s.h_items);
        if (s.d_items) cudaFree(s.d_items);
    }
    if (srv->arena_mem) cudaFree(srv->arena_mem);
    for (fsp_request *r : srv->live) delete r;  // every handle dies with the server
    delete srv;
}

// ---------------------------------------------------------------- a client
namespace {

struct SNode {
    int32_t lb;
    int32_t d;
    std::vector<int16_t> row;  // prefix in row[0..d)
};

}  // namespace

namespace {

// Open nodes of one depth-first search, stored flat: node i has bound lb[i],
// depth d[i] and its prefix in rows[i * n, i * n + d[i]).  No allocation per
// node; the arrays grow geometrically.
struct FlatStack {
    int n = 0;
    std::vector<int32_t> lb, d;
    std::vector<int16_t> rows;
    size_t size() const { return lb.size(); }
    bool empty() const { return lb.empty(); }
    void push(int32_t l, int32_t dd, const int16_t *prefix) {
        lb.push_back(l);
        d.push_back(dd);
        rows.insert(rows.end(), prefix, prefix + n);
    }
    void pop() {
        lb.pop_back();
        d.pop_back();
        rows.resize(rows.size() - (size_t)n);
    }
    const int16_t *row(size_t i) const { return rows.data() + i * (size_t)n; }
};

// One depth-first search whose pools are bounded by the server, or, with no
// server, each by its own plain launch (fsp_bound_pool_host on a private
// stream): the same search, the same pools, so the two can be compared on
// identical work.
struct SearchState {
    fsp_server *srv = nullptr;
    const fsp_instance *inst = nullptr;
    cudaStream_t stream = nullptr;  // plain mode only
    int16_t *h_rows = nullptr;
    int32_t *h_dep = nullptr, *h_out = nullptr;

    ~SearchState() {
        if (h_rows) cudaFreeHost(h_rows);
        if (h_dep) cudaFreeHost(h_dep);
        if (h_out) cudaFreeHost(h_out);
        if (stream) cudaStreamDestroy(stream);
    }
    fsp_status init(size_t cap, int n) {
        if (!srv && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return FSP_ECUDA;
        if (cudaMallocHost((void **)&h_rows, sizeof(int16_t) * cap * n) != cudaSuccess ||
            cudaMallocHost((void **)&h_dep, sizeof(int32_t) * cap) != cudaSuccess ||
            cudaMallocHost((void **)&h_out, sizeof(int32_t) * cap) != cudaSuccess)
            return FSP_ENOMEM;
        return FSP_OK;
    }
    fsp_status bound(int64_t cnt) {
        fsp_status st;
        if (srv) {
            fsp_request *req = nullptr;
            st = fsp_server_submit(srv, inst, h_rows, h_dep, cnt, h_out, &req);
            if (st != FSP_OK) return st;
            st = fsp_request_wait(req, 600000000LL);  // ten minutes: a stuck server ends the search
            if (st == FSP_ETIMEDOUT) fsp_request_cancel(req);
            fsp_request_release(req);
        } else {
            st = fsp_bound_pool_host(inst, h_rows, h_dep, cnt, h_out, stream);
        }
        if (st != FSP_OK) return st;
        for (int64_t i = 0; i < cnt; ++i)
            if (h_out[i] == FSP_LB_INVALID) return FSP_EBADNODE;
        return FSP_OK;
    }
};

}  // namespace

extern "C" fsp_status fsp_server_search(fsp_server *srv, const fsp_instance *inst, int32_t ub0, int32_t expand,
                                        int64_t node_limit, int16_t *best_perm, int32_t *best_makespan,
                                        int64_t *nodes_bounded) {
    if (!inst || expand < 1 || node_limit < 0) return FSP_EINVAL;
    const int n = inst->n;
    const size_t cap = std::max<size_t>((size_t)expand * n, 1);  // children of `expand` parents
    SearchState S;
    S.srv = srv;
    S.inst = inst;
    fsp_status st = S.init(cap, n);
    if (st != FSP_OK) return st;
    int64_t UB = (int64_t)ub0 + 1, count = 0;
    bool found = false;
    std::vector<int16_t> best(n, 0), zero(n, 0);
    FlatStack stack, parents;
    stack.n = parents.n = n;
    // the root
    std::memset(S.h_rows, 0, sizeof(int16_t) * n);
    S.h_dep[0] = 0;
    st = S.bound(1);
    if (st == FSP_OK) {
        ++count;
        if (S.h_out[0] < UB) stack.push(S.h_out[0], 0, zero.data());
    }
    std::vector<int> first(expand + 1);
    std::vector<char> used(n);
    struct Kid {
        int32_t lb, job;
    };
    std::vector<Kid> kids;
    bool cut = false;
    while (st == FSP_OK && !stack.empty()) {
        if (node_limit && count >= node_limit) {
            cut = true;
            break;
        }
        // selection: the top `expand` live nodes of the stack
        parents.lb.clear();
        parents.d.clear();
        parents.rows.clear();
        while (!stack.empty() && (int)parents.size() < expand) {
            const size_t t = stack.size() - 1;
            if (stack.lb[t] < UB) parents.push(stack.lb[t], stack.d[t], stack.row(t));
            stack.pop();
        }
        if (parents.empty()) break;
        // branching: all children of all selected parents form one pool
        int64_t cnt = 0;
        for (size_t p = 0; p < parents.size(); ++p) {
            first[p] = (int)cnt;
            const int d = parents.d[p];
            const int16_t *prow = parents.row(p);
            std::fill(used.begin(), used.end(), 0);
            for (int i = 0; i < d; ++i) used[prow[i]] = 1;
            for (int j = 0; j < n; ++j) {
                if (used[j]) continue;
                int16_t *r = S.h_rows + (size_t)cnt * n;
                std::memcpy(r, prow, sizeof(int16_t) * n);
                r[d] = (int16_t)j;
                S.h_dep[cnt] = d + 1;
                ++cnt;
            }
        }
        first[parents.size()] = (int)cnt;
        st = S.bound(cnt);
        if (st != FSP_OK) break;
        count += cnt;
        // leaves first: a bounded complete schedule is an incumbent at once
        for (int64_t i = 0; i < cnt; ++i)
            if (S.h_dep[i] == n && S.h_out[i] < UB) {
                UB = S.h_out[i];
                found = true;
                std::memcpy(best.data(), S.h_rows + (size_t)i * n, sizeof(int16_t) * n);
            }
        // elimination and depth-first order: the first selected parent's
        // children end on top, each parent's children by (LB, job)
        for (int p = (int)parents.size() - 1; p >= 0; --p) {
            const int d = parents.d[p];
            if (d + 1 == n) continue;
            kids.clear();
            for (int i = first[p]; i < first[p + 1]; ++i)
                if (S.h_out[i] < UB) kids.push_back(Kid{S.h_out[i], i});
            std::sort(kids.begin(), kids.end(), [&](const Kid &x, const Kid &y) {
                const int jx = S.h_rows[(size_t)x.job * n + d], jy = S.h_rows[(size_t)y.job * n + d];
                return x.lb != y.lb ? x.lb < y.lb : jx < jy;
            });
            for (int t = (int)kids.size() - 1; t >= 0; --t)
                stack.push(kids[t].lb, d + 1, S.h_rows + (size_t)kids[t].job * n);
        }
    }
    if (st != FSP_OK) return st;
    if (nodes_bounded) *nodes_bounded = count;
    if (found) {
        if (best_makespan) *best_makespan = (int32_t)UB;
        if (best_perm) std::memcpy(best_perm, best.data(), sizeof(int16_t) * n);
    }
    if (cut) return FSP_ETIMEDOUT;
    return found ? FSP_OK : FSP_ENOTFOUND;
}

// ---------------------------------------------------------------------------
// fsp_server_solve: cooperating depth-first searchers over one server.
//
// One problem, `searchers` host threads.  Each keeps its own stack of open
// nodes and runs the served search's step (pop up to `expand` live nodes,
// submit all their children as one pool, keep the children below UB) against
// a shared incumbent, so an improvement found by one searcher prunes all of
// them at once.  A searcher whose stack runs dry steals half of the fullest
// stack from its bottom -- the shallowest open nodes, whose subtrees are the
// largest.  The search ends when every stack is empty and no searcher holds
// parents in flight.
namespace {

struct Solve {
    const fsp_instance *inst;
    fsp_server *srv;
    int n, expand, searchers;
    int64_t node_limit;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::vector<SNode>> stacks;
    int busy = 0;                 // searchers holding popped parents
    bool stop = false;            // node limit reached or an error
    fsp_status err = FSP_OK;
    std::atomic<int64_t> ub{0};   // prune iff LB >= ub
    std::atomic<int64_t> count{0};
    bool found = false, cut = false;
    std::vector<int16_t> best;
    int64_t steals = 0;
};

// Takes up to `expand` live nodes for searcher w (its own top, else half of
// the fullest stack's bottom); false when the search is over.
bool take_parents(Solve &S, int w, std::vector<SNode> &parents) {
    std::unique_lock<std::mutex> lk(S.mu);
    for (;;) {
        if (S.stop) return false;
        auto &mine = S.stacks[w];
        // pop live nodes, stealing whenever the own stack runs dry, until some
        // are found or every stack is empty (stale nodes are dropped on the way)
        while (parents.empty()) {
            if (mine.empty()) {
                int victim = -1;
                size_t most = 0;
                for (int v = 0; v < S.searchers; ++v)
                    if (v != w && S.stacks[v].size() > most) {
                        most = S.stacks[v].size();
                        victim = v;
                    }
                if (victim < 0) break;
                auto &vs = S.stacks[victim];
                const size_t take = std::max<size_t>(1, vs.size() / 2);
                // the bottom `take` nodes, kept in stack order
                mine.insert(mine.end(), std::make_move_iterator(vs.begin()),
                            std::make_move_iterator(vs.begin() + (ptrdiff_t)take));
                vs.erase(vs.begin(), vs.begin() + (ptrdiff_t)take);
                ++S.steals;
            }
            const int64_t UB = S.ub.load();
            while (!mine.empty() && (int)parents.size() < S.expand) {
                SNode nd = std::move(mine.back());
                mine.pop_back();
                if (nd.lb < UB) parents.push_back(std::move(nd));
            }
        }
        if (!parents.empty()) {
            ++S.busy;
            return true;
        }
        if (S.busy == 0) {  // nothing open anywhere and nothing in flight: done
            S.stop = true;
            S.cv.notify_all();
            return false;
        }
        S.cv.wait_for(lk, std::chrono::milliseconds(50));
    }
}

void searcher_main(Solve &S, int w) {
    const int n = S.n;
    const size_t cap = (size_t)S.expand * n;
    int16_t *h_rows = nullptr;
    int32_t *h_dep = nullptr, *h_out = nullptr;
    auto fail = [&](fsp_status e) {
        std::lock_guard<std::mutex> g(S.mu);
        if (S.err == FSP_OK) S.err = e;
        S.stop = true;
        S.cv.notify_all();
    };
    if (cudaMallocHost((void **)&h_rows, sizeof(int16_t) * cap * n) != cudaSuccess ||
        cudaMallocHost((void **)&h_dep, sizeof(int32_t) * cap) != cudaSuccess ||
        cudaMallocHost((void **)&h_out, sizeof(int32_t) * cap) != cudaSuccess) {
        if (h_rows) cudaFreeHost(h_rows);
        if (h_dep) cudaFreeHost(h_dep);
        fail(FSP_ENOMEM);
        return;
    }
    std::vector<SNode> parents;
    std::vector<int> first(S.expand + 1);
    std::vector<char> used(n);
    struct Kid {
        int32_t lb, job;
    };
    std::vector<Kid> kids;
    std::vector<SNode> pushed;
    while (take_parents(S, w, parents)) {
        // branching: all children of the popped parents form one pool
        int64_t cnt = 0;
        for (size_t p = 0; p < parents.size(); ++p) {
            first[p] = (int)cnt;
            const SNode &nd = parents[p];
            std::fill(used.begin(), used.end(), 0);
            for (int i = 0; i < nd.d; ++i) used[nd.row[i]] = 1;
            for (int j = 0; j < n; ++j) {
                if (used[j]) continue;
                int16_t *r = h_rows + (size_t)cnt * n;
                std::memcpy(r, nd.row.data(), sizeof(int16_t) * nd.d);
                std::memset(r + nd.d, 0, sizeof(int16_t) * (n - nd.d));
                r[nd.d] = (int16_t)j;
                h_dep[cnt] = nd.d + 1;
                ++cnt;
            }
        }
        first[parents.size()] = (int)cnt;
        fsp_request *req = nullptr;
        fsp_status st = fsp_server_submit(S.srv, S.inst, h_rows, h_dep, cnt, h_out, &req);
        if (st == FSP_OK) {
            st = fsp_request_wait(req, 600000000LL);  // ten minutes: a stuck server ends the search
            if (st == FSP_ETIMEDOUT) fsp_request_cancel(req);
            fsp_request_release(req);
        }
        for (int64_t i = 0; st == FSP_OK && i < cnt; ++i)
            if (h_out[i] == FSP_LB_INVALID) st = FSP_EBADNODE;
        if (st != FSP_OK) {
            fail(st);
            std::lock_guard<std::mutex> g(S.mu);
            --S.busy;
            break;
        }
        const int64_t total = S.count.fetch_add(cnt) + cnt;
        // leaves: the shared incumbent
        for (int64_t i = 0; i < cnt; ++i)
            if (h_dep[i] == n && h_out[i] < S.ub.load()) {
                std::lock_guard<std::mutex> g(S.mu);
                if (h_out[i] < S.ub.load()) {
                    S.ub.store(h_out[i]);
                    S.found = true;
                    std::memcpy(S.best.data(), h_rows + (size_t)i * n, sizeof(int16_t) * n);
                }
            }
        // elimination and depth-first order, as in the served search
        const int64_t UB = S.ub.load();
        pushed.clear();
        for (int p = (int)parents.size() - 1; p >= 0; --p) {
            const SNode &nd = parents[p];
            if (nd.d + 1 == n) continue;
            kids.clear();
            for (int i = first[p]; i < first[p + 1]; ++i)
                if (h_out[i] < UB) kids.push_back(Kid{h_out[i], h_rows[(size_t)i * n + nd.d]});
            std::sort(kids.begin(), kids.end(),
                      [](const Kid &x, const Kid &y) { return x.lb != y.lb ? x.lb < y.lb : x.job < y.job; });
            for (int t = (int)kids.size() - 1; t >= 0; --t) {
                SNode c{kids[t].lb, nd.d + 1, nd.row};
                c.row[nd.d] = (int16_t)kids[t].job;
                pushed.push_back(std::move(c));
            }
        }
        parents.clear();
        {
            std::lock_guard<std::mutex> g(S.mu);
            auto &mine = S.stacks[w];
            mine.insert(mine.end(), std::make_move_iterator(pushed.begin()), std::make_move_iterator(pushed.end()));
            --S.busy;
            if (S.node_limit && total >= S.node_limit) {
                S.cut = true;
                S.stop = true;
            }
            S.cv.notify_all();
        }
    }
    cudaFreeHost(h_rows);
    cudaFreeHost(h_dep);
    cudaFreeHost(h_out);
}

}  // namespace

extern "C" fsp_status fsp_server_solve(fsp_server *srv, const fsp_instance *inst, int32_t ub0, int32_t searchers,
                                       int32_t expand, int64_t node_limit, int16_t *best_perm,
                                       int32_t *best_makespan, int64_t *nodes_bounded, int64_t *steals) {
    if (!srv || !inst || searchers < 1 || searchers > 256 || expand < 1 || node_limit < 0) return FSP_EINVAL;
    Solve S;
    S.inst = inst;
    S.srv = srv;
    S.n = inst->n;
    S.expand = expand;
    S.searchers = searchers;
    S.node_limit = node_limit;
    S.stacks.resize(searchers);
    S.best.assign(inst->n, 0);
    S.ub.store((int64_t)ub0 + 1);
    // the root, bounded through the server like every other pool
    {
        std::vector<int16_t> row(inst->n, 0);
        int32_t dep = 0, lb = 0;
        fsp_request *req = nullptr;
        fsp_status st = fsp_server_submit(srv, inst, row.data(), &dep, 1, &lb, &req);
        if (st != FSP_OK) return st;
        st = fsp_request_wait(req, 600000000LL);
        if (st == FSP_ETIMEDOUT) fsp_request_cancel(req);
        fsp_request_release(req);
        if (st != FSP_OK) return st;
        if (lb == FSP_LB_INVALID) return FSP_EBADNODE;
        S.count = 1;
        if (lb < S.ub.load()) S.stacks[0].push_back(SNode{lb, 0, row});
    }
    std::vector<std::thread> threads;
    threads.reserve(searchers);
    for (int w = 0; w < searchers; ++w) threads.emplace_back(searcher_main, std::ref(S), w);
    for (auto &t : threads) t.join();
    if (nodes_bounded) *nodes_bounded = S.count.load();
    if (steals) *steals = S.steals;
    if (S.err != FSP_OK) return S.err;
    if (S.found) {
        if (best_makespan) *best_makespan = (int32_t)S.ub.load();
        if (best_perm) std::memcpy(best_perm, S.best.data(), sizeof(int16_t) * inst->n);
    }
    if (S.cut) return FSP_ETIMEDOUT;
    return S.found ? FSP_OK : FSP_ENOTFOUND;
}
