// Serving form of the method: requests (one matrix each) arrive at any time;
// a fixed pool of workers, each with its own CUDA stream, echelonises them
// concurrently.  A request is admitted when a worker is free AND its
// workspace fits in the server's device arena (the HBM admission cap); any
// queued request that fits may be admitted, so small requests flow past a
// large one that waits for memory (continuous batching: requests that arrive
// while others run join as slots and memory free up, and their work overlaps
// on the GPU).  A worker that admits a small request (one the batched form's
// one-launch kernels take, of work at most gfe_set_server_group_work) also
// admits every other such queued request with the same flags, up to
// MAX_GROUP, and runs the group as one gfe_batch_echelon call: one launch per
// kind of kernel, one thread block per request.  Results are those of
// gfe_echelon on the same matrix.
#include "gfe.h"
#include "gfe_internal.h"

#include <chrono>
#include <condition_variable>
#include <algorithm>
#include <atomic>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

// first-fit allocator over [0, cap) with 256-byte granules
struct Arena {
    size_t cap = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    void init(size_t c) {
        cap = c;
        free_.clear();
        if (c) free_[0] = c;
    }
    bool take(size_t bytes, size_t *off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void give(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    uint64_t ticket;
    gfe_matrix A;
    gfe_result out;
    uint32_t flags;
    cudaEvent_t ready = nullptr;  // the caller's stream at submit time
    size_t ws = 0, off = 0;
    Clock::time_point t_submit, t_done;
    gfe_status status = GFE_EBUSY;
    std::string err;
};

}  // namespace

struct gfe_server {
    int device = 0;
    char *base = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::map<uint64_t, Req *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    int busy = 0;
    std::vector<std::thread> workers;
};

using gfe::cuda_ok;
using gfe::set_error;

namespace gfe {
bool batch_takes_small(const gfe_matrix &A, uint32_t flags);  // gfe_api.cu
}

// most requests one worker takes together into the one-launch kernels
constexpr size_t MAX_GROUP = 256;
// A request joins a group only if its work m n min(m,n) is at most this: one
// CTA runs about 1e11 mul-adds/s, so larger requests would wait longer in
// the group than the blocked planner takes for them on the whole GPU.
static std::atomic<double> g_group_work{2e7};

static bool takes_group(const Req *r) {
    const double work = (double)r->A.m * (double)r->A.n * (double)std::min(r->A.m, r->A.n);
    return work <= g_group_work.load() && gfe::batch_takes_small(r->A, r->flags);
}

// workspace of a group of small requests (gfe_query_batch_workspace), 0 on error
static size_t group_ws(const std::vector<Req *> &g) {
    std::vector<gfe_matrix> As;
    As.reserve(g.size());
    for (Req *r : g) As.push_back(r->A);
    size_t need = 0;
    if (gfe_query_batch_workspace(As.data(), (int32_t)As.size(), g.front()->flags, &need) != GFE_OK) return 0;
    return need;
}

static void worker_loop(gfe_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        std::vector<Req *> group;  // one request, or small ones run by one gfe_batch_echelon
        size_t gws = 0, goff = 0;
        // admit the first queued request whose workspace fits
        for (;;) {
            if (S->stop && S->queue.empty()) break;
            for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
                Req *r = *it;
                if (takes_group(r)) {
                    std::vector<Req *> g{r};
                    for (auto jt = std::next(it); jt != S->queue.end() && g.size() < MAX_GROUP; ++jt)
                        if ((*jt)->flags == r->flags && takes_group(*jt))
                            g.push_back(*jt);
                    // the largest prefix of the group whose workspace fits
                    bool sized = true;
                    for (;;) {
                        const size_t need = group_ws(g);
                        if (!need) {  // cannot size it as a group: the request goes alone (below)
                            sized = false;
                            break;
                        }
                        if (S->arena.take(need, &goff)) {
                            gws = need;
                            break;
                        }
                        if (g.size() == 1) break;
                        g.resize(g.size() / 2);
                    }
                    if (gws) {
                        for (Req *q : g) S->queue.erase(std::find(S->queue.begin(), S->queue.end(), q));
                        group = std::move(g);
                        break;
                    }
                    if (sized) continue;  // no room now: retried when memory comes free
                }
                size_t off = 0;
                if (S->arena.take(r->ws, &off)) {
                    r->off = off;
                    group.push_back(r);
                    S->queue.erase(it);
                    break;
                }
            }
            if (!group.empty() || S->stop) break;
            S->cv_work.wait(lk);
        }
        if (group.empty()) break;
        ++S->busy;
        lk.unlock();
        gfe_status rc = st ? GFE_OK : GFE_ECUDA;
        for (Req *r : group)
            if (rc == GFE_OK && r->ready && cudaStreamWaitEvent(st, r->ready, 0) != cudaSuccess) rc = GFE_ECUDA;
        if (rc == GFE_OK) {
            if (gws) {  // one call for the group; it returns once queued: wait for its end
                std::vector<gfe_matrix> As;
                std::vector<gfe_result> outs;
                for (Req *r : group) {
                    As.push_back(r->A);
                    outs.push_back(r->out);
                }
                rc = gfe_batch_echelon(As.data(), outs.data(), (int32_t)group.size(), group.front()->flags,
                                       S->base + goff, gws, st);
                if (rc == GFE_OK && !cuda_ok(cudaStreamSynchronize(st), "group sync")) rc = GFE_ECUDA;
            } else {
                Req *job = group.front();
                rc = gfe_echelon(&job->A, &job->out, job->flags, S->base + job->off, job->ws, st);
            }
        }
        for (Req *r : group)
            if (r->ready) {
                cudaEventDestroy(r->ready);
                r->ready = nullptr;
            }
        std::string msg = rc ? gfe_last_error() : "";
        lk.lock();
        --S->busy;
        if (gws) S->arena.give(goff, gws);
        else S->arena.give(group.front()->off, group.front()->ws);
        const Clock::time_point now = Clock::now();
        for (Req *r : group) {
            r->status = rc;
            r->err = msg;
            r->t_done = now;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // memory freed: others may fit now
    }
    lk.unlock();
    if (st) cudaStreamDestroy(st);
}

extern "C" {

gfe_status gfe_set_server_group_work(double max_work) {
    g_group_work.store(max_work);
    return GFE_OK;
}

gfe_status gfe_server_create(gfe_server **out, size_t hbm_cap_bytes, int32_t workers, int32_t device) {
    if (!out || hbm_cap_bytes < 4096 || workers < 1 || workers > 64)
        return (set_error("gfe_server_create: bad arguments"), GFE_EINVAL);
    gfe_server *S = new gfe_server();
    S->device = device;
    if (!cuda_ok(cudaSetDevice(device), "cudaSetDevice") ||
        !cuda_ok(cudaMalloc((void **)&S->base, hbm_cap_bytes), "cudaMalloc of the server arena")) {
        delete S;
        return GFE_ENOMEM;
    }
    S->arena.init(hbm_cap_bytes);
    for (int w = 0; w < workers; ++w) S->workers.emplace_back(worker_loop, S);
    *out = S;
    return GFE_OK;
}

gfe_status gfe_submit(gfe_server *S, const gfe_matrix *A, const gfe_result *out, uint32_t flags, void *stream,
                      uint64_t *ticket) {
    if (!S || !A || !out || !ticket) return (set_error("gfe_submit: NULL argument"), GFE_EINVAL);
    size_t ws = 0;
    gfe_status st = gfe_query_workspace(A, flags, &ws);
    if (st) return st;
    if (!out->rank) return (set_error("out->rank is required"), GFE_EINVAL);
    if (((ws + 255) & ~(size_t)255) > S->arena.cap) {
        set_error("request needs " + std::to_string(ws) + " bytes of workspace, more than the server's cap");
        return GFE_ENOMEM;
    }
    Req *r = new Req();
    if (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r->ready, (cudaStream_t)stream) != cudaSuccess) {
        if (r->ready) cudaEventDestroy(r->ready);
        delete r;
        return (set_error("gfe_submit: cannot order the request after its stream"), GFE_ECUDA);
    }
    r->A = *A;
    r->out = *out;
    r->flags = flags;
    r->ws = ws;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        cudaEventDestroy(r->ready);
        delete r;
        return (set_error("server is shutting down"), GFE_EBUSY);
    }
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return GFE_OK;
}

gfe_status gfe_poll(gfe_server *S, uint64_t ticket, gfe_status *done_status) {
    if (!S || !done_status) return (set_error("gfe_poll: NULL argument"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return (set_error("unknown ticket"), GFE_EINVAL);
    *done_status = it->second->status;
    if (it->second->status != GFE_OK && it->second->status != GFE_EBUSY) set_error(it->second->err);
    return it->second->status == GFE_EBUSY ? GFE_EBUSY : GFE_OK;
}

gfe_status gfe_wait(gfe_server *S, uint64_t ticket, int64_t timeout_us, gfe_status *done_status) {
    if (!S || !done_status) return (set_error("gfe_wait: NULL argument"), GFE_EINVAL);
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return (set_error("unknown ticket"), GFE_EINVAL);
    Req *r = it->second;
    auto pred = [&] { return r->status != GFE_EBUSY; };
    if (timeout_us < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
        return (set_error("gfe_wait: timed out"), GFE_ETIMEOUT);
    *done_status = r->status;
    if (r->status != GFE_OK) set_error(r->err);
    return GFE_OK;
}

gfe_status gfe_server_latency(gfe_server *S, uint64_t ticket, double *us, int32_t release) {
    if (!S || !us) return (set_error("gfe_server_latency: NULL argument"), GFE_EINVAL);
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return (set_error("unknown ticket"), GFE_EINVAL);
    Req *r = it->second;
    if (r->status == GFE_EBUSY) return GFE_EBUSY;
    *us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    if (release) {
        S->all.erase(it);
        delete r;
    }
    return GFE_OK;
}

gfe_status gfe_server_destroy(gfe_server *S) {
    if (!S) return GFE_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->all) delete kv.second;
    if (S->base) cudaFree(S->base);
    delete S;
    return GFE_OK;
}

}  // extern "C"
