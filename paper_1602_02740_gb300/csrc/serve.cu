// Serving: continuous batching of multiply requests on one GPU.
//
// tc_serve_submit admits a request when the context's scratch budget and a
// slot allow it and queues it; a worker thread (started on the first submit)
// repeatedly takes every queued request, groups the requests by padded size
// class, and launches each group's whole Toom-Cook pipeline (operand copies
// into padded rows, every level's kernels, result copies) on one of several
// CUDA streams, so groups that arrive while others run overlap on the device.
// Group scratch comes from a stream-ordered memory pool owned by the server
// (allocated and freed in stream order, cached between groups).  Completion
// is observed by polling one event per group; latency is submit -> completion
// seen by the worker.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_internal.h"

namespace tc {

namespace {
double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct Request {
    uint64_t ticket;
    const uint32_t* a;
    size_t na;
    const uint32_t* b;
    size_t nb;
    uint32_t* out;
    size_t cls;       // padded balanced length
    size_t need;      // scratch bytes reserved at admission
    double t_submit;
    int state;        // 0 queued, 1 running, 2 done, < 0 error status
};

struct Group {
    std::vector<Request*> reqs;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    size_t bytes = 0;
    int slot = -1;    // index of this group's bounded-wait error word in Server::err_host
};

struct Server {
    tc_ctx* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> all;
    std::vector<Group*> inflight;  // worker thread only
    std::thread worker;
    bool stopping = false;
    uint64_t next_ticket = 1;
    size_t reserved = 0, slots_used = 0;
    size_t budget = 0;
    static constexpr size_t kMaxSlots = 4096;
    static constexpr size_t kMaxGroup = 1024;
    static constexpr size_t kMaxGroupLimbs = (size_t)1 << 26;
    static constexpr int kStreams = 4;
    cudaStream_t streams[kStreams] = {};
    int rr = 0;
    cudaMemPool_t pool = nullptr;
    // pinned host words, one per group in flight: each group's bounded-wait error
    // word is copied here before its scratch is freed (worker thread only)
    int* err_host = nullptr;
    std::vector<int> free_slots;
    // statistics
    std::vector<double> lat_ms;
    double first_submit = -1, last_done = 0, bits = 0;

    ~Server();
    void run();
    void launch(std::vector<Request*>& reqs);
    bool poll_inflight();
};

static size_t group_bytes(tc_ctx* ctx, size_t count, size_t s) {
    const tc_opts o = plan_for(ctx, s);
    const BatchLayout L = layout_for(count, s, o, false);
    return L.total + 2 * align256(count * s * 4) + align256(count * 2 * s * 4);
}

Server::~Server() {
    for (auto& kv : all) delete kv.second;
    if (err_host) cudaFreeHost(err_host);
}

void Server::launch(std::vector<Request*>& reqs) {
    // group by size class, bounded group size
    std::sort(reqs.begin(), reqs.end(), [](Request* x, Request* y) { return x->cls < y->cls; });
    size_t i = 0;
    while (i < reqs.size()) {
        size_t j = i, limbs = 0;
        const size_t s = reqs[i]->cls;
        while (j < reqs.size() && reqs[j]->cls == s && j - i < kMaxGroup &&
               (limbs == 0 || limbs + s <= kMaxGroupLimbs)) {
            limbs += s;
            ++j;
        }
        Group* g = new Group();
        g->reqs.assign(reqs.begin() + i, reqs.begin() + j);
        g->st = streams[rr++ % kStreams];
        const size_t c = g->reqs.size();
        const tc_opts o = plan_for(ctx, s);
        const BatchLayout L = layout_for(c, s, o, false);
        const size_t rows_end = L.total + 2 * align256(c * s * 4) + align256(c * 2 * s * 4);
        g->bytes = rows_end + 256;  // + the group's bounded-wait error word
        g->slot = free_slots.back();
        free_slots.pop_back();
        err_host[g->slot] = 0;
        cudaError_t e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
        void* scratch = nullptr;
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&scratch, g->bytes, pool, g->st);
        tc_status status = TC_OK;
        if (e == cudaSuccess) {
            char* base = (char*)scratch;
            uint32_t* rA = (uint32_t*)(base + L.total);
            uint32_t* rB = (uint32_t*)(base + L.total + align256(c * s * 4));
            uint32_t* rO = (uint32_t*)(base + L.total + 2 * align256(c * s * 4));
            int* err_dev = (int*)(base + rows_end);
            e = cudaMemsetAsync(rA, 0, 2 * align256(c * s * 4), g->st);
            if (e == cudaSuccess) e = cudaMemsetAsync(err_dev, 0, sizeof(int), g->st);
            for (size_t k = 0; k < c && e == cudaSuccess; ++k) {
                Request* r = g->reqs[k];
                if (r->na) e = cudaMemcpyAsync(rA + k * s, r->a, r->na * 4, cudaMemcpyDeviceToDevice, g->st);
                if (e == cudaSuccess && r->nb)
                    e = cudaMemcpyAsync(rB + k * s, r->b, r->nb * 4, cudaMemcpyDeviceToDevice, g->st);
            }
            if (e == cudaSuccess)
                status = run_uniform(L, base, c, s, rA, (long)s, rB, (long)s, rO, (long)(2 * s), false,
                                     g->st, nullptr, err_dev);
            for (size_t k = 0; k < c && e == cudaSuccess && status == TC_OK; ++k) {
                Request* r = g->reqs[k];
                if (r->na + r->nb)
                    e = cudaMemcpyAsync(r->out, rO + k * 2 * s, (r->na + r->nb) * 4,
                                        cudaMemcpyDeviceToDevice, g->st);
            }
            if (e == cudaSuccess && status == TC_OK)
                e = cudaMemcpyAsync(err_host + g->slot, err_dev, sizeof(int), cudaMemcpyDeviceToHost,
                                    g->st);
            cudaError_t e2 = cudaFreeAsync(scratch, g->st);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && status == TC_OK) e = cudaEventRecord(g->done, g->st);
        if (e != cudaSuccess || status != TC_OK) {
            const int err = status != TC_OK ? (int)status : (int)tc_fail_cuda(e);
            std::lock_guard<std::mutex> lk(mu);
            for (Request* r : g->reqs) {
                r->state = err;
                reserved -= r->need;
                --slots_used;
            }
            if (g->done) cudaEventDestroy(g->done);
            if (scratch || g->done) cudaStreamSynchronize(g->st);  // the slot may be in a copy
            free_slots.push_back(g->slot);
            delete g;
        } else {
            inflight.push_back(g);
        }
        i = j;
    }
}

bool Server::poll_inflight() {
    bool any = false;
    for (size_t i = 0; i < inflight.size();) {
        Group* g = inflight[i];
        const cudaError_t q = cudaEventQuery(g->done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = now_s();
        const bool timed_out = q == cudaSuccess && err_host[g->slot] != 0;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Request* r : g->reqs) {
                r->state = q != cudaSuccess ? (int)tc_fail_cuda(q) : timed_out ? (int)TC_ETIMEOUT : 2;
                reserved -= r->need;
                --slots_used;
                if (q == cudaSuccess && !timed_out) {
                    lat_ms.push_back((t - r->t_submit) * 1e3);
                    bits += 32.0 * (double)(r->na + r->nb);
                    last_done = std::max(last_done, t);
                }
            }
        }
        cudaEventDestroy(g->done);
        free_slots.push_back(g->slot);
        delete g;
        inflight[i] = inflight.back();
        inflight.pop_back();
        any = true;
    }
    return any;
}

void Server::run() {
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (queue.empty() && inflight.empty()) {
                if (stopping) break;
                cv.wait_for(lk, std::chrono::microseconds(500));
            }
            while (!queue.empty()) {
                Request* r = queue.front();
                queue.pop_front();
                r->state = 1;
                batch.push_back(r);
            }
        }
        // products with an empty operand are zero: no GPU work
        std::vector<Request*> work;
        for (Request* r : batch) {
            if (r->na == 0 || r->nb == 0) {
                cudaError_t e = (r->na + r->nb) ? cudaMemsetAsync(r->out, 0, (r->na + r->nb) * 4, streams[0])
                                                : cudaSuccess;
                if (e == cudaSuccess) e = cudaStreamSynchronize(streams[0]);
                const double t = now_s();
                std::lock_guard<std::mutex> lk(mu);
                r->state = e == cudaSuccess ? 2 : (int)tc_fail_cuda(e);
                reserved -= r->need;
                --slots_used;
                if (e == cudaSuccess) {
                    lat_ms.push_back((t - r->t_submit) * 1e3);
                    bits += 32.0 * (double)(r->na + r->nb);
                    last_done = std::max(last_done, t);
                }
            } else {
                work.push_back(r);
            }
        }
        if (!work.empty()) launch(work);
        const bool done_any = poll_inflight();
        if (batch.empty() && !done_any && !inflight.empty())
            std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

static std::mutex g_server_mu;

// The context's server, started on first use.  The caller holds g_server_mu.
static Server* get_server_locked(tc_ctx* ctx, tc_status* st) {
    *st = TC_OK;
    if (ctx->server) return ctx->server;
    Server* s = new Server();
    s->ctx = ctx;
    s->budget = ctx->budget;
    cudaError_t e = cudaSetDevice(ctx->device);
    for (int i = 0; i < Server::kStreams && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = (uint64_t)ctx->budget;  // cache freed group scratch up to the budget
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) {
        // at most one group per admitted request is in flight
        e = cudaHostAlloc(&s->err_host, Server::kMaxSlots * sizeof(int), cudaHostAllocDefault);
        if (e == cudaSuccess)
            for (int i = (int)Server::kMaxSlots - 1; i >= 0; --i) s->free_slots.push_back(i);
    }
    if (e != cudaSuccess) {
        *st = tc_fail_cuda(e);
        for (auto x : s->streams)
            if (x) cudaStreamDestroy(x);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return nullptr;
    }
    s->worker = std::thread([s] { s->run(); });
    ctx->server = s;
    return s;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_serve_submit(tc_ctx* ctx, const uint32_t* a, size_t na, const uint32_t* b,
                                     size_t nb, uint32_t* out, uint64_t* ticket) {
    if (!ctx || !ticket || (na && !a) || (nb && !b) || (na + nb && !out)) return TC_EINVAL;
    const size_t L = std::max(na, nb);
    if (L > ((size_t)1 << 28)) return TC_EINVAL;
    const size_t cls = L ? size_class(L) : 0;
    if (cls && !plan_valid(plan_for(ctx, cls), cls)) return TC_EINVAL;
    const size_t need = cls ? group_bytes(ctx, 1, cls) : 0;
    if (need > ctx->budget) return TC_ENOMEM;  // could never be admitted
    tc_status st;
    Request* r = new Request{0, a, na, b, nb, out, cls, need, now_s(), 0};
    Server* s = nullptr;
    {
        // g_server_mu held throughout: tc_serve_stop cannot detach the server meanwhile
        std::lock_guard<std::mutex> glk(g_server_mu);
        s = get_server_locked(ctx, &st);
        if (!s) {
            delete r;
            return st;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping || s->slots_used >= Server::kMaxSlots || s->reserved + need > s->budget) {
            delete r;
            return TC_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->reserved += need;
        ++s->slots_used;
        if (s->first_submit < 0) s->first_submit = r->t_submit;
        s->queue.push_back(r);
        s->all[r->ticket] = r;
        *ticket = r->ticket;  // r may be released by a poll once the locks are dropped
        s->cv.notify_one();
    }
    return TC_OK;
}

// The server is read under g_server_mu, which tc_serve_stop holds while it
// detaches the server, so a poll never sees a server that is being deleted.
// A final state (done or an error) releases the ticket: the worker no longer
// refers to a request once its state is final.
extern "C" tc_status tc_serve_poll(tc_ctx* ctx, uint64_t ticket) {
    if (!ctx) return TC_EINVAL;
    std::lock_guard<std::mutex> glk(g_server_mu);
    Server* s = ctx->server;
    if (!s) return TC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return TC_EINVAL;
    const int state = it->second->state;
    if (state == 1 || state == 0) return TC_EPENDING;
    delete it->second;
    s->all.erase(it);
    return state == 2 ? TC_OK : (tc_status)state;
}

extern "C" tc_status tc_serve_stats(tc_ctx* ctx, double* p50_ms, double* p99_ms, double* bits_per_s,
                                    uint64_t* completed) {
    if (!ctx) return TC_EINVAL;
    double p50 = 0, p99 = 0, bps = 0;
    uint64_t n = 0;
    std::vector<double> lat;
    double bits = 0, t0 = 0, t1 = 0;
    {
        std::lock_guard<std::mutex> glk(g_server_mu);  // see tc_serve_poll
        if (Server* s = ctx->server) {
            std::lock_guard<std::mutex> lk(s->mu);
            lat = s->lat_ms;
            bits = s->bits;
            t0 = s->first_submit;
            t1 = s->last_done;
        }
    }
    {
        n = lat.size();
        if (n) {
            std::sort(lat.begin(), lat.end());
            p50 = lat[(size_t)(0.50 * (n - 1))];
            p99 = lat[(size_t)(0.99 * (n - 1))];
            if (t1 > t0) bps = bits / (t1 - t0);
        }
    }
    if (p50_ms) *p50_ms = p50;
    if (p99_ms) *p99_ms = p99;
    if (bits_per_s) *bits_per_s = bps;
    if (completed) *completed = n;
    return TC_OK;
}

extern "C" tc_status tc_serve_stop(tc_ctx* ctx) {
    if (!ctx) return TC_EINVAL;
    Server* s;
    {
        std::lock_guard<std::mutex> lk(g_server_mu);
        s = ctx->server;
        ctx->server = nullptr;
    }
    if (!s) return TC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_one();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(ctx->device);
    for (auto x : s->streams)
        if (x) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return TC_OK;
}
