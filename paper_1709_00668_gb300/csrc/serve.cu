// Serving loop: many tensor streams, each absorbed by its own SamBaTen
// context (Alg. 1 per batch), updated concurrently on one GPU.
//
// The paper absorbs a single stream.  Here a server keeps every stream's
// store, factors and marginals resident on the device and runs update
// batches from many streams at once: `slots` worker threads each drive one
// sbt_update at a time, on the CUDA streams of that tensor stream's own
// context, so the kernels of different streams' updates overlap on the GPU.
// A queued batch is admitted as soon as a slot is free and the device bytes
// its stream will hold after the update (sbt_update_bytes, computed on the
// host) fit the memory budget together with every other stream's bytes.
// Batches of one stream run one at a time in submission order; batches of
// different streams are admitted in arrival order, skipping those that do
// not fit yet.  Every kernel reduces in a fixed order, so a stream's results
// do not depend on which other batches shared the GPU.
//
// batch_als: one worker admits up to `slots` batches at a time.  Each runs
// sbt_update's steps up to the start of its summary ALS on its own context's
// stream; the pending ALS of those whose streams take the persistent ALS
// (CUDA-core path) then run together, up to PA_MAX_SETS compatible updates
// per persistent cooperative launch on the server's stream (ordered after
// the contexts' streams by events, and they after it); then each update
// matches and commits.  A set's arithmetic inside the launch is its own, so
// every stream's result equals its update alone.
#include "sambaten.h"
#include "sbt_internal.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

sbt_status fail(sbt_status s, const std::string &msg) {
    sbt::set_last_error(msg);
    return s;
}

struct Request {
    uint64_t ticket = 0;
    int32_t sid = 0;
    sbt_tensor X{};
    Clock::time_point t_submit, t_start, t_end;
    bool done = false;
    sbt_request_result res{};
    std::string err;  // message of a failed batch, handed to the thread that waits for it
};

struct Stream {
    sbt_ctx *ctx = nullptr;
    std::deque<Request *> queue;  // not yet started, in submission order
    bool busy = false;            // a batch of this stream is in flight
    bool closing = false;
    uint64_t bytes = 0;           // device bytes held (or reserved for the batch in flight)
};

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    const double f = pos - (double)lo;
    return v[lo] * (1.0 - f) + v[hi] * f;
}

}  // namespace

struct sbt_server {
    sbt_server_options opt{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers: a batch may be admissible
    std::condition_variable cv_done;  // waiters: a batch finished / a stream went idle
    std::map<int32_t, Stream> streams;
    std::deque<int32_t> ready;  // streams with a queued batch and none in flight, by arrival
    std::unordered_map<uint64_t, Request *> requests;
    int32_t next_sid = 1;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    // accounting
    uint64_t resident = 0, peak_resident = 0;
    int64_t in_flight = 0, queued = 0;
    int64_t submitted = 0, completed = 0, failed = 0, slices = 0;
    std::vector<double> lat_total, lat_service;
    Clock::time_point t_reset, busy_since;
    double busy_ms = 0.0;
    int64_t waiters = 0;  // threads inside sbt_server_wait (destroy frees nothing before they leave)
    // batch_als: the server's stream, events, descriptor and barrier words
    cudaStream_t bst = nullptr;
    std::vector<cudaEvent_t> bev;  // PA_MAX_SETS + 1
    sbt::AlsDesc *bdesc = nullptr;
    unsigned *bsync = nullptr;     // the grid barrier's words, then the err word
    unsigned *h_berr = nullptr;    // pinned copy of the err word
    int64_t als_launches = 0, als_sets = 0;

    void worker();
    void worker_batched();
    // run one admitted batch of items (the lock not held)
    struct Item {
        int32_t sid = 0;
        Request *q = nullptr;
        sbt_ctx *ctx = nullptr;
        sbt_status st = SBT_OK;
        std::string err;
        bool deferred = false;
        int64_t K = 0;
        uint64_t bytes = 0;
    };
    Item start_locked(int32_t sid);
    void finish_item_locked(Item &it);
    void run_items(std::vector<Item> &items);
    // the first admissible stream of `ready` (-1: none); fails batches that can never fit
    int32_t pick_locked();
    void finish_locked(Request *q, sbt_status st);
};

void sbt_server::finish_locked(Request *q, sbt_status st) {
    q->t_end = Clock::now();
    q->done = true;
    q->res.status = st;
    q->res.stream = q->sid;
    q->res.queue_ms = ms_between(q->t_submit, q->t_start);
    q->res.service_ms = ms_between(q->t_start, q->t_end);
    q->res.total_ms = ms_between(q->t_submit, q->t_end);
    if (st == SBT_OK) {
        completed += 1;
        slices += q->X.K;
        lat_total.push_back(q->res.total_ms);
        lat_service.push_back(q->res.service_ms);
    } else {
        failed += 1;
    }
}

int32_t sbt_server::pick_locked() {
    for (auto it = ready.begin(); it != ready.end();) {
        const int32_t sid = *it;
        Stream &s = streams[sid];
        Request *q = s.queue.front();
        uint64_t after = 0;
        sbt_status st = sbt_update_bytes(s.ctx, q->X.K, &after);
        if (st == SBT_OK && after > opt.mem_budget) {
            st = SBT_E_NOMEM;
            sbt::set_last_error("batch needs more device memory than the whole budget");
        }
        if (st != SBT_OK) {  // can never run: fail it, keep the stream's order
            s.queue.pop_front();
            queued -= 1;
            q->err = sbt_last_error();
            q->t_start = Clock::now();
            finish_locked(q, st);
            if (s.queue.empty()) {
                it = ready.erase(it);
            } else {
                ++it;
            }
            cv_done.notify_all();
            continue;
        }
        const uint64_t grow = after > s.bytes ? after - s.bytes : 0;
        if (resident + grow <= opt.mem_budget) {
            ready.erase(it);
            resident += grow;
            s.bytes += grow;
            peak_resident = std::max(peak_resident, resident);
            return sid;
        }
        ++it;
    }
    return -1;
}

// The first queued batch of stream sid goes in flight.
sbt_server::Item sbt_server::start_locked(int32_t sid) {
    Stream &s = streams[sid];
    Item it;
    it.sid = sid;
    it.q = s.queue.front();
    it.ctx = s.ctx;
    s.queue.pop_front();
    queued -= 1;
    s.busy = true;
    if (in_flight == 0) busy_since = Clock::now();
    in_flight += 1;
    it.q->t_start = Clock::now();
    return it;
}

// A batch in flight is done: the stream's bytes, the result, the next batch.
void sbt_server::finish_item_locked(Item &it) {
    Stream &s = streams[it.sid];
    resident = resident - s.bytes + it.bytes;
    s.bytes = it.bytes;
    it.q->res.K = it.K;
    it.q->err = it.err;
    finish_locked(it.q, it.st);
    in_flight -= 1;
    if (in_flight == 0) busy_ms += ms_between(busy_since, Clock::now());
    s.busy = false;
    if (!s.queue.empty()) ready.push_back(it.sid);
}

void sbt_server::worker() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        int32_t sid = -1;
        cv_work.wait(lock, [&] {
            if (stop) return true;
            sid = pick_locked();
            return sid >= 0;
        });
        if (sid < 0) return;  // stop
        Item it = start_locked(sid);
        lock.unlock();
        it.st = sbt_update(it.ctx, &it.q->X);
        if (it.st == SBT_OK) it.st = sbt_factors(it.ctx, nullptr, nullptr, nullptr, nullptr, &it.K);
        if (it.st != SBT_OK) it.err = sbt_last_error();
        sbt_device_bytes(it.ctx, &it.bytes);
        lock.lock();
        finish_item_locked(it);
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

// batch_als: admit up to `slots` batches, run them (their summary ALS
// batched), finish them; again.
void sbt_server::worker_batched() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        std::vector<Item> items;
        cv_work.wait(lock, [&] {
            if (stop) return true;
            const int32_t sid = pick_locked();
            if (sid >= 0) items.push_back(start_locked(sid));
            return !items.empty();
        });
        if (items.empty()) return;  // stop
        for (int32_t sid; (int)items.size() < opt.slots && (sid = pick_locked()) >= 0;)
            items.push_back(start_locked(sid));
        lock.unlock();
        run_items(items);
        lock.lock();
        for (Item &it : items) finish_item_locked(it);
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

void sbt_server::run_items(std::vector<Item> &items) {
    // 1. every update up to its summary ALS (the whole update where it cannot wait)
    for (Item &it : items) {
        it.st = sbt::update_deferred(it.ctx, &it.q->X, &it.deferred);
        if (it.st != SBT_OK) it.err = sbt_last_error();
    }
    // 2. the pending ALS, up to PA_MAX_SETS compatible sets per persistent launch
    std::vector<Item *> pend;
    for (Item &it : items)
        if (it.st == SBT_OK && it.deferred) pend.push_back(&it);
    std::vector<char> taken(pend.size(), 0);
    for (size_t a = 0; a < pend.size(); ++a) {
        if (taken[a]) continue;
        std::vector<Item *> grp;
        std::vector<sbt::AlsDesc> ds;
        std::vector<cudaStream_t> sts;
        int sms = 0;
        for (size_t b = a; b < pend.size() && (int)grp.size() < sbt::PA_MAX_SETS; ++b) {
            if (taken[b]) continue;
            sbt::AlsDesc d;
            cudaStream_t st = nullptr;
            int ns = 0;
            if (sbt::deferred_als(pend[b]->ctx, &d, &st, &ns) != SBT_OK) continue;
            if (!ds.empty() && !sbt::persistent_compatible(ds[0], d)) continue;
            taken[b] = 1;
            grp.push_back(pend[b]);
            ds.push_back(d);
            sts.push_back(st);
            sms = ns;
        }
        int max_iters = 1;
        for (const sbt::AlsDesc &d : ds) max_iters = std::max(max_iters, d.max_iters);
        cudaError_t e = cudaSuccess;
        for (size_t k = 0; k < grp.size() && e == cudaSuccess; ++k) {
            e = cudaEventRecord(bev[k], sts[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(bst, bev[k], 0);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(bsync + sbt::PA_SYNC_WORDS, 0, sizeof(unsigned), bst);
        if (e == cudaSuccess)
            e = sbt::launch_als_persistent(ds.data(), (int)ds.size(), bdesc, max_iters, bsync, bsync + sbt::PA_SYNC_WORDS,
                                           sms, bst);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_berr, bsync + sbt::PA_SYNC_WORDS, sizeof(unsigned), cudaMemcpyDeviceToHost, bst);
        const cudaError_t er = cudaEventRecord(bev[sbt::PA_MAX_SETS], bst);
        if (e == cudaSuccess) e = er;
        for (size_t k = 0; k < grp.size() && er == cudaSuccess; ++k) cudaStreamWaitEvent(sts[k], bev[sbt::PA_MAX_SETS], 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(bst);
        const bool timeout = e == cudaSuccess && (*h_berr & sbt::ERR_TIMEOUT);
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lock(mu);
            als_launches += 1;
            als_sets += (int64_t)grp.size();
        }
        if (e != cudaSuccess || timeout) {
            for (Item *it : grp) {
                sbt::update_abandon(it->ctx);
                it->st = timeout ? SBT_E_TIMEOUT : SBT_E_CUDA;
                it->err = timeout ? std::string("batched ALS: a grid barrier gave up")
                                  : std::string("batched ALS launch: ") + cudaGetErrorString(e);
            }
        }
    }
    // 3. match and commit
    for (Item *it : pend)
        if (it->st == SBT_OK) {
            it->st = sbt::update_complete(it->ctx);
            if (it->st != SBT_OK) it->err = sbt_last_error();
        }
    for (Item &it : items) {
        if (it.st == SBT_OK) {
            it.st = sbt_factors(it.ctx, nullptr, nullptr, nullptr, nullptr, &it.K);
            if (it.st != SBT_OK) it.err = sbt_last_error();
        }
        sbt_device_bytes(it.ctx, &it.bytes);
    }
}

extern "C" sbt_status sbt_server_default_options(sbt_server_options *o) {
    if (!o) return fail(SBT_E_INVALID, "null options");
    o->slots = 4;
    o->mem_budget = 0;
    o->device = -1;
    o->batch_als = 0;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_create(const sbt_server_options *o, sbt_server **out) {
    if (!out) return fail(SBT_E_INVALID, "null output pointer");
    *out = nullptr;
    sbt_server_options opt;
    sbt_server_default_options(&opt);
    if (o) opt = *o;
    if (opt.slots <= 0) opt.slots = 4;
    if (opt.slots > 64) return fail(SBT_E_INVALID, "slots must be <= 64");
    if (opt.batch_als != 0 && opt.batch_als != 1) return fail(SBT_E_INVALID, "batch_als must be 0 or 1");
    int dev = opt.device;
    if (dev < 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (opt.mem_budget == 0) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaError_t e = cudaSetDevice(dev);
        size_t fr = 0, tot = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
        cudaSetDevice(prev);
        if (e != cudaSuccess) return fail(SBT_E_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
        opt.mem_budget = (uint64_t)(0.9 * (double)fr);
    }
    sbt_server *srv = new sbt_server();
    srv->opt = opt;
    srv->device = dev;
    srv->t_reset = Clock::now();
    if (opt.batch_als) {
        // the batched launches' stream, events, descriptors and barrier words
        int prev = 0;
        cudaGetDevice(&prev);
        cudaError_t e = cudaSetDevice(dev);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&srv->bst, cudaStreamNonBlocking);
        for (int k = 0; k <= sbt::PA_MAX_SETS && e == cudaSuccess; ++k) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) srv->bev.push_back(ev);
        }
        if (e == cudaSuccess) e = cudaMalloc(&srv->bdesc, sbt::PA_MAX_SETS * sizeof(sbt::AlsDesc));
        if (e == cudaSuccess) e = cudaMalloc(&srv->bsync, (sbt::PA_SYNC_WORDS + 1) * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMallocHost(&srv->h_berr, sizeof(unsigned));
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            sbt_server_destroy(srv);
            return fail(SBT_E_CUDA, std::string("batched ALS resources: ") + cudaGetErrorString(e));
        }
        srv->workers.emplace_back([srv] { srv->worker_batched(); });
    } else {
        for (int w = 0; w < opt.slots; ++w) srv->workers.emplace_back([srv] { srv->worker(); });
    }
    *out = srv;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_open_stream(sbt_server *srv, const sbt_tensor *X0, int32_t R,
                                             const sbt_options *opts, int32_t *sid) {
    if (!srv || !X0 || !opts || !sid) return fail(SBT_E_INVALID, "null argument");
    if (X0->I < 1 || X0->J < 1 || X0->K < 1) return fail(SBT_E_SHAPE, "X0 must be non-empty");
    // the store alone must fit before anything is allocated
    const int64_t kcap = opts->K_capacity > 0 ? opts->K_capacity : 2 * X0->K;
    const uint64_t store_bytes =
        (uint64_t)std::max<int64_t>(kcap, X0->K + 1) * (uint64_t)X0->I * (uint64_t)((X0->J + 7) / 8 * 8) *
        (X0->dtype == SBT_F64 ? 8u : 4u);
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (srv->stop) return fail(SBT_E_STATE, "server is shutting down");
        if (srv->resident + store_bytes > srv->opt.mem_budget)
            return fail(SBT_E_NOMEM, "stream store does not fit the server's memory budget");
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    sbt_options o = *opts;
    sbt_ctx *ctx = nullptr;
    sbt_status st = sbt_init(X0, R, &o, &ctx);
    uint64_t bytes = 0;
    if (st == SBT_OK) st = sbt_device_bytes(ctx, &bytes);
    cudaSetDevice(prev);
    if (st != SBT_OK) {
        if (ctx) sbt_destroy(ctx);
        return st;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->resident + bytes > srv->opt.mem_budget) {
        sbt_destroy(ctx);
        return fail(SBT_E_NOMEM, "stream does not fit the server's memory budget");
    }
    const int32_t id = srv->next_sid++;
    Stream &s = srv->streams[id];
    s.ctx = ctx;
    s.bytes = bytes;
    srv->resident += bytes;
    srv->peak_resident = std::max(srv->peak_resident, srv->resident);
    *sid = id;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_submit(sbt_server *srv, int32_t sid, const sbt_tensor *X_new, uint64_t *ticket) {
    if (!srv || !X_new || !ticket) return fail(SBT_E_INVALID, "null argument");
    if (X_new->K < 1) return fail(SBT_E_SHAPE, "empty batch");
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->streams.find(sid);
    if (it == srv->streams.end() || it->second.closing) return fail(SBT_E_INVALID, "unknown stream");
    if (srv->stop) return fail(SBT_E_STATE, "server is shutting down");
    Request *q = new Request();
    q->ticket = srv->next_ticket++;
    q->sid = sid;
    q->X = *X_new;
    q->t_submit = Clock::now();
    Stream &s = it->second;
    const bool was_idle = s.queue.empty() && !s.busy;
    s.queue.push_back(q);
    if (was_idle) srv->ready.push_back(sid);
    srv->requests[q->ticket] = q;
    srv->queued += 1;
    srv->submitted += 1;
    *ticket = q->ticket;
    srv->cv_work.notify_one();
    return SBT_OK;
}

extern "C" sbt_status sbt_server_wait(sbt_server *srv, uint64_t ticket, int32_t timeout_ms,
                                      sbt_request_result *res) {
    if (!srv) return fail(SBT_E_INVALID, "null server");
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->requests.find(ticket);
    if (it == srv->requests.end()) return fail(SBT_E_INVALID, "unknown ticket");
    Request *q = it->second;
    auto pred = [&] { return q->done; };
    srv->waiters += 1;
    bool ok = true;
    if (timeout_ms < 0) srv->cv_done.wait(lock, pred);
    else ok = srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred);
    srv->waiters -= 1;
    if (srv->waiters == 0) srv->cv_done.notify_all();  // a destroy may wait for the last waiter
    if (!ok) return fail(SBT_E_TIMEOUT, "batch not finished within the timeout");
    if (res) *res = q->res;
    // a failed batch's message becomes this thread's last error
    if (q->res.status != SBT_OK) sbt::set_last_error(q->err);
    srv->requests.erase(it);
    delete q;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_stream_ctx(sbt_server *srv, int32_t sid, sbt_ctx **ctx) {
    if (!srv || !ctx) return fail(SBT_E_INVALID, "null argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->streams.find(sid);
    if (it == srv->streams.end()) return fail(SBT_E_INVALID, "unknown stream");
    if (it->second.busy || !it->second.queue.empty()) return fail(SBT_E_STATE, "stream has batches queued or in flight");
    *ctx = it->second.ctx;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_close_stream(sbt_server *srv, int32_t sid) {
    if (!srv) return fail(SBT_E_INVALID, "null server");
    std::unique_lock<std::mutex> lock(srv->mu);
    auto it = srv->streams.find(sid);
    if (it == srv->streams.end() || it->second.closing) return fail(SBT_E_INVALID, "unknown stream");
    it->second.closing = true;
    srv->cv_done.wait(lock, [&] { return !srv->streams[sid].busy && srv->streams[sid].queue.empty(); });
    Stream &s = srv->streams[sid];
    sbt_ctx *ctx = s.ctx;
    srv->resident -= s.bytes;
    srv->streams.erase(sid);
    lock.unlock();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    sbt_destroy(ctx);
    cudaSetDevice(prev);
    srv->cv_work.notify_all();  // memory freed: batches waiting for it may fit now
    return SBT_OK;
}

extern "C" sbt_status sbt_server_stats(sbt_server *srv, sbt_serving_stats *st) {
    if (!srv || !st) return fail(SBT_E_INVALID, "null argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    const auto now = Clock::now();
    st->submitted = srv->submitted;
    st->completed = srv->completed;
    st->failed = srv->failed;
    st->queued = srv->queued;
    st->in_flight = srv->in_flight;
    st->streams = (int64_t)srv->streams.size();
    st->resident_bytes = srv->resident;
    st->peak_resident_bytes = srv->peak_resident;
    st->mem_budget = srv->opt.mem_budget;
    st->latency_p50_ms = percentile(srv->lat_total, 0.5);
    st->latency_p99_ms = percentile(srv->lat_total, 0.99);
    st->service_p50_ms = percentile(srv->lat_service, 0.5);
    st->service_p99_ms = percentile(srv->lat_service, 0.99);
    const double el = ms_between(srv->t_reset, now);
    const double busy = srv->busy_ms + (srv->in_flight > 0 ? ms_between(srv->busy_since, now) : 0.0);
    st->busy_fraction = el > 0 ? busy / el : 0.0;
    st->slices = srv->slices;
    st->elapsed_s = el / 1e3;
    st->als_launches = srv->als_launches;
    st->als_sets = srv->als_sets;
    return SBT_OK;
}

extern "C" sbt_status sbt_server_stats_reset(sbt_server *srv) {
    if (!srv) return fail(SBT_E_INVALID, "null server");
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->submitted = srv->completed = srv->failed = srv->slices = 0;
    srv->lat_total.clear();
    srv->lat_service.clear();
    srv->t_reset = Clock::now();
    srv->busy_ms = 0.0;
    srv->als_launches = srv->als_sets = 0;
    if (srv->in_flight > 0) srv->busy_since = srv->t_reset;
    srv->peak_resident = srv->resident;
    return SBT_OK;
}

extern "C" void sbt_server_destroy(sbt_server *srv) {
    if (!srv) return;
    {
        std::unique_lock<std::mutex> lock(srv->mu);
        srv->stop = true;
        // batches not yet started end with SBT_E_STATE
        for (auto &kv : srv->streams) {
            for (Request *q : kv.second.queue) {
                q->t_start = Clock::now();
                srv->finish_locked(q, SBT_E_STATE);
            }
            srv->queued -= (int64_t)kv.second.queue.size();
            kv.second.queue.clear();
        }
        srv->ready.clear();
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    for (auto &t : srv->workers) t.join();  // in-flight batches finish first
    {
        // every ticket is done now; threads woken inside sbt_server_wait
        // leave before the requests and the server are freed
        std::unique_lock<std::mutex> lock(srv->mu);
        srv->cv_done.notify_all();
        srv->cv_done.wait(lock, [&] { return srv->waiters == 0; });
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    for (auto &kv : srv->streams) sbt_destroy(kv.second.ctx);
    if (srv->bst) cudaStreamSynchronize(srv->bst);
    for (cudaEvent_t ev : srv->bev) cudaEventDestroy(ev);
    if (srv->bst) cudaStreamDestroy(srv->bst);
    if (srv->bdesc) cudaFree(srv->bdesc);
    if (srv->bsync) cudaFree(srv->bsync);
    if (srv->h_berr) cudaFreeHost(srv->h_berr);
    cudaSetDevice(prev);
    for (auto &kv : srv->requests) delete kv.second;
    delete srv;
}
