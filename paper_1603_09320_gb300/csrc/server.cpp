// server.cpp -- continuous-batching request loop over resident indexes
// (hnsw_server_*).  The paper has no serving component; this is the request
// path around the batched search of Alg. 5.
//
// Requests (index, n queries, k, ef, options; caller-owned host buffers) go
// into a FIFO.  A dispatcher thread admits the request at the head as soon
// as (a) one of the server's slots is free -- a slot is a CUDA stream with
// pinned host staging -- and (b) the request's device buffers fit in the
// device arena, whose budget is fixed from the free device memory at
// creation.  An admitted request copies its queries in, runs hnsw_search_ex
// on its slot's stream and copies the results back; requests admitted while
// others are still on the GPU run concurrently with them.  A host function
// enqueued after the copies marks the request complete; the dispatcher then
// copies the results into the caller's buffers and returns the slot and the
// arena range.  Every wait of the host on the device is bounded by the
// caller's timeout (hnsw_server_wait), and destroy waits for requests in
// flight.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.hpp"

namespace hnswgb {
namespace {

using Clock = std::chrono::steady_clock;

uint64_t up256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// First-fit allocator over the byte range [0, cap) of the device arena.
class Arena {
   public:
    explicit Arena(uint64_t cap) : cap_(cap) {
        if (cap) free_[0] = cap;
    }
    bool alloc(uint64_t sz, uint64_t& off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < sz) continue;
            off = it->first;
            const uint64_t rest = it->second - sz;
            free_.erase(it);
            if (rest) free_[off + sz] = rest;
            used_ += sz;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t sz) {
        used_ -= sz;
        auto it = free_.emplace(off, sz).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {  // merge right
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {  // merge left
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }
    uint64_t cap() const { return cap_; }

   private:
    uint64_t cap_, used_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

struct Request {
    uint64_t ticket = 0;
    hnsw_request r{};
    uint32_t d = 0;
    uint64_t bytes = 0, off = 0;
    int slot = -1;
    Clock::time_point submitted, finished;
    hnsw_status status = HNSW_OK;
    std::string error;
    std::atomic<bool> device_done{false};  // set by the stream callback
    bool complete = false;     // results in the caller's buffers
};

struct Slot {
    cudaStream_t stream = nullptr;
    void* pinned = nullptr;
    uint64_t pinned_bytes = 0;
    Request* req = nullptr;
};

}  // namespace
}  // namespace hnswgb

using namespace hnswgb;

struct hnsw_server {
    int device = 0;
    std::vector<hnsw_index*> indexes;
    std::vector<Slot> slots;
    void* arena_base = nullptr;
    std::unique_ptr<Arena> arena;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::mutex mu;
    std::condition_variable cv;       // wakes the dispatcher
    std::condition_variable done_cv;  // wakes waiters
    std::thread worker;
    bool stopping = false;
    uint64_t next_ticket = 1;
    hnsw_server_stats stats{};
};

namespace {

// Runs on the CUDA runtime's callback thread after a request's copies: it
// takes no lock (the dispatcher may hold the server mutex across CUDA calls),
// only publishes the flag and wakes the dispatcher, which also re-checks on a
// short timeout in case this notification falls between its check and wait.
void CUDART_CB on_device_done(void* p) {
    auto* pair = static_cast<std::pair<hnsw_server*, Request*>*>(p);
    pair->second->device_done.store(true, std::memory_order_release);
    pair->first->cv.notify_all();
    delete pair;
}

// Issues one admitted request on its slot's stream (called with mu held).
void dispatch(hnsw_server* sv, Request* rq, int si) {
    Slot& sl = sv->slots[si];
    const hnsw_request& r = rq->r;
    const uint64_t qb = uint64_t(r.n) * rq->d * 4, ob = uint64_t(r.n) * uint64_t(r.k) * 4;
    char* dbase = static_cast<char*>(sv->arena_base) + rq->off;
    float* dq = reinterpret_cast<float*>(dbase);
    uint32_t* di = reinterpret_cast<uint32_t*>(dbase + up256(qb));
    float* dd = reinterpret_cast<float*>(dbase + up256(qb) + up256(ob));
    const uint64_t need_pinned = up256(qb) + 2 * up256(ob);
    rq->slot = si;
    sl.req = rq;
    cudaError_t e = cudaSuccess;
    if (sl.pinned_bytes < need_pinned) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.pinned_bytes = 0;
        e = cudaMallocHost(&sl.pinned, need_pinned);
        if (e == cudaSuccess) sl.pinned_bytes = need_pinned;
    }
    hnsw_status st = HNSW_OK;
    if (e != cudaSuccess) {
        st = fail(HNSW_ENOMEM, "server: pinned staging");
    } else {
        char* hp = static_cast<char*>(sl.pinned);
        std::memcpy(hp, r.queries, qb);
        e = cudaMemcpyAsync(dq, hp, qb, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) {
            hnsw_search_params p{};
            p.k = r.k;
            p.ef = r.ef;
            p.rerank = r.rerank;
            p.stop_threshold = r.stop_threshold;
            p.stop_period = r.stop_period;
            st = hnsw_search_ex(sv->indexes[r.index], &p, dq, r.n, di, dd, nullptr, sl.stream);
        } else {
            st = fail(HNSW_ECUDA, std::string("server: H2D: ") + cudaGetErrorString(e));
        }
        if (st == HNSW_OK) {
            e = cudaMemcpyAsync(hp + up256(qb), di, ob, cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hp + up256(qb) + up256(ob), dd, ob, cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess)
                e = cudaLaunchHostFunc(sl.stream, on_device_done, new std::pair<hnsw_server*, Request*>(sv, rq));
            if (e != cudaSuccess) st = fail(HNSW_ECUDA, std::string("server: ") + cudaGetErrorString(e));
        }
    }
    if (st != HNSW_OK) {  // nothing more runs for this request on the device
        rq->status = st;
        rq->error = hnsw_last_error();
        cudaStreamSynchronize(sl.stream);
        rq->device_done.store(true, std::memory_order_release);
    }
}

// Copies results out and releases the slot and arena range (mu held).
void complete(hnsw_server* sv, Request* rq) {
    Slot& sl = sv->slots[rq->slot];
    const hnsw_request& r = rq->r;
    if (rq->status == HNSW_OK) {
        const uint64_t qb = uint64_t(r.n) * rq->d * 4, ob = uint64_t(r.n) * uint64_t(r.k) * 4;
        const char* hp = static_cast<const char*>(sl.pinned);
        std::memcpy(r.out_ids, hp + up256(qb), ob);
        std::memcpy(r.out_dists, hp + up256(qb) + up256(ob), ob);
        sv->stats.completed++;
    } else {
        sv->stats.failed++;
    }
    sv->arena->release(rq->off, rq->bytes);
    sl.req = nullptr;
    rq->finished = Clock::now();
    rq->complete = true;
    sv->stats.in_flight--;
}

void worker_loop(hnsw_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progress = false;
        for (auto& sl : sv->slots)
            if (sl.req && sl.req->device_done.load(std::memory_order_acquire)) {
                complete(sv, sl.req);
                progress = true;
            }
        if (progress) sv->done_cv.notify_all();
        // admit from the head of the queue while a slot and arena space are free
        while (!sv->pending.empty()) {
            int si = -1;
            for (size_t i = 0; i < sv->slots.size(); ++i)
                if (!sv->slots[i].req) {
                    si = int(i);
                    break;
                }
            if (si < 0) break;
            Request* rq = sv->pending.front();
            uint64_t off = 0;
            if (!sv->arena->alloc(rq->bytes, off)) break;  // wait for memory to free up
            rq->off = off;
            sv->pending.pop_front();
            sv->stats.queued--;
            sv->stats.in_flight++;
            dispatch(sv, rq, si);
        }
        sv->stats.bytes_in_use = sv->arena->used();
        if (sv->stopping && sv->pending.empty() && sv->stats.in_flight == 0) break;
        if (sv->stats.in_flight > 0)
            sv->cv.wait_for(lk, std::chrono::microseconds(200));
        else
            sv->cv.wait(lk);
    }
}

}  // namespace

extern "C" hnsw_status hnsw_server_create(const hnsw_server_params* p, hnsw_server** out) {
    if (!p || !out || p->n_slots < 1 || p->n_slots > 64) return fail(HNSW_EINVAL, "hnsw_server_create: 1..64 slots");
    *out = nullptr;
    std::unique_ptr<hnsw_server> sv(new hnsw_server());
    cudaGetDevice(&sv->device);
    uint64_t budget = p->memory_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_server_create: ") + cudaGetErrorString(e));
        budget = fr / 4;
        if (budget > (uint64_t(4) << 30)) budget = uint64_t(4) << 30;
    }
    budget = up256(budget);
    if (cudaMalloc(&sv->arena_base, budget) != cudaSuccess) {
        cudaGetLastError();
        return fail(HNSW_ENOMEM, "hnsw_server_create: device arena");
    }
    sv->arena.reset(new Arena(budget));
    sv->stats.budget = budget;
    sv->slots.resize(size_t(p->n_slots));
    for (auto& sl : sv->slots)
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto& s2 : sv->slots)
                if (s2.stream) cudaStreamDestroy(s2.stream);
            cudaFree(sv->arena_base);
            return fail(HNSW_ECUDA, "hnsw_server_create: stream");
        }
    hnsw_server* raw = sv.get();
    sv->worker = std::thread(worker_loop, raw);
    *out = sv.release();
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_add_index(hnsw_server* sv, hnsw_index* ix, int32_t* id) {
    if (!sv || !ix || !id) return fail(HNSW_EINVAL, "hnsw_server_add_index: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->indexes.push_back(ix);
    *id = int32_t(sv->indexes.size() - 1);
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_submit(hnsw_server* sv, const hnsw_request* r, uint64_t* ticket) {
    if (!sv || !r || !ticket) return fail(HNSW_EINVAL, "hnsw_server_submit: null argument");
    std::unique_ptr<Request> rq(new Request());
    rq->r = *r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r->index < 0 || size_t(r->index) >= sv->indexes.size())
            return fail(HNSW_EINVAL, "hnsw_server_submit: unknown index");
        hnsw_index_info info{};
        hnsw_get_index_info(sv->indexes[r->index], &info);
        rq->d = info.d;
    }
    if (r->n < 1 || r->k < 1 || r->ef < 1 || !r->queries || !r->out_ids || !r->out_dists)
        return fail(HNSW_EINVAL, "hnsw_server_submit: bad request");
    const uint64_t qb = uint64_t(r->n) * rq->d * 4, ob = uint64_t(r->n) * uint64_t(r->k) * 4;
    rq->bytes = up256(qb) + 2 * up256(ob);
    if (rq->bytes > sv->arena->cap())
        return fail(HNSW_EINVAL, "hnsw_server_submit: request larger than the memory budget");
    rq->submitted = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return fail(HNSW_EBUSY, "hnsw_server_submit: server is stopping");
    rq->ticket = sv->next_ticket++;
    *ticket = rq->ticket;
    sv->pending.push_back(rq.get());
    sv->stats.submitted++;
    sv->stats.queued++;
    sv->reqs.emplace(rq->ticket, std::move(rq));
    sv->cv.notify_all();
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_poll(hnsw_server* sv, uint64_t ticket, int32_t* done) {
    if (!sv || !done) return fail(HNSW_EINVAL, "hnsw_server_poll: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(HNSW_EINVAL, "hnsw_server_poll: unknown ticket");
    *done = it->second->complete ? 1 : 0;
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_wait(hnsw_server* sv, uint64_t ticket, int32_t timeout_ms, double* latency_ms) {
    if (!sv) return fail(HNSW_EINVAL, "hnsw_server_wait: null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(HNSW_EINVAL, "hnsw_server_wait: unknown ticket");
    Request* rq = it->second.get();
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!rq->complete) {
        if (timeout_ms < 0) {
            sv->done_cv.wait(lk);
        } else if (sv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !rq->complete) {
            return fail(HNSW_ETIMEOUT, "hnsw_server_wait: request not complete within the timeout");
        }
    }
    if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(rq->finished - rq->submitted).count();
    const hnsw_status st = rq->status;
    const std::string err = rq->error;
    sv->reqs.erase(it);  // the ticket is consumed
    if (st != HNSW_OK) return fail(st, "hnsw_server_wait: " + err);
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_get_stats(hnsw_server* sv, hnsw_server_stats* out) {
    if (!sv || !out) return fail(HNSW_EINVAL, "hnsw_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->bytes_in_use = sv->arena->used();
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_destroy(hnsw_server* sv) {
    if (!sv) return HNSW_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& sl : sv->slots) {
        if (sl.stream) {
            cudaStreamSynchronize(sl.stream);
            cudaStreamDestroy(sl.stream);
        }
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    cudaFree(sv->arena_base);
    delete sv;
    return HNSW_OK;
}
