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
#include <algorithm>
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
// defined in search.cu: one launch over the queries of several requests
hnsw_status search_group(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n, int max_k,
                         int max_ef, const uint32_t* q_kef, const uint64_t* q_out, uint32_t* ids, float* dists,
                         cudaStream_t s);

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
    uint64_t bytes = 0;   // device bytes of this request alone (admission check)
    uint64_t q0 = 0, o0 = 0;  // first query / output slot inside its group
    Clock::time_point submitted, finished;
    hnsw_status status = HNSW_OK;
    std::string error;
    bool complete = false;  // results in the caller's buffers
};

struct Slot {
    cudaStream_t stream = nullptr;
    void* pinned = nullptr;
    uint64_t pinned_bytes = 0;
    std::vector<Request*> group;           // requests of the launch on this slot
    uint64_t off = 0, bytes = 0;           // their arena range
    std::atomic<bool> device_done{false};  // set by the stream callback
    bool releasing = false;                // results being copied out
};

}  // namespace
}  // namespace hnswgb

using namespace hnswgb;

struct hnsw_server {
    int device = 0;
    std::vector<hnsw_index*> indexes;
    std::vector<std::unique_ptr<Slot>> slots;
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

// Runs on the CUDA runtime's callback thread after a group's copies: it
// takes no lock (the dispatcher may hold the server mutex across CUDA calls),
// only publishes the flag and wakes the dispatcher, which also re-checks on a
// short timeout in case this notification falls between its check and wait.
void CUDART_CB on_device_done(void* p) {
    auto* pair = static_cast<std::pair<hnsw_server*, Slot*>*>(p);
    pair->second->device_done.store(true, std::memory_order_release);
    pair->first->cv.notify_all();
    delete pair;
}

// A group: requests admitted together into one launch (same index, same
// options, same ef bucket).  Device and pinned layouts are identical:
// [queries][ids][dists][k|ef per query][output offset per query], each
// section 256-byte aligned.
struct GroupLayout {
    uint64_t nq = 0, nout = 0, q = 0, ids = 0, dists = 0, kef = 0, out = 0, total = 0;
};

GroupLayout layout_of(const std::vector<Request*>& g) {
    GroupLayout L;
    uint32_t d = g.front()->d;
    for (Request* r : g) {
        L.nq += uint64_t(r->r.n);
        L.nout += uint64_t(r->r.n) * uint64_t(r->r.k);
    }
    L.q = 0;
    L.ids = up256(L.nq * d * 4);
    L.dists = L.ids + up256(L.nout * 4);
    L.kef = L.dists + up256(L.nout * 4);
    L.out = L.kef + up256(L.nq * 4);
    L.total = L.out + up256(L.nq * 8);
    return L;
}

bool compatible(const Request* a, const Request* b) {
    auto bucket = [](const hnsw_request& r) {
        int e = r.ef > r.k ? r.ef : r.k, b = 32;
        while (b < e) b <<= 1;
        return b;
    };
    return a->r.index == b->r.index && a->r.rerank == b->r.rerank && a->r.stop_threshold == b->r.stop_threshold &&
           a->r.stop_period == b->r.stop_period && bucket(a->r) == bucket(b->r);
}

// Issues one admitted group on its slot's stream.  Called WITHOUT the server
// mutex: it touches only its slot (reserved by the caller), the group's arena
// range and the group's requests, none of which another thread uses until the
// slot's device_done flag is set.
void dispatch(hnsw_server* sv, hnsw_index* ix, Slot& sl) {
    std::vector<Request*>& g = sl.group;
    const GroupLayout L = layout_of(g);
    const uint32_t d = g.front()->d;
    char* db = static_cast<char*>(sv->arena_base) + sl.off;
    cudaError_t e = cudaSuccess;
    if (sl.pinned_bytes < L.total) {
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.pinned_bytes = 0;
        e = cudaMallocHost(&sl.pinned, L.total);
        if (e == cudaSuccess) sl.pinned_bytes = L.total;
    }
    hnsw_status st = HNSW_OK;
    if (e != cudaSuccess) {
        st = fail(HNSW_ENOMEM, "server: pinned staging");
    } else {
        char* hp = static_cast<char*>(sl.pinned);
        uint32_t* kef = reinterpret_cast<uint32_t*>(hp + L.kef);
        uint64_t* oo = reinterpret_cast<uint64_t*>(hp + L.out);
        uint64_t qi = 0, ob = 0;
        int max_k = 1, max_ef = 1;
        for (Request* r : g) {
            std::memcpy(hp + L.q + qi * d * 4, r->r.queries, uint64_t(r->r.n) * d * 4);
            r->q0 = qi;
            r->o0 = ob;
            for (int64_t j = 0; j < r->r.n; ++j) {
                kef[qi + j] = uint32_t(r->r.k) | (uint32_t(r->r.ef) << 16);
                oo[qi + j] = ob + uint64_t(j) * uint64_t(r->r.k);
            }
            qi += uint64_t(r->r.n);
            ob += uint64_t(r->r.n) * uint64_t(r->r.k);
            max_k = r->r.k > max_k ? r->r.k : max_k;
            max_ef = r->r.ef > max_ef ? r->r.ef : max_ef;
        }
        e = cudaMemcpyAsync(db + L.q, hp + L.q, L.ids - L.q, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(db + L.kef, hp + L.kef, L.total - L.kef, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) {
            const hnsw_request& r0 = g.front()->r;
            hnsw_search_params p{};
            p.k = max_k;
            p.ef = max_ef;
            p.rerank = r0.rerank;
            p.stop_threshold = r0.stop_threshold;
            p.stop_period = r0.stop_period;
            st = search_group(ix, p, reinterpret_cast<const float*>(db + L.q), uint32_t(L.nq),
                              max_k, max_ef, reinterpret_cast<const uint32_t*>(db + L.kef),
                              reinterpret_cast<const uint64_t*>(db + L.out), reinterpret_cast<uint32_t*>(db + L.ids),
                              reinterpret_cast<float*>(db + L.dists), sl.stream);
        } else {
            st = fail(HNSW_ECUDA, std::string("server: H2D: ") + cudaGetErrorString(e));
        }
        if (st == HNSW_OK) {
            e = cudaMemcpyAsync(hp + L.ids, db + L.ids, L.kef - L.ids, cudaMemcpyDeviceToHost, sl.stream);
            if (e == cudaSuccess) e = cudaLaunchHostFunc(sl.stream, on_device_done, new std::pair<hnsw_server*, Slot*>(sv, &sl));
            if (e != cudaSuccess) st = fail(HNSW_ECUDA, std::string("server: ") + cudaGetErrorString(e));
        }
    }
    if (st != HNSW_OK) {  // nothing more runs for this group on the device
        const std::string err = hnsw_last_error();
        for (Request* r : g) {
            r->status = st;
            r->error = err;
        }
        cudaStreamSynchronize(sl.stream);
        sl.device_done.store(true, std::memory_order_release);
    }
}

// Copies a finished group's results into the callers' buffers (no mutex:
// the slot and its requests belong to the dispatcher until released).
void copy_out(Slot& sl) {
    const GroupLayout L = layout_of(sl.group);
    const char* hp = static_cast<const char*>(sl.pinned);
    for (Request* r : sl.group)
        if (r->status == HNSW_OK) {
            const uint64_t ob = uint64_t(r->r.n) * uint64_t(r->r.k) * 4;
            std::memcpy(r->r.out_ids, hp + L.ids + r->o0 * 4, ob);
            std::memcpy(r->r.out_dists, hp + L.dists + r->o0 * 4, ob);
        }
}

// Marks the group complete and releases the slot and arena range (mu held).
void release(hnsw_server* sv, Slot& sl) {
    const auto now = Clock::now();
    for (Request* r : sl.group) {
        if (r->status == HNSW_OK)
            sv->stats.completed++;
        else
            sv->stats.failed++;
        r->finished = now;
        r->complete = true;
        sv->stats.in_flight--;
    }
    sv->arena->release(sl.off, sl.bytes);
    sl.group.clear();
    sl.device_done.store(false, std::memory_order_relaxed);
}

constexpr uint64_t kMaxGroupQueries = 8192;
constexpr int kGroupWindow = 512;

void worker_loop(hnsw_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        std::vector<Slot*> done;
        for (auto& slp : sv->slots)
            if (!slp->group.empty() && !slp->releasing && slp->device_done.load(std::memory_order_acquire)) {
                slp->releasing = true;
                done.push_back(slp.get());
            }
        if (!done.empty()) {
            lk.unlock();
            for (Slot* sl : done) copy_out(*sl);
            lk.lock();
            for (Slot* sl : done) {
                release(sv, *sl);
                sl->releasing = false;
            }
            sv->done_cv.notify_all();
        }
        // admit groups from the head of the queue while a slot and arena space are free
        while (!sv->pending.empty()) {
            int si = -1;
            for (size_t i = 0; i < sv->slots.size(); ++i)
                if (sv->slots[i]->group.empty()) {
                    si = int(i);
                    break;
                }
            if (si < 0) break;
            // the head, plus compatible requests further back (up to a window)
            std::vector<Request*> g{sv->pending.front()};
            uint64_t nq = uint64_t(g[0]->r.n);
            int scanned = 0;
            for (auto it = std::next(sv->pending.begin()); it != sv->pending.end() && scanned < kGroupWindow;
                 ++it, ++scanned)
                if (compatible(*it, g[0]) && nq + uint64_t((*it)->r.n) <= kMaxGroupQueries) {
                    g.push_back(*it);
                    nq += uint64_t((*it)->r.n);
                }
            uint64_t off = 0;
            bool fits = false;
            for (;;) {
                if (sv->arena->alloc(layout_of(g).total, off)) {
                    fits = true;
                    break;
                }
                if (g.size() == 1) break;
                g.pop_back();  // a smaller group
            }
            if (!fits) break;  // the head does not fit now: wait for completions
            for (Request* r : g) sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
            sv->stats.queued -= g.size();
            sv->stats.in_flight += g.size();
            Slot& sl = *sv->slots[si];
            sl.group = g;  // reserves the slot
            sl.off = off;
            sl.bytes = layout_of(g).total;
            hnsw_index* ix = sv->indexes[g.front()->r.index];
            lk.unlock();
            dispatch(sv, ix, sl);
            lk.lock();
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
    for (int i = 0; i < p->n_slots; ++i) sv->slots.emplace_back(new Slot());
    for (auto& sl : sv->slots)
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto& s2 : sv->slots)
                if (s2->stream) cudaStreamDestroy(s2->stream);
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
    rq->bytes = up256(qb) + 2 * up256(ob) + up256(uint64_t(r->n) * 4) + up256(uint64_t(r->n) * 8);
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

extern "C" hnsw_status hnsw_server_cancel(hnsw_server* sv, uint64_t ticket) {
    if (!sv) return fail(HNSW_EINVAL, "hnsw_server_cancel: null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(HNSW_EINVAL, "hnsw_server_cancel: unknown ticket");
    Request* rq = it->second.get();
    auto pit = std::find(sv->pending.begin(), sv->pending.end(), rq);
    if (rq->complete || pit == sv->pending.end())
        return fail(HNSW_EBUSY, "hnsw_server_cancel: the request is already admitted or complete");
    sv->pending.erase(pit);
    sv->stats.queued--;
    sv->stats.cancelled++;
    rq->status = HNSW_ECANCELED;
    rq->error = "cancelled before admission";
    rq->finished = Clock::now();
    rq->complete = true;
    sv->done_cv.notify_all();
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
        if (sl->stream) {
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
        if (sl->pinned) cudaFreeHost(sl->pinned);
    }
    cudaFree(sv->arena_base);
    delete sv;
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_server_replay(hnsw_server* sv, const hnsw_request* reqs, const double* arrival_s,
                                          int64_t n, int32_t timeout_ms, double* latency_ms, double* submit_s) {
    if (!sv || (n > 0 && (!reqs || !arrival_s || !latency_ms))) return fail(HNSW_EINVAL, "hnsw_server_replay: null argument");
    std::vector<uint64_t> tickets(size_t(n > 0 ? n : 0));
    const auto t0 = Clock::now();
    for (int64_t i = 0; i < n; ++i) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        if (submit_s) submit_s[i] = std::chrono::duration<double>(Clock::now() - t0).count();
        const hnsw_status st = hnsw_server_submit(sv, &reqs[i], &tickets[size_t(i)]);
        if (st != HNSW_OK) {
            for (int64_t j = 0; j < i; ++j) hnsw_server_wait(sv, tickets[size_t(j)], -1, nullptr);
            return st;
        }
    }
    hnsw_status first = HNSW_OK;
    for (int64_t i = 0; i < n; ++i) {
        const hnsw_status st = hnsw_server_wait(sv, tickets[size_t(i)], timeout_ms, &latency_ms[i]);
        if (st != HNSW_OK && first == HNSW_OK) first = st;
    }
    return first;
}
