// builder.cpp -- multi-threaded host construction of the HNSW graph
// (arXiv:1603.09320, Alg. 1 INSERT with Alg. 3 / Alg. 4 neighbour selection).
//
// Section 4.1 notes that construction parallelises with few synchronisation
// points.  Here every element has a spin lock guarding its neighbour lists,
// and one mutex guards the enter point: an element whose level exceeds the
// current top level holds it for its whole insertion, so the enter point and
// the top level change together (Alg. 1's enter-point update).  Worker threads take
// element ids in increasing order from an atomic counter; with one thread the
// build is Alg. 1 applied to elements 0..N-1 in order.
//
// Comparisons use the key (distance, id).  Alg. 4's acceptance test is read
// strictly: e joins R only if dist(e, base) < dist(e, r) for every r in R.
// Distances are fp32 (squared L2, or 1 - <a,b> for cosine).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.hpp"

namespace hnswgb {
namespace {

typedef float v4f __attribute__((vector_size(16)));

inline v4f ld4(const float* p) {
    v4f v;
    std::memcpy(&v, p, 16);
    return v;
}

float dist_l2(const float* a, const float* b, uint32_t d) {
    v4f s0 = {0, 0, 0, 0}, s1 = {0, 0, 0, 0};
    uint32_t i = 0;
    for (; i + 8 <= d; i += 8) {
        v4f t0 = ld4(a + i) - ld4(b + i);
        v4f t1 = ld4(a + i + 4) - ld4(b + i + 4);
        s0 += t0 * t0;
        s1 += t1 * t1;
    }
    v4f s = s0 + s1;
    float r = (s[0] + s[1]) + (s[2] + s[3]);
    for (; i < d; ++i) {
        float t = a[i] - b[i];
        r += t * t;
    }
    return r;
}

float dist_cos(const float* a, const float* b, uint32_t d) {
    v4f s0 = {0, 0, 0, 0}, s1 = {0, 0, 0, 0};
    uint32_t i = 0;
    for (; i + 8 <= d; i += 8) {
        s0 += ld4(a + i) * ld4(b + i);
        s1 += ld4(a + i + 4) * ld4(b + i + 4);
    }
    v4f s = s0 + s1;
    float r = (s[0] + s[1]) + (s[2] + s[3]);
    for (; i < d; ++i) r += a[i] * b[i];
    return 1.0f - r;
}

struct Item {
    float d;
    uint32_t id;
};
inline bool key_less(const Item& a, const Item& b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }
struct MinTop {  // std heap comparator: nearest on top
    bool operator()(const Item& a, const Item& b) const { return key_less(b, a); }
};
struct MaxTop {  // furthest on top
    bool operator()(const Item& a, const Item& b) const { return key_less(a, b); }
};

class SpinLock {
   public:
    void lock() {
        while (f_.exchange(1, std::memory_order_acquire)) {
            while (f_.load(std::memory_order_relaxed)) std::this_thread::yield();
        }
    }
    void unlock() { f_.store(0, std::memory_order_release); }

   private:
    std::atomic<uint8_t> f_{0};
};

struct Graph {
    const float* data = nullptr;
    uint64_t N = 0;
    uint32_t d = 0;
    int metric = 0;
    hnsw_build_params p{};
    std::vector<uint8_t> level;
    std::vector<uint32_t> links0;  // N rows of [count, Mmax0 ids]
    std::vector<uint64_t> upoff;   // word offset of an element's layer-1 row in linksU
    std::vector<uint32_t> linksU;  // rows of [count, Mmax ids]
    std::unique_ptr<SpinLock[]> locks;
    std::mutex top;
    uint32_t ep = kNoId;
    int maxlevel = -1;

    const float* row(uint32_t i) const { return data + uint64_t(i) * d; }
    float dist(const float* a, const float* b) const {
        return metric == 0 ? dist_l2(a, b, d) : dist_cos(a, b, d);
    }
    uint32_t cap(int lc) const { return lc == 0 ? p.Mmax0 : p.Mmax; }
    uint32_t* list(uint32_t i, int lc) {
        return lc == 0 ? &links0[uint64_t(i) * (p.Mmax0 + 1)]
                       : &linksU[upoff[i] + uint64_t(lc - 1) * (p.Mmax + 1)];
    }
};

// Per-thread scratch: epoch-tagged visited marks and heap storage.
struct Ctx {
    std::vector<uint32_t> mark;
    uint32_t epoch = 0;
    std::vector<Item> C, W, tmp, cand, R, Wd;
    std::vector<uint32_t> nb;
    explicit Ctx(uint64_t N) : mark(N, 0) {}
    void new_epoch() {
        if (++epoch == 0) {
            std::fill(mark.begin(), mark.end(), 0);
            epoch = 1;
        }
    }
};

// Copies neighbourhood(i) at layer lc under i's lock.
void read_list(Graph& g, uint32_t i, int lc, std::vector<uint32_t>& out) {
    g.locks[i].lock();
    const uint32_t* l = g.list(i, lc);
    out.assign(l + 1, l + 1 + l[0]);
    g.locks[i].unlock();
}

// Alg. 2 SEARCH-LAYER(q, ep, ef, lc); W returned in cx.W sorted by key.
void search_layer(Graph& g, Ctx& cx, const float* q, const std::vector<Item>& ep, uint32_t ef, int lc) {
    cx.new_epoch();
    auto& C = cx.C;
    auto& W = cx.W;
    C.clear();
    W.clear();
    for (const Item& e : ep) {  // start: v, C and W hold the enter points
        if (cx.mark[e.id] == cx.epoch) continue;
        cx.mark[e.id] = cx.epoch;
        C.push_back(e);
        std::push_heap(C.begin(), C.end(), MinTop());
        W.push_back(e);
        std::push_heap(W.begin(), W.end(), MaxTop());
    }
    while (!C.empty()) {  // while C is not empty
        std::pop_heap(C.begin(), C.end(), MinTop());
        Item c = C.back();  // the nearest of C
        C.pop_back();
        if (key_less(W.front(), c)) break;  // stop: c is further than the furthest of W
        read_list(g, c.id, lc, cx.nb);
        for (uint32_t e : cx.nb) {  // each neighbour of c
            if (cx.mark[e] == cx.epoch) continue;  // visited
            cx.mark[e] = cx.epoch;                  // mark visited
            Item ei{g.dist(q, g.row(e)), e};
            if (key_less(ei, W.front()) || W.size() < ef) {  // admit: closer than the furthest, or W not full
                C.push_back(ei);
                std::push_heap(C.begin(), C.end(), MinTop());
                W.push_back(ei);
                std::push_heap(W.begin(), W.end(), MaxTop());
                if (W.size() > ef) {  // drop the furthest
                    std::pop_heap(W.begin(), W.end(), MaxTop());
                    W.pop_back();
                }
            }
        }
    }
    std::sort(W.begin(), W.end(), key_less);
}

// Steepest descent on layer lc (Alg. 2 with ef = 1 under key order).
Item greedy(Graph& g, Ctx& cx, const float* q, Item cur, int lc) {
    for (;;) {
        Item b = cur;
        read_list(g, cur.id, lc, cx.nb);
        for (uint32_t e : cx.nb) {
            Item ei{g.dist(q, g.row(e)), e};
            if (key_less(ei, b)) b = ei;
        }
        if (b.id == cur.id) return cur;
        cur = b;
    }
}

// Alg. 3 / Alg. 4 over candidates `C` (distances to `base`), result in R.
void select_neighbors(Graph& g, Ctx& cx, const float* base, uint32_t base_id, std::vector<Item>& C,
                      uint32_t M, int lc, std::vector<Item>& R) {
    R.clear();
    std::sort(C.begin(), C.end(), key_less);
    if (!g.p.heuristic) {  // Alg. 3
        for (size_t i = 0; i < C.size() && R.size() < M; ++i) R.push_back(C[i]);
        return;
    }
    auto& Wq = cx.tmp;  // working queue, kept sorted
    Wq.assign(C.begin(), C.end());
    if (g.p.extend_candidates) {  // extendCandidates
        cx.new_epoch();
        for (const Item& e : C) cx.mark[e.id] = cx.epoch;
        std::vector<uint32_t> adj;
        for (const Item& e : C) {
            read_list(g, e.id, lc, adj);
            for (uint32_t a : adj) {
                if (cx.mark[a] == cx.epoch || a == base_id) continue;
                cx.mark[a] = cx.epoch;
                Wq.push_back(Item{g.dist(base, g.row(a)), a});
            }
        }
        std::sort(Wq.begin(), Wq.end(), key_less);
    }
    auto& Wd = cx.Wd;
    Wd.clear();
    for (size_t i = 0; i < Wq.size() && R.size() < M; ++i) {  // accept when closer to the base than to every element of R
        const Item& e = Wq[i];
        bool good = true;
        for (const Item& r : R)
            if (!(e.d < g.dist(g.row(e.id), g.row(r.id)))) {
                good = false;
                break;
            }
        if (good)
            R.push_back(e);
        else
            Wd.push_back(e);  // discarded, in key order
    }
    if (g.p.keep_pruned)  // refill R from the discarded, nearest first
        for (size_t i = 0; i < Wd.size() && R.size() < M; ++i) R.push_back(Wd[i]);
}

// Alg. 1's reverse link and shrink for one neighbour e: add q to neighbourhood(e) at lc and
// shrink it with the selection rule when it exceeds the cap.
void link_back(Graph& g, Ctx& cx, uint32_t e, uint32_t q, int lc) {
    const uint32_t cap = g.cap(lc);
    for (;;) {
        g.locks[e].lock();
        uint32_t* l = g.list(e, lc);
        for (uint32_t j = 0; j < l[0]; ++j)
            if (l[1 + j] == q) {
                g.locks[e].unlock();
                return;
            }
        if (l[0] < cap) {
            l[1 + l[0]] = q;
            l[0]++;
            g.locks[e].unlock();
            return;
        }
        std::vector<uint32_t> before(l + 1, l + 1 + l[0]);
        // with extendCandidates the selection reads other lists: do it unlocked
        // and retry if neighbourhood(e) changed meanwhile
        const bool unlocked = g.p.extend_candidates != 0;
        if (unlocked) g.locks[e].unlock();
        cx.cand.clear();
        const float* ev = g.row(e);
        for (uint32_t x : before) cx.cand.push_back(Item{g.dist(ev, g.row(x)), x});
        cx.cand.push_back(Item{g.dist(ev, g.row(q)), q});
        select_neighbors(g, cx, ev, e, cx.cand, cap, lc, cx.R);
        if (unlocked) {
            g.locks[e].lock();
            l = g.list(e, lc);
            if (l[0] != before.size() || !std::equal(before.begin(), before.end(), l + 1)) {
                g.locks[e].unlock();
                continue;
            }
        }
        l[0] = uint32_t(cx.R.size());
        for (size_t j = 0; j < cx.R.size(); ++j) l[1 + j] = cx.R[j].id;
        g.locks[e].unlock();
        return;
    }
}

void insert(Graph& g, Ctx& cx, uint32_t q) {
    const int l = g.level[q];
    const float* qv = g.row(q);
    std::unique_lock<std::mutex> top(g.top);
    const int L = g.maxlevel;
    const uint32_t ep0 = g.ep;
    if (l <= L) top.unlock();  // only a new top element keeps the lock

    Item cur{g.dist(qv, g.row(ep0)), ep0};
    for (int lc = L; lc > l; --lc) cur = greedy(g, cx, qv, cur, lc);  // greedy descent above the element's level
    std::vector<Item> eps{cur};
    std::vector<Item> W;
    const int top_lc = std::min(L, l);
    std::vector<std::vector<Item>> sels(size_t(std::max(top_lc, -1) + 1));
    for (int lc = top_lc; lc >= 0; --lc) {  // the element's layers, top down
        search_layer(g, cx, qv, eps, g.p.ef_construction, lc);
        W = cx.W;
        cx.cand.assign(W.begin(), W.end());
        std::vector<Item>& sel = sels[size_t(lc)];
        select_neighbors(g, cx, qv, q, cx.cand, g.p.M, lc, sel);
        g.locks[q].lock();
        uint32_t* ql = g.list(q, lc);
        ql[0] = 0;
        for (const Item& s : sel)
            if (s.id != q) ql[1 + ql[0]++] = s.id;
        g.locks[q].unlock();
        eps.swap(W);  // ep <- W
    }
    // the reverse links once neighbourhood(q) is written on
    // every layer: q is unreachable until the first of them, so no concurrent
    // insertion can enter layer 0 at q while q's layer-0 list is still empty.
    // Sequentially this is the same graph: a search on layer lc - 1 reads no
    // list that the reverse links on layer lc change.
    for (int lc = top_lc; lc >= 0; --lc)
        for (const Item& s : sels[size_t(lc)])
            if (s.id != q) link_back(g, cx, s.id, q, lc);
    if (l > L) {  // a new top level moves the enter point
        g.ep = q;
        g.maxlevel = l;
    }
}

}  // namespace
}  // namespace hnswgb

using namespace hnswgb;

extern "C" hnsw_status hnsw_build(const float* data, uint64_t N, uint32_t d, hnsw_metric metric,
                                  const hnsw_build_params* params, const double* level_u,
                                  void** out_blob, uint64_t* out_bytes) {
    if (!params || !out_blob || !out_bytes || (N > 0 && (!data || !level_u)))
        return fail(HNSW_EINVAL, "hnsw_build: null pointer");
    const hnsw_build_params& p = *params;
    if (d == 0 || N >= (1ull << 31) || p.M == 0 || p.M > p.Mmax || p.M > p.Mmax0 || p.Mmax0 > 64 ||
        p.Mmax > 64 || !(p.mL > 0) || p.ef_construction == 0 || (metric != HNSW_L2SQ && metric != HNSW_COSINE))
        return fail(HNSW_EINVAL, "hnsw_build: invalid parameters");
    try {
        Graph g;
        g.data = data;
        g.N = N;
        g.d = d;
        g.metric = int(metric);
        g.p = p;
        g.level.resize(N);
        g.upoff.resize(N);
        uint64_t rows = 0;
        for (uint64_t i = 0; i < N; ++i) {
            const double u = level_u[i];
            if (!(u > 0.0 && u <= 1.0)) return fail(HNSW_EINVAL, "hnsw_build: level_u outside (0,1]");
            const double lv = std::floor(-std::log(u) * p.mL);  // the level draw of Alg. 1
            if (lv > 255) return fail(HNSW_EINVAL, "hnsw_build: level above 255");
            g.level[i] = uint8_t(lv);
            g.upoff[i] = rows * (p.Mmax + 1);
            rows += g.level[i];
        }
        g.links0.assign(N * (p.Mmax0 + 1), 0);
        g.linksU.assign(rows * (p.Mmax + 1), 0);
        g.locks.reset(new SpinLock[N > 0 ? N : 1]);
        if (N > 0) {
            g.ep = 0;  // the first element becomes the enter point with no links
            g.maxlevel = g.level[0];
        }
        int nt = p.n_threads > 0 ? p.n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
        std::atomic<uint64_t> next{1};
        auto work = [&]() {
            Ctx cx(N);
            for (;;) {
                uint64_t i = next.fetch_add(1);
                if (i >= N) break;
                insert(g, cx, uint32_t(i));
            }
        };
        if (nt == 1 || N < 2) {
            work();
        } else {
            // the first elements one at a time: while the graph is tiny,
            // concurrent insertions would start from an enter point whose
            // links are not written yet and keep only the one or two elements
            // they find
            const uint64_t n_seq = std::min<uint64_t>(N, 1024);
            {
                Ctx cx(N);
                for (uint64_t i = 1; i < n_seq; ++i) insert(g, cx, uint32_t(i));
            }
            next = n_seq;
            std::vector<std::thread> th;
            for (int t = 0; t < nt; ++t) th.emplace_back(work);
            for (auto& t : th) t.join();
        }
        // serialise
        BlobLayout lay = BlobLayout::of(N, d, p.Mmax0, p.Mmax, rows);
        uint8_t* b = static_cast<uint8_t*>(std::calloc(lay.total, 1));
        if (!b) return fail(HNSW_ENOMEM, "hnsw_build: blob allocation failed");
        std::memcpy(b + lay.data, data, N * d * 4ull);
        std::memcpy(b + lay.level, g.level.data(), N);
        for (uint64_t i = 0; i < N; ++i) {
            const uint32_t* l = g.list(uint32_t(i), 0);
            uint8_t* r = b + lay.nbr0 + i * p.Mmax0 * 4ull;
            for (uint32_t j = 0; j < p.Mmax0; ++j) wr<uint32_t>(r + 4ull * j, j < l[0] ? l[1 + j] : kNoId);
        }
        uint64_t rr = 0;
        for (uint64_t i = 0; i < N; ++i)
            for (int lc = 1; lc <= g.level[i]; ++lc, ++rr) {
                const uint32_t* l = g.list(uint32_t(i), lc);
                uint8_t* r = b + lay.nbrU + rr * p.Mmax * 4ull;
                for (uint32_t j = 0; j < p.Mmax; ++j) wr<uint32_t>(r + 4ull * j, j < l[0] ? l[1 + j] : kNoId);
            }
        BlobHeader h{};
        h.version = 1;
        h.metric = uint32_t(metric);
        h.N = N;
        h.d = d;
        h.M = p.M;
        h.Mmax = p.Mmax;
        h.Mmax0 = p.Mmax0;
        h.maxlevel = N ? uint32_t(g.maxlevel) : 0;
        h.ep = N ? g.ep : kNoId;
        h.flags = (p.heuristic ? 1u : 0u) | (p.extend_candidates ? 2u : 0u) | (p.keep_pruned ? 4u : 0u);
        h.efC = p.ef_construction;
        h.mL = p.mL;
        h.n_upper_rows = rows;
        h.checksum = fnv1a64(b + 128, lay.total - 128);
        write_header(b, h);
        *out_blob = b;
        *out_bytes = lay.total;
        return HNSW_OK;
    } catch (const std::bad_alloc&) {
        return fail(HNSW_ENOMEM, "hnsw_build: out of host memory");
    } catch (...) {
        return fail(HNSW_EINVAL, "hnsw_build: unexpected failure");
    }
}

extern "C" void hnsw_free_blob(void* blob) { std::free(blob); }
