// search.cu -- batched K-NN-SEARCH (arXiv:1603.09320, Alg. 5) on one GPU.
//
// One warp answers one query at a time; warps pull query indexes from a
// device work counter until the batch is exhausted (persistent kernel).
//
// Per query:
//   1. greedy ef=1 descent through layers L..1 (Alg. 5's descent).  Under key
//      order (distance, id), SEARCH-LAYER with ef=1 is steepest descent: move
//      to the best of the current element's neighbours while it beats the
//      current element.  No visited set is needed for that.
//   2. SEARCH-LAYER(q, ep, ef', 0) (Alg. 2, ef' = max(ef, K)) as ONE list W in
//      shared memory, sorted by key and capped at ef', with an "expanded" bit
//      per entry instead of the two priority queues: under key order the
//      unextracted candidates that can still be expanded before Alg. 2's
//      stop test fires are exactly the unexpanded entries of W, so "extract
//      the nearest of C" is "take the first unexpanded entry" and the loop
//      ends when none is left.  All unvisited neighbours of the expanded
//      element are scored together and merged at once; inserting them one at
//      a time by Alg. 2's admission and eviction leaves the same top-ef' of
//      the union.
//   3. the K first entries of W (Alg. 5's result), or, with rerank, the K best
//      of W by exact fp32 distance recomputed from the fp32 copy.
//
// Visited set: a 4-way bucketed hash of element ids in shared memory; when a
// bucket is full one of its slots is overwritten, and two lanes storing into
// the same free slot at the same instant keep only one id, so the set may
// FORGET an element.  Forgetting never changes
// the result: an element met again is either already in W (its key equals an
// entry's key and the merge drops it) or, being outside W after it was
// visited, has a key above the furthest entry of a full W and is rejected.
// It only costs a repeated distance evaluation, counted in n_eval.
//
// Distances: each row is read as 16-byte chunks by a team of TEAM lanes
// (consecutive lanes read consecutive chunks, so a team's load of one row is
// one contiguous segment), U rows per team in flight, partial sums reduced by
// warp shuffles inside the team.  fp32 accumulation throughout.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.hpp"
#include "index.cuh"
#include "stopnet.cuh"

namespace hnswgb {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxDeg = 64;  // neighbour slots scored per expansion

// Tuning switches (compile time).  HNSW_PREFETCH_ROWS: after the visited
// check, every lane owning a new neighbour prefetches its whole row into L2,
// so the later gather rounds of the batch hit L2 instead of waiting on DRAM
// one after another.  HNSW_PREFETCH_NEXT: while an element is expanded, the
// neighbour row of the next unexpanded entry of W is loaded speculatively;
// it is the next element to expand unless the current batch inserts a better
// one.
#ifndef HNSW_PREFETCH_ROWS
#define HNSW_PREFETCH_ROWS 0
#endif
#ifndef HNSW_PREFETCH_NEXT
#define HNSW_PREFETCH_NEXT 1
#endif
// HNSW_STOP_SKIP_IMPROVING: outside trace recording, a due check is put off
// while the expansion just done changed the K nearest of W (the search is
// still improving its answer), to the first later expansion that does not
#ifndef HNSW_STOP_SKIP_IMPROVING
#define HNSW_STOP_SKIP_IMPROVING 1
#endif
// HNSW_STOP_NOINLINE: the stop check (features + network) as a called
// function instead of inline code in the layer-0 loop
#ifndef HNSW_STOP_NOINLINE
#define HNSW_STOP_NOINLINE 0
#endif
#if HNSW_STOP_NOINLINE
#define HNSW_STOP_FN __device__ __noinline__
#else
#define HNSW_STOP_FN __device__ __forceinline__
#endif
// rows gathered per team and round for fp32 rows of 128 coordinates and for
// bf16/f16 rows of up to 128 coordinates
#ifndef HNSW_F32_U
#define HNSW_F32_U 2
#endif
#ifndef HNSW_B16_U
#define HNSW_B16_U 2
#endif
// HNSW_FP8_U: rows a team of fp8 rows keeps in flight (2: 64 registers,
// 32 warps per SM; 8 took 96 registers, 20 warps, and ran 1.7x slower)
#ifndef HNSW_FP8_U
#define HNSW_FP8_U 2
#endif
// HNSW_F16_U: the same for f16 rows (2: 64 registers; 4 took 80 registers
// and ran 1.2x slower).  HNSW_F16_NARROW: full f16 rows at the narrow budget
// (56, 36 warps): -1.5% overlapped but +8% for a batch alone, so off
#ifndef HNSW_F16_U
#define HNSW_F16_U 2
#endif
#ifndef HNSW_F16_NARROW
#define HNSW_F16_NARROW 0
#endif
// HNSW_MERGE_BALLOT: a merge with at most HNSW_MERGE_BALLOT_MAX candidates
// finds their places in W by ballots over the entries held in registers
// instead of a binary search
#ifndef HNSW_MERGE_BALLOT
#define HNSW_MERGE_BALLOT 1
#endif
#ifndef HNSW_MERGE_BALLOT_MAX
#define HNSW_MERGE_BALLOT_MAX 3
#endif
// HNSW_SORT_CHECK: after the rerank, W is sorted only when some adjacent
// pair is out of order
#ifndef HNSW_SORT_CHECK
#define HNSW_SORT_CHECK 1
#endif
// HNSW_MIXED_SUB: for bf16 / f16 rows and squared L2, x - q in one
// mixed-precision subtraction per coordinate (the 16-bit x taken as it is
// stored, q in fp32, the difference rounded once to fp32: the same value as
// decoding x to fp32 and subtracting)
#ifndef HNSW_MIXED_SUB
#define HNSW_MIXED_SUB 1
#endif

// x - q for the two 16-bit values of w (low half first), rounded once to fp32
template <int ST>
__device__ __forceinline__ void sub_halves(uint32_t w, float q0, float q1, float& t0, float& t1) {
    if (ST == HNSW_BF16)
        asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n sub.rn.f32.bf16 %0, l, %3;\n sub.rn.f32.bf16 %1, h, %4;\n}"
            : "=f"(t0), "=f"(t1) : "r"(w), "f"(q0), "f"(q1));
    else
        asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n sub.rn.f32.f16 %0, l, %3;\n sub.rn.f32.f16 %1, h, %4;\n}"
            : "=f"(t0), "=f"(t1) : "r"(w), "f"(q0), "f"(q1));
}

struct SearchArgs {
    DevIndex ix;
    const float* q;
    uint32_t n;
    int k;
    int efp;
    int efcap;      // power of two >= efp
    int hlog;       // log2 visited slots
    int warp_smem;  // bytes of shared memory per warp
    // per-warp layout: W, the visited set, ids, dst, nbuf (kMaxDeg entries
    // each) and aux (64 bytes) at fixed places, then at these byte offsets
    // from the warp's region: ck and lbs (present only when merge_batch or a
    // stop check may use them) and qs (the rerank's copy of q, in the
    // visited set's bytes when they suffice: it is filled after the search)
    int off_ck, off_lbs, off_qs;
    int rerank;
    uint32_t* out_ids;
    float* out_dists;
    hnsw_query_stats* stats;
    uint32_t* work;
    // learned stop: model (null: none), decision threshold on the logit,
    // check period in layer-0 expansions (0: no checks)
    const StopDev* stop;
    float stop_logit;
    int stop_period;
    // trace mode (tr_count != null): record every check, never stop early
    float* tr_feat;      // [n][tr_max][6]
    uint32_t* tr_topk;   // [n][tr_max][k]
    float* tr_logit;     // [n][tr_max] (only with a model)
    int32_t* tr_count;   // [n] checks recorded
    int tr_max;
    // two-pass scheduling: mode 0 = descent and beam per query in input order;
    // mode 1 = descent only, writing the layer-0 enter key and the upper-layer
    // counters of every query; mode 2 = beam only, queries taken in `order`
    // grouped launch (several requests in one launch): per-query k (low 16
    // bits) and ef (high 16 bits), and the first output slot of each query;
    // null: k, efp and qi * k for every query
    const uint32_t* q_kef;
    const uint64_t* q_out;
    int mode;
    uint64_t* ep_keys;   // [n]
    uint32_t* up_cnt;    // [n][2]: distance evaluations, rows read on layers >= 1
    const uint32_t* order;
    // deferral (mode 0, null: off): a query whose descent ends nearer than
    // the mean descent distance of the queries before it is pushed, with its
    // layer-0 enter key and upper-layer counters, and its beam runs once the
    // input queue is drained, so that the far (long) searches start first.
    // dfr_ctl: [0] records pushed, [1] claim tickets taken, [2] error (a
    // record that never appeared), [3] descents seen, [4] their distance sum
    // (fp32), [5] input-queue queries past their decision.
    // dfr_rec[i]: enter key low / high word, counters (rows read on layers
    // >= 1 << 20 | distance evaluations), query index -- written last, all
    // ones until then.
    uint32_t* dfr_ctl;
    uint4* dfr_rec;  // [n]
    int dfr_hold;    // test hook: query 0's decision is never counted
    uint32_t* err;   // the index's error word (host memory mapped on the device)
};

// ---- keys -----------------------------------------------------------------
// key = ord(dist) << 32 | id << 1 | expanded.  key >> 1 orders (dist, id).
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
__device__ __forceinline__ uint64_t mkkey(float d, uint32_t id) {
    return (uint64_t(f2ord(d)) << 32) | (uint64_t(id) << 1);
}
__device__ __forceinline__ uint32_t key_id(uint64_t k) { return uint32_t(k >> 1) & 0x7fffffffu; }
__device__ __forceinline__ float key_dist(uint64_t k) { return ord2f(uint32_t(k >> 32)); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
    const uint32_t hi = uint32_t(v >> 32), lo = uint32_t(v);
    const uint32_t mh = __reduce_min_sync(kFull, hi);
    const uint32_t ml = __reduce_min_sync(kFull, hi == mh ? lo : 0xffffffffu);
    return (uint64_t(mh) << 32) | ml;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// 16-byte asynchronous global -> shared copy (no registers held while in flight)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Row gathers are random and not reused by this SM: keep them out of L1 so
// that L1 holds what is reused (the stop network's weights).
#ifndef HNSW_ROW_NO_L1
#define HNSW_ROW_NO_L1 0
#endif
__device__ __forceinline__ uint4 ld_row_chunk(const uint4* p) {
    uint4 v;
#if HNSW_ROW_NO_L1
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
#else
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
#endif
    return v;
}

// ---- storage decoding -----------------------------------------------------
template <int ST>
struct Store;
template <>
struct Store<HNSW_F32> {
    static constexpr int CPC = 4;
    __device__ static void decode(const uint4& v, float* x) {
        x[0] = __uint_as_float(v.x); x[1] = __uint_as_float(v.y);
        x[2] = __uint_as_float(v.z); x[3] = __uint_as_float(v.w);
    }
};
template <>
struct Store<HNSW_BF16> {
    static constexpr int CPC = 8;
    __device__ static void decode(const uint4& v, float* x) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[2 * i] = __uint_as_float(w[i] << 16);
            x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};
template <>
struct Store<HNSW_F16> {
    static constexpr int CPC = 8;
    __device__ static void decode(const uint4& v, float* x) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h;
            memcpy(&h, &w[i], 4);
            const float2 f = __half22float2(h);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
};
template <>
struct Store<HNSW_FP8E4M3> {
    static constexpr int CPC = 16;
    __device__ static void decode(const uint4& v, float* x) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const __nv_fp8x2_storage_t pr = __nv_fp8x2_storage_t((w[i] >> (16 * j)) & 0xffffu);
                const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3);
                __half2 h;
                memcpy(&h, &hr, 4);
                const float2 f = __half22float2(h);
                x[4 * i + 2 * j] = f.x;
                x[4 * i + 2 * j + 1] = f.y;
            }
        }
    }
};

// ---- batched distance of n rows -------------------------------------------
// FULL: every row has exactly TEAM * CPL chunks (no per-chunk bounds test)
template <int ST, int TEAM, int CPL, int U, bool FULL>
struct Dist {
    static constexpr int CPC = Store<ST>::CPC;
    static constexpr int QF = CPL * CPC;  // query coordinates held per lane
    static constexpr int TEAMS = 32 / TEAM;
    static constexpr int RPR = TEAMS * U;  // rows per round
    static constexpr bool MIXED = HNSW_MIXED_SUB && (ST == HNSW_BF16 || ST == HNSW_F16);

    __device__ static void load_q(const float* qp, uint32_t d, float (&qr)[QF], int lane) {
        const int tl = lane % TEAM;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = tl + c * TEAM;
#pragma unroll
            for (int j = 0; j < CPC; ++j) {
                const uint32_t co = uint32_t(ch * CPC + j);
                qr[c * CPC + j] = co < d ? qp[co] : 0.0f;
            }
        }
    }

    // out[r] = distance(q, row ids[r]) for r < n
    __device__ static void run(const DevIndex& ix, const float (&qr)[QF], const uint32_t* ids, int n,
                               float* out, int lane) {
        const int team = lane / TEAM, tl = lane % TEAM;
        const uint32_t C = ix.row_chunks;
        for (int base = 0; base < n; base += RPR) {
            uint4 v[U][CPL];
            float sc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = base + u * TEAMS + team;
                const bool live = r < n;
                const uint32_t id = live ? ids[r] : 0u;
                const uint4* rowp = ix.vec + uint64_t(id) * C;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const uint32_t ch = uint32_t(tl + c * TEAM);
                    if (live && (FULL || ch < C))
                        v[u][c] = ld_row_chunk(rowp + ch);
                    else
                        v[u][c] = make_uint4(0u, 0u, 0u, 0u);
                }
                if (ST == HNSW_FP8E4M3) sc[u] = live ? __ldg(ix.scale + id) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float acc = 0.0f;
                if (MIXED && ix.metric == HNSW_L2SQ) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const uint32_t w[4] = {v[u][c].x, v[u][c].y, v[u][c].z, v[u][c].w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float t0, t1;
                            sub_halves<ST>(w[i], qr[c * CPC + 2 * i], qr[c * CPC + 2 * i + 1], t0, t1);
                            acc = fmaf(t0, t0, acc);
                            acc = fmaf(t1, t1, acc);
                        }
                    }
                } else {
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    float x[CPC];
                    Store<ST>::decode(v[u][c], x);
                    if (ix.metric == HNSW_L2SQ) {
#pragma unroll
                        for (int j = 0; j < CPC; ++j) {
                            const float xv = ST == HNSW_FP8E4M3 ? x[j] * sc[u] : x[j];
                            const float t = qr[c * CPC + j] - xv;
                            acc = fmaf(t, t, acc);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < CPC; ++j) {
                            const float xv = ST == HNSW_FP8E4M3 ? x[j] * sc[u] : x[j];
                            acc = fmaf(qr[c * CPC + j], xv, acc);
                        }
                    }
                }
                }
#pragma unroll
                for (int o = TEAM / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
                const int r = base + u * TEAMS + team;
                if (tl == 0 && r < n) out[r] = ix.metric == HNSW_L2SQ ? acc : 1.0f - acc;
            }
        }
    }
};

// exact fp32 distances from the fp32 copy (rerank): every row's lines are
// first requested into L2 (a lane per row), then teams of 8 lanes take a row
// each, 4 rows per warp round, every chunk a lane reads of its row (up to 32
// chunks per pass) loaded before any is used; q in shared memory
__device__ void dist32_rows(const DevIndex& ix, const float* qs, const uint32_t* ids, int n, float* out, int lane) {
    const int team = lane >> 3, tl = lane & 7;
    const uint32_t C = ix.row_chunks32;
    for (int r = lane; r < n; r += 32) {
        const uint8_t* rp = reinterpret_cast<const uint8_t*>(ix.vec32 + uint64_t(ids[r]) * C);
        for (uint32_t b = 0; b < C * 16; b += 128) prefetch_l2(rp + b);
    }
    const float4* q4 = reinterpret_cast<const float4*>(qs);
    for (int base = 0; base < n; base += 4) {
        const int r = base + team;
        const bool live = r < n;
        const uint4* rowp = ix.vec32 + uint64_t(live ? ids[r] : 0u) * C;
        float acc = 0.0f;
        for (uint32_t cb = 0; cb < C; cb += 32) {
            uint4 v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t ch = cb + uint32_t(tl + 8 * c);
                v[c] = (live && ch < C) ? ld_row_chunk(rowp + ch) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t ch = cb + uint32_t(tl + 8 * c);
                if (ch >= C) break;
                const float4 qq = q4[ch];
                const float qv[4] = {qq.x, qq.y, qq.z, qq.w};
                const float x[4] = {__uint_as_float(v[c].x), __uint_as_float(v[c].y), __uint_as_float(v[c].z),
                                    __uint_as_float(v[c].w)};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (ix.metric == HNSW_L2SQ) {
                        const float t = qv[j] - x[j];
                        acc = fmaf(t, t, acc);
                    } else {
                        acc = fmaf(qv[j], x[j], acc);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (tl == 0 && live) out[r] = ix.metric == HNSW_L2SQ ? acc : 1.0f - acc;
    }
}

// ---- visited set ------------------------------------------------------------
// 4-way bucketed hash of element ids: one 16-byte shared load reads a whole
// bucket; a miss stores the id into the bucket's first empty slot, or, when
// the bucket is full, over slot (id & 3) -- the set then forgets that slot's
// element (harmless, see the file header).  Two lanes of a warp inserting
// into the same slot at once lose one of the ids the same way.
// Returns true when `id` was not in the set (and records it).
__device__ __forceinline__ bool visit_new(uint32_t* H, int hlog, uint32_t id, uint32_t& flags) {
    const uint32_t b = (id * 2654435761u) >> (34 - hlog);  // bucket index, 2^(hlog-2) buckets
    uint4* bp = reinterpret_cast<uint4*>(H) + b;
    const uint4 v = *bp;
    if (v.x == id || v.y == id || v.z == id || v.w == id) return false;
    uint32_t* sl = reinterpret_cast<uint32_t*>(bp);
    int slot = v.x == kNone ? 0 : (v.y == kNone ? 1 : (v.z == kNone ? 2 : (v.w == kNone ? 3 : -1)));
    if (slot < 0) {
        slot = int(id & 3u);
        flags |= 1u;
    }
    sl[slot] = id;
    return true;
}

__device__ __forceinline__ int lower_bound_key(const uint64_t* W, int size, uint64_t k1) {
    int lo = 0, hi = size;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((W[mid] >> 1) < k1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Merges the n scored neighbours (ids[], dst[]) into W; returns the smallest
// index that received a new entry (INT_MAX if none).
__device__ int merge_batch(uint64_t* W, int& size, int efp, const uint32_t* ids, const float* dst, int n,
                           uint64_t* ck, uint32_t* lbs, int lane) {
    const bool full = size >= efp;
    const uint64_t wlast = size > 0 ? (W[size - 1] >> 1) : 0ull;
    int m = 0;
    for (int h = 0; h < n; h += 32) {
        const int j = h + lane;
        bool ok = false;
        uint64_t k = 0;
        int lb = 0;
        if (j < n) {
            k = mkkey(dst[j], ids[j]);
            ok = !(full && (k >> 1) > wlast);
            if (ok) {
                lb = lower_bound_key(W, size, k >> 1);
                if (lb < size && (W[lb] >> 1) == (k >> 1)) ok = false;  // already in W
            }
        }
        const unsigned msk = __ballot_sync(kFull, ok);
        if (ok) {
            const int pos = m + __popc(msk & lanemask_lt());
            ck[pos] = k;
            lbs[pos] = uint32_t(lb);
        }
        m += __popc(msk);
    }
    __syncwarp();
    if (m == 0) return INT_MAX;
    if (m == 1) {  // one new entry (the common case once W is full): shift and insert
        const int lb = int(lbs[0]);
        const uint64_t k = ck[0];
        int hi = min(size, efp - 1);
        while (hi > lb) {
            const int lo = max(lb, hi - 32);
            const int i = lo + lane;
            const uint64_t v = i < hi ? W[i] : 0ull;
            __syncwarp();
            if (i < hi) W[i + 1] = v;
            __syncwarp();
            hi = lo;
        }
        if (lane == 0) W[lb] = k;
        size = min(efp, size + 1);
        __syncwarp();
        return lb;
    }
    // final positions of the new entries: lb + rank among the new entries
    uint64_t myk[2] = {0ull, 0ull};
    int mypos[2] = {INT_MAX, INT_MAX};
    uint32_t mylb = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int j = t * 32 + lane;
        if (j < m) {
            const uint64_t k = ck[j];
            int r = 0;
            for (int i = 0; i < m; ++i) r += (ck[i] >> 1) < (k >> 1);
            myk[t] = k;
            mypos[t] = int(lbs[j]) + r;
            mylb = min(mylb, lbs[j]);
        }
    }
    const int lbmin = int(__reduce_min_sync(kFull, mylb));
    // shift the old entries from lbmin up, top chunk first
    int hi = size;
    while (hi > lbmin) {
        const int lo = max(lbmin, hi - 32);
        const int i = lo + lane;
        const bool act = i < hi;
        uint64_t v = 0ull;
        int cnt = 0;
        if (act) {
            v = W[i];
            for (int j = 0; j < m; ++j) cnt += int(lbs[j]) <= i;
        }
        __syncwarp();
        if (act && i + cnt < efp) W[i + cnt] = v;
        __syncwarp();
        hi = lo;
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
        if (mypos[t] < efp) W[mypos[t]] = myk[t];
    size = min(efp, size + m);
    __syncwarp();
    return lbmin;
}

// merge_batch for a list of at most 64 entries and at most 32 new
// neighbours (a lane each).  Every surviving neighbour finds its lower bound
// in W by a binary search of its own; one pass over the survivors then gives
// each its rank among them (its final position is lower bound + rank) and
// each W entry the number of survivors placed before it; W is read into
// registers (entries lane and lane + 32) before any write, and every entry is
// written once.  Same result as merge_batch.
__device__ int merge_small(uint64_t* W, int& size, int efp, const uint32_t* ids, const float* dst, int n,
                           int lane) {
    // W's entries lane and lane + 32 (beyond size: all ones, above every key)
    const uint64_t w0 = lane < size ? W[lane] : ~0ull;
    const uint64_t w1 = lane + 32 < size ? W[lane + 32] : ~0ull;
    const bool full = size >= efp;
    const uint64_t wlast = size > 0 ? (W[size - 1] >> 1) : 0ull;
    uint64_t k = 0, k1 = 0;
    bool ok = false;
    int lb = 0;
    if (lane < n) {
        k = mkkey(dst[lane], ids[lane]);
        k1 = k >> 1;
        ok = !(full && k1 > wlast);
    }
    const uint32_t cand = __ballot_sync(kFull, ok);
    if (cand == 0) return INT_MAX;
#if HNSW_MERGE_BALLOT
    if (__popc(cand) <= HNSW_MERGE_BALLOT_MAX) {
        // few candidates: each one's lower bound and duplicate test by two
        // ballots over the entries held in registers (keys compared without
        // the expanded bit: new keys have it clear)
        const uint64_t m0 = w0 & ~1ull, m1 = w1 & ~1ull;
        for (uint32_t bits = cand; bits; bits &= bits - 1) {
            const int sl = __ffs(bits) - 1;
            const uint64_t ks = __shfl_sync(kFull, k, sl);
            const int l = __popc(__ballot_sync(kFull, m0 < ks)) + __popc(__ballot_sync(kFull, m1 < ks));
            const bool dup = __any_sync(kFull, m0 == ks || m1 == ks);  // already in W
            if (lane == sl) {
                lb = l;
                ok = !dup;
            }
        }
    } else
#endif
    if (ok) {
#pragma unroll
        for (int step = 32; step > 0; step >>= 1)  // entries of W below k1
            if (lb + step <= size && (W[lb + step - 1] >> 1) < k1) lb += step;
        if (lb < size && (W[lb] >> 1) == k1) ok = false;  // already in W
    }
    const uint32_t surv = __ballot_sync(kFull, ok);
    if (surv == 0) return INT_MAX;
    int rank = 0, c0 = 0, c1 = 0;  // survivors below my key; placed before my W entries
    for (uint32_t bits = surv; bits; bits &= bits - 1) {
        const int sl = __ffs(bits) - 1;
        const uint64_t ks = __shfl_sync(kFull, k1, sl);
        const int ls = __shfl_sync(kFull, lb, sl);
        rank += ks < k1;
        c0 += ls <= lane;
        c1 += ls <= lane + 32;
    }
    __syncwarp();
    if (lane < size && lane + c0 < efp) W[lane + c0] = w0;
    if (lane + 32 < size && lane + 32 + c1 < efp) W[lane + 32 + c1] = w1;
    int pos = INT_MAX;
    if (ok) {
        pos = lb + rank;
        if (pos < efp)
            W[pos] = k;
        else
            pos = INT_MAX;
    }
    size = min(efp, size + __popc(surv));
    __syncwarp();
    return int(__reduce_min_sync(kFull, uint32_t(pos)));
}

// warp-wide bitonic sort of n (power of two) keys in shared memory
__device__ void warp_sort(uint64_t* a, int n, int lane) {
    for (int kk = 2; kk <= n; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const uint64_t x = a[i], y = a[p];
                    const bool up = (i & kk) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[p] = x;
                    }
                }
            }
            __syncwarp();
        }
}


// ---- deferred queries (mode 0) ----------------------------------------------
// Both run on one lane.  A claim takes the next ticket (one atomic, no
// retries) and waits for that slot's record -- written by a warp that holds
// the slot and is running -- or, when every query of the input queue has
// passed its decision and the slot was never pushed, gives up the ticket.
// The warps it waits for hold input-queue queries already (the queue is
// drained before any claim) and decide right after their descent.  The wait
// is bounded (2^20 polls, 0.1 to 1 s): a record that does not appear by then
// sets the error word and the claim gives up.
constexpr int kDeferSpin = 1 << 20;
constexpr uint32_t kDeferWarmup = 32;  // descents seen before any is deferred
// the automatic schedule defers in batches of up to 2^24 queries (256 MB of
// records); in larger ones the tail is a small part of the batch
constexpr uint64_t kDeferAutoMax = 1ull << 24;

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

// A pushed record (its .w = query index), or .w = kNone when none is left.
__device__ uint4 claim_deferred(const SearchArgs& a) {
    uint32_t* ctl = a.dfr_ctl;
    const uint32_t d = atomicAdd(ctl + 1, 1u);
    if (d >= a.n) return make_uint4(0u, 0u, 0u, kNone);
    const uint32_t* rw = reinterpret_cast<const uint32_t*>(a.dfr_rec + d);
    for (int it = 0; it < kDeferSpin; ++it) {
        const uint32_t q = ld_volatile_u32(rw + 3);
        if (q != kNone) {
            __threadfence();
            return make_uint4(ld_volatile_u32(rw), ld_volatile_u32(rw + 1), ld_volatile_u32(rw + 2), q);
        }
        if (ld_volatile_u32(ctl + 5) >= a.n) {  // every decision made: the pushes are final
            __threadfence();
            if (d >= ld_volatile_u32(ctl + 0)) return make_uint4(0u, 0u, 0u, kNone);
        }
        __nanosleep(128);
    }
    atomicExch(ctl + 2, 1u);
    if (a.err) {
        *reinterpret_cast<volatile uint32_t*>(a.err) = 1u;
        __threadfence_system();
    }
    return make_uint4(0u, 0u, 0u, kNone);
}

// Pushes query qi (layer-0 enter key, upper-layer counters) when its descent
// distance is below the mean of those seen before it; counts the decision
// (after the record is written) either way and returns whether it pushed.
__device__ bool maybe_defer(const SearchArgs& a, uint32_t qi, uint64_t cur, uint32_t n_eval, uint32_t n_stepU) {
    uint32_t* ctl = a.dfr_ctl;
    const float d1 = key_dist(cur);
    const uint32_t seen = atomicAdd(ctl + 3, 1u);
    const float sum = atomicAdd(reinterpret_cast<float*>(ctl + 4), d1);
    const bool push = seen >= kDeferWarmup && d1 * float(seen) < sum && n_eval < (1u << 20) && n_stepU < (1u << 12);
    if (push) {
        const uint32_t s = atomicAdd(ctl + 0, 1u);
        volatile uint32_t* rw = reinterpret_cast<volatile uint32_t*>(a.dfr_rec + s);
        rw[0] = uint32_t(cur);
        rw[1] = uint32_t(cur >> 32);
        rw[2] = (n_stepU << 20) | n_eval;
        __threadfence();
        rw[3] = qi;
    }
    __threadfence();
    if (!(a.dfr_hold && qi == 0)) atomicAdd(ctl + 5, 1u);
    return push;
}

// ---- the kernel -------------------------------------------------------------
// STOP: the build with learned-stop checks and trace recording (the plain
// search is compiled without them and keeps its smaller register budget).
// One learned-stop check of a warp's search: the six features of the state
// of W (aux: 1/d1, log1p(d1), layer-0 distance evaluations at entry) written
// to aux[4..9], and the network's logit (0 without a network).  log1p of the
// per-check features is taken as log(1 + x) with the fast logarithm.
HNSW_STOP_FN float stop_check(const StopDev* model, const uint64_t* W, int size, int kq, float* aux,
                              uint32_t n_eval0, uint32_t stale, float* hs, int lane) {
    const float inv_d1 = aux[0];
    float f[kStopIn];
    f[0] = __logf(1.0f + fmaxf(key_dist(W[0]) * inv_d1, 0.0f));
    f[1] = __logf(1.0f + fmaxf(key_dist(W[size - 1]) * inv_d1, 0.0f));
    f[2] = __logf(1.0f + float(n_eval0));
    f[3] = aux[1];
    f[4] = __logf(1.0f + float(stale));
    f[5] = __logf(1.0f + fmaxf(key_dist(W[kq - 1]) * inv_d1, 0.0f));
    float fv = f[0];
#pragma unroll
    for (int i = 1; i < kStopIn; ++i) fv = lane == i ? f[i] : fv;
    if (lane < kStopIn) aux[4 + lane] = fv;
    return model ? stop_logit<true>(model, f, hs, lane) : 0.0f;
}

// Register budget of each instantiation (per thread).  56 -- 9 blocks of 128
// threads resident per SM, 36 warps -- where the kernel fits in it without
// spilling (full bf16 rows of 2 chunks per lane, the 2-lane teams of low-d
// rows); 64 (8 blocks) for the other narrow ones; more where the rows in
// flight need them (fp32 128-d: 72; with the stop, the bounds checks or partial rows 80; fp8 with 8 rows
// per team, when HNSW_FP8_U asks for them: 96; f16 with 4 rows per team, when HNSW_F16_U asks: 80).  Without an explicit budget
// the compiler chose budgets that spilled.  Blocks of up to 256 threads are
// allowed so that large per-warp state (wide beams) can be packed into the
// shared memory of an SM (see the launch).
#ifndef HNSW_NARROW_REGS
#define HNSW_NARROW_REGS 56
#endif
// HNSW_STOP_NARROW: the learned-stop build of those instances takes the same
// budget (the bf16 one then spills 4 bytes, cheaper than 4 fewer warps per SM)
#ifndef HNSW_STOP_NARROW
#define HNSW_STOP_NARROW 1
#endif
template <int ST, int TEAM, int CPL, int U, bool FULL, bool STOP, bool CHECK>
constexpr int search_max_regs() {
    return (ST == HNSW_F32 && CPL == 4) ? ((STOP || CHECK || !FULL) ? 80 : 72)
         : (ST == HNSW_FP8E4M3 && U == 8) ? 96
         : (ST == HNSW_F16 && U == 4) ? 80
         : ((!STOP || HNSW_STOP_NARROW) && !CHECK &&
            (((ST == HNSW_BF16 || (ST == HNSW_F16 && HNSW_F16_NARROW)) && TEAM == 8 && CPL == 2 && FULL) || TEAM == 2)) ? HNSW_NARROW_REGS
                                                                              : 64;
}

// CHECK: the bounds-checked build (hnsw_search_params.check_bounds): every
// element id read from the graph is tested against N and every upper-row
// index against the rows allocated before any use; a query that meets a bad
// one sets stats flag bit 2 and leaves its search (its results are what W
// holds), with no device fault and no trap.
template <int ST, int TEAM, int CPL, int U, bool FULL, bool STOP, bool CHECK = false>
__global__ void __launch_bounds__(256) __maxnreg__((search_max_regs<ST, TEAM, CPL, U, FULL, STOP, CHECK>()))
    hnsw_search_kernel(const SearchArgs a) {
    using D = Dist<ST, TEAM, CPL, U, FULL>;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    uint8_t* wbase = smem + (threadIdx.x >> 5) * a.warp_smem;
    uint64_t* W = reinterpret_cast<uint64_t*>(wbase);
    uint32_t* H = reinterpret_cast<uint32_t*>(wbase + a.efcap * 8);
    uint32_t* ids = H + (1 << a.hlog);
    float* dst = reinterpret_cast<float*>(ids + kMaxDeg);
    uint32_t* nbuf = reinterpret_cast<uint32_t*>(dst + kMaxDeg);  // staged neighbour row (16-byte aligned)
    // per-query scalars read only at stop checks (kept out of registers):
    // 1/d1, log1p(d1), n_eval at layer 0 entry, checks recorded; [4..9] the
    // features of the last check
    float* aux = reinterpret_cast<float*>(nbuf + kMaxDeg);
    uint32_t* n_checks = reinterpret_cast<uint32_t*>(aux + 3);
    const DevIndex& ix = a.ix;
    const int hsz = 1 << a.hlog;
    for (;;) {
        uint32_t qi = 0;
        if (lane == 0) qi = atomicAdd(a.work, 1u);
        qi = __shfl_sync(kFull, qi, 0);
        // a deferred query taken up again (its enter key and counters parked
        // in aux words 10-12 until the beam starts)
        bool resumed = false;
        if (qi >= a.n) {
            if (CHECK || !a.dfr_ctl) break;
            // the input queue is drained: the deferred queries' beams
            if (lane == 0) {
                const uint4 r = claim_deferred(a);
                uint32_t* park = reinterpret_cast<uint32_t*>(aux) + 10;
                park[0] = r.x;
                park[1] = r.y;
                park[2] = r.z;
                qi = r.w;
            }
            qi = __shfl_sync(kFull, qi, 0);
            if (qi == kNone) break;
            resumed = true;
        }
        if (a.mode == 2) qi = __ldg(a.order + qi);
        const float* qp = a.q + uint64_t(qi) * ix.d;
        // per-query k and ef of a grouped launch (k is reread where needed so
        // that only ef stays live through the search)
        int efq = a.efp;
        if (a.q_kef) {
            const uint32_t v = __ldg(a.q_kef + qi);
            efq = max(int(v & 0xffffu), int(v >> 16));
        }
        float qr[D::QF];
        D::load_q(qp, ix.d, qr, lane);
        for (int i = lane; i < (hsz >> 2); i += 32)
            reinterpret_cast<uint4*>(H)[i] = make_uint4(kNone, kNone, kNone, kNone);
        uint32_t n_eval = 0, n_exp0 = 0, n_stepU = 0, flags = 0;
        if (STOP && lane == 0) *n_checks = 0;
        int size = 0;
        __syncwarp();
        bool bad = CHECK && ix.N > 0 && !(ix.ep < ix.N);  // bounds-checked build: a bad id or row met
        if (ix.N > 0 && !bad) {
            uint64_t cur = 0;
            if (resumed) {  // the descent ran before the query was deferred
                const uint32_t* park = reinterpret_cast<const uint32_t*>(aux) + 10;
                cur = (uint64_t(park[1]) << 32) | park[0];
                n_eval = park[2] & 0xfffffu;
                n_stepU = park[2] >> 20;
            } else if (a.mode == 2) {  // the descent ran in the first pass
                cur = a.ep_keys[qi];
                n_eval = a.up_cnt[2 * uint64_t(qi)];
                n_stepU = a.up_cnt[2 * uint64_t(qi) + 1];
            } else {
            // enter point and greedy descent (Alg. 5)
            if (lane == 0) ids[0] = ix.ep;
            __syncwarp();
            D::run(ix, qr, ids, 1, dst, lane);
            __syncwarp();
            cur = mkkey(dst[0], ix.ep);
            n_eval = 1;
            uint32_t cur_uo = ix.maxlevel >= 1 ? __ldg(ix.upoff + key_id(cur)) : kNone;  // cur's first upper row
            for (int lc = ix.maxlevel; lc >= 1 && !bad; --lc) {
                for (;;) {
                    const uint64_t row = uint64_t(cur_uo) + uint64_t(lc - 1);
                    if (CHECK && !(row < ix.urows)) {  // c absent from layer lc, or a bad offset
                        bad = true;
                        break;
                    }
                    const uint32_t* urow = ix.nbrU + row * ix.sU;
                    int n = 0;
                    __syncwarp();
                    for (int h = 0; h < int(ix.Mmax); h += 32) {
                        const int j = h + lane;
                        uint32_t e = j < int(ix.Mmax) ? __ldg(urow + j) : kNone;
                        if (CHECK && e != kNone && !(e < ix.N)) {
                            bad = true;
                            e = kNone;
                        }
                        const bool v = e != kNone;
                        const unsigned m = __ballot_sync(kFull, v);
                        if (v) ids[n + __popc(m & lanemask_lt())] = e;
                        n += __popc(m);
                    }
                    if (CHECK && __any_sync(kFull, bad)) {
                        bad = true;
                        break;
                    }
                    __syncwarp();
                    D::run(ix, qr, ids, n, dst, lane);
                    __syncwarp();
                    n_eval += n;
                    ++n_stepU;  // one upper-layer element expanded (its row read)
                    uint64_t kb = lane < n ? mkkey(dst[lane], ids[lane]) : ~0ull;
                    kb = warp_min_u64(kb);
                    if ((kb >> 1) < (cur >> 1)) {
                        cur = kb;
                        cur_uo = __ldg(ix.upoff + key_id(kb));
                    } else {
                        break;
                    }
                }
            }
            }
            if (a.mode == 1) {  // first pass: keep the layer-0 enter point for the second
                if (lane == 0) {
                    a.ep_keys[qi] = cur;
                    a.up_cnt[2 * uint64_t(qi)] = n_eval;
                    a.up_cnt[2 * uint64_t(qi) + 1] = n_stepU;
                }
                __syncwarp();
                continue;
            }
            if (!CHECK && a.dfr_ctl && !resumed) {
                bool deferred = false;
                if (lane == 0) deferred = maybe_defer(a, qi, cur, n_eval, n_stepU);
                if (__shfl_sync(kFull, deferred, 0)) continue;  // its beam runs later
            }
            // layer 0 beam (Alg. 2 with ef')
            if (lane == 0) {
                W[0] = cur & ~1ull;
                visit_new(H, a.hlog, key_id(cur), flags);
            }
            size = 1;
            int scan = 0;
            const int deg = int(ix.Mmax0);
            if (STOP && lane == 0) {
                const float d1 = key_dist(cur);  // where the upper-layer descent ended
                aux[0] = 1.0f / fmaxf(d1, 1e-12f);
                aux[1] = log1pf(fmaxf(d1, 0.0f));
                aux[2] = __uint_as_float(n_eval);
            }
            // stale (expansions since the K nearest of W last changed) in the
            // high half, expansions left to the next check in the low half
            uint32_t stale_cd = STOP ? uint32_t(a.stop_period) : 0u;
            uint32_t nxt_id = kNone;  // element whose neighbour row is staged in nbuf
            __syncwarp();
            for (;;) {
                if (CHECK && bad) break;  // the descent met a bad id or row: W holds its last element
                int p = -1;
                // the window of W where p was found: its unexpanded entries
                // (bit per lane) and this lane's entry, for the next one after p
                unsigned win_m = 0u;
                uint32_t win_id = 0u;
                for (int s = scan; s < size; s += 32) {
                    // the low word of a key holds the id and the expanded bit
                    const int i = s + lane;
                    const uint32_t wlo = i < size ? reinterpret_cast<const uint32_t*>(W)[2 * i] : 1u;
                    const bool un = !(wlo & 1u);
                    const unsigned m = __ballot_sync(kFull, un);
                    if (m) {
                        const int b = __ffs(m) - 1;
                        p = s + b;
                        win_m = b < 31 ? (m & (~0u << (b + 1))) : 0u;
                        win_id = (wlo >> 1) & 0x7fffffffu;
                        break;
                    }
                }
                if (p < 0) {  // every entry of W expanded: Alg. 2 stops
                    if (nxt_id != kNone) cp_async_wait_all();
                    break;
                }
                const uint64_t kc = W[p];
                __syncwarp();
                if (lane == 0) W[p] = kc | 1ull;
                ++n_exp0;
                const uint32_t c = key_id(kc);
                const uint32_t* nrow = ix.nbr0 + uint64_t(c) * ix.s0;
                // was this row staged in shared memory during the previous expansion?
                const bool staged = c == nxt_id;
                if (nxt_id != kNone) {
                    cp_async_wait_all();
                    __syncwarp();
                }
                uint32_t e0 = kNone, e1 = kNone;
                if (staged) {
                    e0 = lane < deg ? nbuf[lane] : kNone;
                    if (deg > 32) e1 = lane + 32 < deg ? nbuf[32 + lane] : kNone;
                } else {
                    e0 = lane < deg ? __ldg(nrow + lane) : kNone;
                    if (deg > 32) e1 = lane + 32 < deg ? __ldg(nrow + 32 + lane) : kNone;
                }
                __syncwarp();
                if (CHECK && __any_sync(kFull, (e0 != kNone && !(e0 < ix.N)) || (e1 != kNone && !(e1 < ix.N)))) {
                    bad = true;  // no copy is in flight here: the staged row was waited for above
                    nxt_id = kNone;
                    break;
                }
#if HNSW_PREFETCH_NEXT
                // the next unexpanded entry after p is expanded next unless this
                // batch inserts a better element: stage its neighbour row now
                nxt_id = kNone;
                {
                    // within the window of p when it holds one, else the 32
                    // entries after p
                    unsigned m = win_m;
                    uint32_t id = win_id;
                    if (!m) {
                        const int i = p + 1 + lane;
                        const uint32_t wlo = i < size ? reinterpret_cast<const uint32_t*>(W)[2 * i] : 1u;
                        m = __ballot_sync(kFull, !(wlo & 1u));
                        id = (wlo >> 1) & 0x7fffffffu;
                    }
                    if (m) {
                        nxt_id = __shfl_sync(kFull, id, __ffs(m) - 1);
                        const uint32_t* np = ix.nbr0 + uint64_t(nxt_id) * ix.s0;
                        if (lane * 4 < deg) cp_async16(nbuf + lane * 4, np + lane * 4);
                        cp_async_commit();
                    }
                }
#endif
                int n = 0;
                {
                    const bool nw = e0 != kNone && visit_new(H, a.hlog, e0, flags);
                    const unsigned m = __ballot_sync(kFull, nw);
                    if (nw) ids[__popc(m & lanemask_lt())] = e0;
                    n = __popc(m);
                }
                if (deg > 32) {
                    const bool nw = e1 != kNone && visit_new(H, a.hlog, e1, flags);
                    const unsigned m = __ballot_sync(kFull, nw);
                    if (nw) ids[n + __popc(m & lanemask_lt())] = e1;
                    n += __popc(m);
                }
                __syncwarp();
                int first_new = INT_MAX;
                if (n > 0) {
#if HNSW_PREFETCH_ROWS
                    // rows beyond the first gather round: start their DRAM reads now
                    if (n > D::RPR) {
                        for (int j = D::RPR + lane; j < n; j += 32) {
                            const uint8_t* rp =
                                reinterpret_cast<const uint8_t*>(ix.vec + uint64_t(ids[j]) * ix.row_chunks);
                            for (uint32_t b = 0; b < ix.row_chunks * 16; b += 128) prefetch_l2(rp + b);
                        }
                    }
#endif
                    D::run(ix, qr, ids, n, dst, lane);
                    __syncwarp();
                    n_eval += n;
                    first_new = (a.efcap <= 64 && n <= 32)
                                    ? merge_small(W, size, efq, ids, dst, n, lane)
                                    : merge_batch(W, size, efq, ids, dst, n,
                                                  reinterpret_cast<uint64_t*>(wbase + a.off_ck),
                                                  reinterpret_cast<uint32_t*>(wbase + a.off_lbs), lane);
                }
                scan = min(p + 1, first_new);
                if (STOP && a.stop_period > 0) {
                    const int kq = a.q_kef ? int(__ldg(a.q_kef + qi) & 0xffffu) : a.k;
                    // stale: expansions since an element entered the K nearest of W
                    // (once W holds K entries: since its K-th key last decreased),
                    // saturating at 65535
                    stale_cd = first_new < kq ? (stale_cd & 0xffffu) : __vaddus2(stale_cd, 0x10000u);
                    stale_cd -= 1u;
                    bool check = (stale_cd & 0xffffu) == 0u;
                    if (HNSW_STOP_SKIP_IMPROVING && check && !a.tr_count && first_new < kq) {
                        check = false;  // put off to the next expansion
                        stale_cd |= 1u;
                    }
                    if (check) stale_cd |= uint32_t(a.stop_period);
                    if (size >= kq && check) {
                        __syncwarp();
                        const StopDev* model = a.stop;  // global memory, read through L1
                        const float logit = stop_check(model, W, size, kq, aux, n_eval - __float_as_uint(aux[2]),
                                                       stale_cd >> 16, reinterpret_cast<float*>(wbase + a.off_ck), lane);
                        if (a.tr_count) {
                            __syncwarp();
                            const uint32_t c = *n_checks;
                            if (c < uint32_t(a.tr_max)) {
                                const uint64_t slot = uint64_t(qi) * uint64_t(a.tr_max) + c;
                                if (lane < kStopIn) a.tr_feat[slot * kStopIn + lane] = aux[4 + lane];
                                if (lane == 0 && a.tr_logit) a.tr_logit[slot] = logit;
                                for (int i = lane; i < a.k; i += 32) a.tr_topk[slot * uint64_t(a.k) + i] = key_id(W[i]);
                            }
                            __syncwarp();
                            if (lane == 0) *n_checks = c + 1;
                        } else if (model && logit > a.stop_logit) {
                            flags |= 2u;  // learned stop: W's top-K is predicted final
                            if (nxt_id != kNone) cp_async_wait_all();
                            __syncwarp();
                            break;
                        }
                    }
                }
            }
        }
        // results (the K nearest of W, Alg. 5)
        if (a.rerank && size > 0) {
            float* qs = reinterpret_cast<float*>(wbase + a.off_qs);
            const float* qrow = a.q + uint64_t(qi) * ix.d;  // re-derived: keeps qp out of the loop's registers
            __syncwarp();
            for (uint32_t i = lane; i < ix.row_chunks32 * 4; i += 32) qs[i] = i < ix.d ? qrow[i] : 0.0f;
            __syncwarp();
            for (int b = 0; b < size; b += kMaxDeg) {
                const int nb = min(kMaxDeg, size - b);
                for (int i = lane; i < nb; i += 32) ids[i] = key_id(W[b + i]);
                __syncwarp();
                dist32_rows(ix, qs, ids, nb, dst, lane);
                __syncwarp();
                for (int i = lane; i < nb; i += 32) W[b + i] = mkkey(dst[i], ids[i]);
                __syncwarp();
            }
            for (int i = size + lane; i < a.efcap; i += 32) W[i] = ~0ull;
            __syncwarp();
#if HNSW_SORT_CHECK
            // keys are distinct (distinct ids): W needs no sort when every
            // adjacent pair is still in order
            bool unsorted = false;
            for (int i = lane; i + 1 < size; i += 32) unsorted |= W[i] > W[i + 1];
            if (__any_sync(kFull, unsorted))
#endif
                warp_sort(W, a.efcap, lane);
        }
        const int kq = a.q_kef ? int(__ldg(a.q_kef + qi) & 0xffffu) : a.k;
        const uint64_t obase = a.q_kef ? __ldg(a.q_out + qi) : uint64_t(qi) * uint64_t(a.k);
        for (int i = lane; i < kq; i += 32) {
            uint32_t oid = kNone;
            float od = __int_as_float(0x7f800000);
            if (i < size) {
                const uint64_t kk = W[i];
                oid = key_id(kk);
                od = key_dist(kk);
            }
            a.out_ids[obase + i] = oid;
            a.out_dists[obase + i] = od;
        }
        if (CHECK && bad) flags |= 4u;
        if (STOP && a.tr_count && lane == 0) a.tr_count[qi] = int(min(*n_checks, uint32_t(a.tr_max)));
        if (a.stats && lane == 0) {
            hnsw_query_stats s;
            s.n_eval = n_eval;
            s.n_exp0 = n_exp0;
            s.n_stepU = n_stepU;
            s.flags = flags;
            a.stats[qi] = s;
        }
        __syncwarp();
    }
}

// ---- ordering of the second pass --------------------------------------------
// Queries whose upper-layer descent ends far from them tend to need more
// layer-0 expansions; starting them first shortens the tail of the batch
// (longest-first list scheduling).  The order need not be exact: one block
// takes a chunk of up to kSortChunk queries and places them by a counting
// sort into kOrderBuckets buckets spanning the chunk's range of descent
// distances (linear in the distances' ordered bit patterns, so about
// logarithmic in the distances), farthest first; chunks are ordered
// independently.  Block barriers only (no spin-waits); launched with one
// thread per bucket.
constexpr int kSortChunk = 16384;
constexpr int kOrderBuckets = 1024;
static_assert(kOrderBuckets == 1024, "the prefix sum takes one bucket per thread of a 1024-thread block");

__global__ void __launch_bounds__(1024) order_by_descent(const uint64_t* __restrict__ ep_keys, uint32_t n,
                                                        uint32_t* __restrict__ order) {
    __shared__ uint32_t hist[kOrderBuckets];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t range[2];
    const uint32_t base = blockIdx.x * uint32_t(kSortChunk);
    const uint32_t m = min(uint32_t(kSortChunk), n - base);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < kOrderBuckets; i += blockDim.x) hist[i] = 0u;
    if (t == 0) {
        range[0] = ~0u;
        range[1] = 0u;
    }
    __syncthreads();
    // the chunk's range of ordered distance bits (the high word of a key)
    uint32_t lo = ~0u, hi = 0u;
    for (uint32_t i = t; i < m; i += blockDim.x) {
        const uint32_t v = uint32_t(ep_keys[base + i] >> 32);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if (lane == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
    __syncthreads();
    lo = range[0];
    hi = range[1];
    const uint64_t span = uint64_t(hi - lo) + 1u;  // >= 1 (m >= 1)
    // bucket of a key: 0 for the farthest enter point
    auto bucket = [&](uint32_t i) {
        const uint32_t v = uint32_t(ep_keys[base + i] >> 32);
        return uint32_t((uint64_t(hi - v) * uint64_t(kOrderBuckets)) / span);
    };
    for (uint32_t i = t; i < m; i += blockDim.x) atomicAdd(&hist[bucket(i)], 1u);
    __syncthreads();
    // exclusive prefix sum of the histogram (one entry per thread)
    const uint32_t x = t < kOrderBuckets ? hist[t] : 0u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int nw = int(blockDim.x) >> 5;
        uint32_t w = lane < nw ? wsum[lane] : 0u, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) wsum[lane] = wi - w;  // exclusive over warps
    }
    __syncthreads();
    if (t < kOrderBuckets) hist[t] = wsum[wid] + inc - x;
    __syncthreads();
    // scatter: the slots of a bucket go to its queries in any order
    for (uint32_t i = t; i < m; i += blockDim.x) order[base + atomicAdd(&hist[bucket(i)], 1u)] = base + i;
}

// ---- host side --------------------------------------------------------------
namespace {

using KernelFn = void (*)(const SearchArgs);

struct KernelChoice {
    KernelFn fn;
    const char* name;
};

template <int ST, int TEAM, int CPL, int U>
KernelChoice pick(uint32_t chunks, bool stop) {
    if (chunks == uint32_t(TEAM * CPL))
        return {stop ? hnsw_search_kernel<ST, TEAM, CPL, U, true, true> : hnsw_search_kernel<ST, TEAM, CPL, U, true, false>,
                "hnsw_search_kernel"};
    return {stop ? hnsw_search_kernel<ST, TEAM, CPL, U, false, true> : hnsw_search_kernel<ST, TEAM, CPL, U, false, false>,
            "hnsw_search_kernel"};
}

// (storage, chunks per row) -> instantiation
bool choose_kernel(int storage, uint32_t chunks, bool stop, KernelChoice& kc) {
    switch (storage) {
        case HNSW_F32:
            if (chunks <= 2) { kc = pick<HNSW_F32, 2, 1, 2>(chunks, stop); return true; }
            if (chunks <= 8) { kc = pick<HNSW_F32, 8, 1, 8>(chunks, stop); return true; }
            if (chunks <= 32) { kc = pick<HNSW_F32, 8, 4, HNSW_F32_U>(chunks, stop); return true; }
            if (chunks <= 128) { kc = pick<HNSW_F32, 32, 4, 1>(chunks, stop); return true; }
            return false;
        case HNSW_BF16:
            if (chunks <= 2) { kc = pick<HNSW_BF16, 2, 1, 2>(chunks, stop); return true; }
            if (chunks <= 16) { kc = pick<HNSW_BF16, 8, 2, HNSW_B16_U>(chunks, stop); return true; }
            if (chunks <= 64) { kc = pick<HNSW_BF16, 32, 2, 1>(chunks, stop); return true; }
            return false;
        case HNSW_F16:
            if (chunks <= 2) { kc = pick<HNSW_F16, 2, 1, 2>(chunks, stop); return true; }
            if (chunks <= 16) { kc = pick<HNSW_F16, 8, 2, HNSW_F16_U>(chunks, stop); return true; }
            if (chunks <= 64) { kc = pick<HNSW_F16, 32, 2, 1>(chunks, stop); return true; }
            return false;
        case HNSW_FP8E4M3:
            if (chunks <= 8) { kc = pick<HNSW_FP8E4M3, 8, 1, HNSW_FP8_U>(chunks, stop); return true; }
            if (chunks <= 32) { kc = pick<HNSW_FP8E4M3, 32, 1, 1>(chunks, stop); return true; }
            return false;
    }
    return false;
}

// The bounds-checked build, for f32 rows of up to 32 chunks and bf16 rows of
// up to 16 (d <= 128 either way).
template <int ST, int TEAM, int CPL, int U>
KernelChoice pick_checked(uint32_t chunks) {
    if (chunks == uint32_t(TEAM * CPL))
        return {hnsw_search_kernel<ST, TEAM, CPL, U, true, false, true>, "hnsw_search_kernel (checked)"};
    return {hnsw_search_kernel<ST, TEAM, CPL, U, false, false, true>, "hnsw_search_kernel (checked)"};
}

bool choose_kernel_checked(int storage, uint32_t chunks, KernelChoice& kc) {
    if (storage == HNSW_F32 && chunks <= 8) { kc = pick_checked<HNSW_F32, 8, 1, 8>(chunks); return true; }
    if (storage == HNSW_F32 && chunks <= 32) { kc = pick_checked<HNSW_F32, 8, 4, HNSW_F32_U>(chunks); return true; }
    if (storage == HNSW_BF16 && chunks <= 16) { kc = pick_checked<HNSW_BF16, 8, 2, HNSW_B16_U>(chunks); return true; }
    return false;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int ceil_log2(uint64_t x) {
    int r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

// Warps per block (1..8) that put the most warps of kernel fn on an SM
// given `warp_smem` bytes of shared memory per warp (the fewest warps per
// block among equals: finer-grained blocks), and the blocks per SM then.
// Small per-warp state is bound by registers (4-warp blocks); a wide beam's
// state is bound by shared memory, where the block size decides how much of
// an SM's 228 KB the blocks fill.  Cached per (device, kernel, size).
bool block_choice(KernelFn fn, size_t warp_smem, int& warps, int& per_sm) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, std::pair<int, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, reinterpret_cast<const void*>(fn), warp_smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            warps = it->second.first;
            per_sm = it->second.second;
            return true;
        }
    }
    int best = 0;
    warps = 0;
    per_sm = 0;
    for (int w : {4, 5, 6, 7, 8, 3, 2, 1}) {
        const size_t sm = size_t(w) * warp_smem;
        if (sm > 227 * 1024) continue;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, w * 32, sm) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (b * w > best) {
            best = b * w;
            warps = w;
            per_sm = b;
        }
    }
    if (best == 0) return false;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {warps, per_sm};
    return true;
}

}  // namespace

// Upper bound of the automatic visited set: about 8-16 slots per beam entry,
// 1,024 to 4,096 slots (a layer-0 search evaluates some 10-30 x ef'
// elements); the launch takes the largest size up to it that costs no
// resident warps, and not below kMinAutoHlog.
constexpr int kMinAutoHlog = 8;
int auto_visited_log2(int efp) {
    int l = ceil_log2(uint64_t(efp) * 8);
    return l < 10 ? 10 : (l > 12 ? 12 : l);
}

hnsw_status launch_search_mode(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n,
                               uint32_t* ids, float* dists, hnsw_query_stats* stats, cudaStream_t s,
                               uint32_t* work, const StopModel* stop, int mode, uint64_t* ep_keys,
                               uint32_t* up_cnt, const uint32_t* order, const uint32_t* q_kef = nullptr,
                               const uint64_t* q_out = nullptr, const DevIndex* view = nullptr,
                               uint32_t* dfr_ctl = nullptr, uint4* dfr_rec = nullptr) {
    const DevIndex D = view ? *view : dev_snapshot(ix);
    KernelChoice kc;
    if (p.check_bounds) {
        if (stop != nullptr) return fail(HNSW_EINVAL, "search: check_bounds with the learned stop or a trace");
        if (!choose_kernel_checked(D.storage, D.row_chunks, kc))
            return fail(HNSW_EINVAL, "search: check_bounds is built for f32 rows of d <= 128 and bf16 of d <= 128");
    } else if (!choose_kernel(D.storage, D.row_chunks, stop != nullptr && stop->period > 0, kc)) {
        return fail(HNSW_EINVAL, "search: unsupported row size");
    }
    SearchArgs a{};
    a.ix = D;
    a.q = q;
    a.n = n;
    a.k = p.k;
    a.efp = p.ef > p.k ? p.ef : p.k;
    a.efcap = 1 << ceil_log2(uint64_t(a.efp < 32 ? 32 : a.efp));
    a.rerank = p.rerank;
    a.out_ids = ids;
    a.out_dists = dists;
    a.stats = stats;
    a.work = work;
    a.mode = mode;
    a.q_kef = q_kef;
    a.q_out = q_out;
    a.ep_keys = ep_keys;
    a.up_cnt = up_cnt;
    a.order = order;
    a.dfr_ctl = p.check_bounds ? nullptr : dfr_ctl;
    a.dfr_rec = dfr_rec;
    a.dfr_hold = ix->hold_decisions.load() ? 1 : 0;
    a.err = ix->d_err;
    if (stop) {
        a.stop = static_cast<const StopDev*>(stop->stop);
        a.stop_logit = stop->logit_threshold;
        a.stop_period = stop->period;
        a.tr_feat = stop->tr_feat;
        a.tr_topk = stop->tr_topk;
        a.tr_logit = stop->tr_logit;
        a.tr_count = stop->tr_count;
        a.tr_max = stop->tr_max;
    }
    const bool stop_build = stop != nullptr && stop->period > 0;
    const size_t row32 = size_t(D.row_chunks32) * 16;
    // per-warp layout with a visited set of 2^hl slots (every piece a
    // multiple of 16 bytes); sets the offsets in t, returns the bytes
    auto layout = [&](int hl, SearchArgs& t) {
        const size_t hbytes = (size_t(1) << hl) * 4;
        size_t per_warp = size_t(t.efcap) * 8 + hbytes + kMaxDeg * 12 + 64;
        // merge_batch (W above 64 entries, or a neighbour batch above 32) and
        // the stop check's scratch use ck and lbs
        if (stop_build || t.efcap > 64 || D.s0 > 32) {
            t.off_ck = int(per_warp);
            t.off_lbs = int(per_warp + kMaxDeg * 8);
            per_warp += kMaxDeg * 12;
        } else {
            t.off_ck = t.off_lbs = 0;
        }
        if (!p.rerank || hbytes >= row32) {
            t.off_qs = t.efcap * 8;  // the visited set's bytes
        } else {
            t.off_qs = int(per_warp);
            per_warp += row32;
        }
        return per_warp;
    };
    int hl = p.visited_log2 > 0 ? p.visited_log2 : auto_visited_log2(a.efp);
    if (p.visited_log2 <= 0) {
        // automatic: the largest set, down to 2^8 slots, that keeps as many
        // warps resident as the smallest does.  A forgotten element only
        // costs a repeated evaluation, while the warps resident decide how
        // much of the gathers' latency is hidden (a wide beam's state is
        // bound by shared memory, a narrow one's by registers).
        SearchArgs t = a;
        const size_t most = std::min<size_t>(227 * 1024, size_t(8) * layout(hl, t));
        const hnsw_status st = raise_smem_limit(reinterpret_cast<const void*>(kc.fn), most, "search");
        if (st != HNSW_OK) return st;
        int w0 = 0, b0 = 0;
        if (!block_choice(kc.fn, layout(kMinAutoHlog, t), w0, b0))
            return fail(HNSW_ECUDA, "search: occupancy query failed");
        for (; hl > kMinAutoHlog; --hl) {
            const size_t pw = layout(hl, t);
            int w = 0, b = 0;
            if (pw <= 227 * 1024 && block_choice(kc.fn, pw, w, b) && w * b >= w0 * b0) break;
        }
    }
    a.hlog = hl;
    const size_t per_warp = layout(hl, a);
    a.warp_smem = int(per_warp);
    if (size_t(a.warp_smem) > 227 * 1024)
        return fail(HNSW_EINVAL, "search: ef/visited set too large for shared memory");
    int dev = 0, sms = 0, per_sm = 0, warps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        const size_t most = std::min<size_t>(227 * 1024, size_t(8) * a.warp_smem);
        const hnsw_status st = raise_smem_limit(reinterpret_cast<const void*>(kc.fn), most, "search");
        if (st != HNSW_OK) return st;
    }
    if (!block_choice(kc.fn, size_t(a.warp_smem), warps, per_sm))
        return fail(HNSW_ECUDA, "search: occupancy query failed");
    const size_t smem = size_t(warps) * a.warp_smem;
    const uint64_t need = (uint64_t(n) + warps - 1) / warps;
    const uint64_t cap = uint64_t(per_sm) * uint64_t(sms);
    const unsigned grid = unsigned(need < cap ? need : cap);
    kc.fn<<<grid, warps * 32, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("search launch: ") + cudaGetErrorString(e));
    return HNSW_OK;
}

hnsw_status launch_search(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n,
                          uint32_t* ids, float* dists, hnsw_query_stats* stats, cudaStream_t s,
                          uint32_t* work, const StopModel* stop) {
    return launch_search_mode(ix, p, q, n, ids, dists, stats, s, work, stop, 0, nullptr, nullptr, nullptr);
}

// One-pass launch over an explicit device view of the index (graph
// construction and insertion search views that are not published).
hnsw_status launch_search_view(hnsw_index* ix, const DevIndex& view, const hnsw_search_params& p, const float* q,
                               uint32_t n, uint32_t* ids, float* dists, cudaStream_t s, uint32_t* work) {
    return launch_search_mode(ix, p, q, n, ids, dists, nullptr, s, work, nullptr, 0, nullptr, nullptr, nullptr,
                              nullptr, nullptr, &view);
}

// Grouped launch for the server: n queries of several requests on one index,
// per-query k/ef packed in q_kef and output offsets in q_out (device arrays),
// with max_k and max_ef sizing the per-warp state.
hnsw_status launch_search_group(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n,
                                int max_k, int max_ef, const uint32_t* q_kef, const uint64_t* q_out,
                                uint32_t* ids, float* dists, cudaStream_t s, uint32_t* work,
                                const StopModel* stop) {
    hnsw_search_params pp = p;
    pp.k = max_k;
    pp.ef = max_ef;
    cudaError_t e = cudaMemsetAsync(work, 0, 4, s);
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("search group: ") + cudaGetErrorString(e));
    return launch_search_mode(ix, pp, q, n, ids, dists, nullptr, s, work, stop, 0, nullptr, nullptr, nullptr,
                              q_kef, q_out);
}

// A pair of work counters for one call (slots 2i and 2i+1 of the index's
// ring): concurrent calls on one index use different counters.
uint32_t take_work_slots(hnsw_index* ix) {
    return (ix->work_next.fetch_add(1) % uint32_t(kWorkSlots / 2)) * 2u;
}

// The scheduling scratch (two passes, deferral) comes from the device's
// default stream-ordered pool, which by default hands freed memory back at
// every synchronisation, so that the next call maps it again.  This process
// keeps up to 256 MB of it cached (an attribute of the process's pool,
// nothing of the device's settings).
#ifndef HNSW_POOL_KEEP
#define HNSW_POOL_KEEP 1
#endif
void keep_pool_memory() {
#if HNSW_POOL_KEEP
    static std::mutex mu;
    static std::map<int, bool> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = 256ull << 20;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
#endif
}

// Reads and clears the index's error word (set by a kernel whose bounded wait
// ran out); call after the work that may set it has completed.
bool take_device_error(hnsw_index* ix) {
    if (!ix->h_err) return false;
    volatile uint32_t* w = ix->h_err;
    if (*w == 0u) return false;
    *w = 0u;
    return true;
}

// One launch over the queries of several requests of one index (the
// server's grouped dispatch); device buffers; asynchronous on s.
hnsw_status search_group(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n, int max_k,
                         int max_ef, const uint32_t* q_kef, const uint64_t* q_out, uint32_t* ids, float* dists,
                         cudaStream_t s) {
    if (max_k < 1 || max_k > kMaxK || (max_ef > max_k ? max_ef : max_k) > kMaxEf)
        return fail(HNSW_EINVAL, "search group: k or ef out of range");
    if (p.rerank && !ix->dev.vec32) return fail(HNSW_EINVAL, "search group: rerank needs the fp32 copy");
    if (p.stop_period > 65535) return fail(HNSW_EINVAL, "search group: stop_period above 65535");
    StopModel sm{};
    const StopModel* smp = nullptr;
    if (p.stop_threshold > 0.0f && p.stop_threshold < 1.0f) {
        if (!ix->d_stop) return fail(HNSW_EINVAL, "search group: stop_threshold in (0,1) needs a stop model");
        sm.stop = ix->d_stop;
        sm.logit_threshold = logf(p.stop_threshold / (1.0f - p.stop_threshold));
        sm.period = p.stop_period > 0 ? p.stop_period : 8;
        smp = &sm;
    }
    return launch_search_group(ix, p, q, n, max_k, max_ef, q_kef, q_out, ids, dists, s,
                               ix->d_work + take_work_slots(ix), smp);
}

}  // namespace hnswgb

using namespace hnswgb;

extern "C" hnsw_status hnsw_search_ex(hnsw_index* ix, const hnsw_search_params* p, const float* queries, int64_t n,
                                      uint32_t* out_ids, float* out_dists, hnsw_query_stats* stats, void* stream) {
    if (!ix || !p) return fail(HNSW_EINVAL, "hnsw_search: null index or params");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(HNSW_EINVAL, "hnsw_search: n out of range");
    if (p->k < 1 || p->k > kMaxK || p->ef < 1) return fail(HNSW_EINVAL, "hnsw_search: k or ef out of range");
    if ((p->ef > p->k ? p->ef : p->k) > kMaxEf) return fail(HNSW_EINVAL, "hnsw_search: ef' above 1024");
    if (p->visited_log2 != 0 && (p->visited_log2 < 5 || p->visited_log2 > 15))
        return fail(HNSW_EINVAL, "hnsw_search: visited_log2 outside [5,15]");
    if (p->schedule < 0 || p->schedule > 3) return fail(HNSW_EINVAL, "hnsw_search: schedule outside [0,3]");
    if (p->rerank && !ix->dev.vec32) return fail(HNSW_EINVAL, "hnsw_search: rerank needs the fp32 copy");
    if (p->stop_period > 65535) return fail(HNSW_EINVAL, "hnsw_search: stop_period above 65535");
    if (n == 0) return HNSW_OK;
    if (!queries || !out_ids || !out_dists) return fail(HNSW_EINVAL, "hnsw_search: null buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // releases this call's hold on its stream's staging buffer on every return
    struct StageLease {
        hnsw_index* ix = nullptr;
        void* stream = nullptr;
        ~StageLease() {
            if (!ix) return;
            std::lock_guard<std::mutex> lk(ix->stage_mu);
            for (auto& st : ix->stages)
                if (st.stream == stream && st.in_use > 0) --st.in_use;
        }
    } lease;
    const bool dq = is_device_ptr(queries), di = is_device_ptr(out_ids), dd = is_device_ptr(out_dists);
    const bool ds = stats ? is_device_ptr(stats) : true;
    const size_t qb = size_t(n) * ix->dev.d * 4, ob = size_t(n) * p->k * 4, sb = stats ? size_t(n) * 16 : 0;
    const float* q = queries;
    uint32_t* ids = out_ids;
    float* dists = out_dists;
    hnsw_query_stats* st = stats;
    if (!dq || !di || !dd || !ds) {
        const size_t need = al256(qb) + 2 * al256(ob) + al256(sb);
        void* sbuf = nullptr;
        {
            // this stream's staging buffer (calls on different streams may run
            // concurrently; cudaFree synchronises the device before a buffer
            // is replaced or dropped, and only idle buffers are dropped)
            std::lock_guard<std::mutex> lk(ix->stage_mu);
            hnsw_index::Stage* e = nullptr;
            for (auto& st : ix->stages)
                if (st.stream == stream) e = &st;
            if (!e) {
                if (int(ix->stages.size()) >= kMaxStages) {
                    auto it = ix->stages.begin();
                    while (it != ix->stages.end() && it->in_use > 0) ++it;
                    if (it == ix->stages.end())
                        return fail(HNSW_EINVAL, "hnsw_search: more than 16 concurrent host-memory calls on one index");
                    if (it->buf) cudaFree(it->buf);
                    ix->stages.erase(it);
                }
                ix->stages.push_back({stream, nullptr, 0, 0});
                e = &ix->stages.back();
            }
            if (e->bytes < need) {
                if (e->buf) cudaFree(e->buf);
                e->buf = nullptr;
                e->bytes = 0;
                if (cudaMalloc(&e->buf, need) != cudaSuccess) {
                    cudaGetLastError();
                    e->buf = nullptr;
                    return fail(HNSW_ENOMEM, "hnsw_search: staging buffer");
                }
                e->bytes = need;
            }
            ++e->in_use;
            sbuf = e->buf;
        }
        lease.ix = ix;
        lease.stream = stream;
        uint8_t* sp = static_cast<uint8_t*>(sbuf);
        if (!dq) {
            q = reinterpret_cast<const float*>(sp);
            cudaError_t e = cudaMemcpyAsync(sp, queries, qb, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search: H2D: ") + cudaGetErrorString(e));
        }
        sp += al256(qb);
        if (!di) ids = reinterpret_cast<uint32_t*>(sp);
        sp += al256(ob);
        if (!dd) dists = reinterpret_cast<float*>(sp);
        sp += al256(ob);
        if (!ds) st = reinterpret_cast<hnsw_query_stats*>(sp);
    }
    uint32_t* work = ix->d_work + take_work_slots(ix);
    cudaError_t e = cudaMemsetAsync(work, 0, 8, s);
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search: memset: ") + cudaGetErrorString(e));
    StopModel sm{};
    const StopModel* smp = nullptr;
    if (p->stop_threshold > 0.0f && p->stop_threshold < 1.0f) {
        if (!ix->d_stop) return fail(HNSW_EINVAL, "hnsw_search: stop_threshold in (0,1) needs a stop model");
        sm.stop = ix->d_stop;
        sm.logit_threshold = logf(p->stop_threshold / (1.0f - p->stop_threshold));
        sm.period = p->stop_period > 0 ? p->stop_period : 8;
        smp = &sm;
    }
    // schedule: 0 automatic (deferral for 33 to 2^24 queries, else one pass),
    // 1 one pass in input order, 2 two passes, 3 deferral
    const DevIndex snap = dev_snapshot(ix);  // both passes search the same version
    const bool two = snap.N > 0 && !p->check_bounds && p->schedule == 2;
    const bool defer = !two && snap.N > 0 && !p->check_bounds &&
                       (p->schedule == 3 ||
                        (p->schedule == 0 && uint64_t(n) > kDeferWarmup && uint64_t(n) <= kDeferAutoMax));
    hnsw_status r = HNSW_OK;
    if (!two && !defer) {
        r = launch_search_mode(ix, *p, q, uint32_t(n), ids, dists, st, s, work, smp, 0, nullptr, nullptr, nullptr,
                               nullptr, nullptr, &snap);
        if (r != HNSW_OK) return r;
    } else if (defer) {
        // stream-ordered scratch: control words (64 bytes, zero) and one
        // 16-byte record per query (all ones until written)
        void* scr = nullptr;
        const size_t bc = 256, br = al256(size_t(n) * 16);
        keep_pool_memory();
        e = cudaMallocAsync(&scr, bc + br, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(HNSW_ENOMEM, "hnsw_search: scheduling scratch");
        }
        uint32_t* ctl = static_cast<uint32_t*>(scr);
        uint4* rec = reinterpret_cast<uint4*>(static_cast<char*>(scr) + bc);
        if ((e = cudaMemsetAsync(ctl, 0, bc, s)) != cudaSuccess || (e = cudaMemsetAsync(rec, 0xff, br, s)) != cudaSuccess)
            r = fail(HNSW_ECUDA, std::string("hnsw_search: memset: ") + cudaGetErrorString(e));
        if (r == HNSW_OK)
            r = launch_search_mode(ix, *p, q, uint32_t(n), ids, dists, st, s, work, smp, 0, nullptr, nullptr,
                                   nullptr, nullptr, nullptr, &snap, ctl, rec);
        cudaFreeAsync(scr, s);
        if (r != HNSW_OK) return r;
    } else {
        // stream-ordered scratch: enter keys [n] u64, upper counters [n][2] u32, order [n] u32
        void* scr = nullptr;
        const size_t bk = al256(size_t(n) * 8), bc = al256(size_t(n) * 8), bo = al256(size_t(n) * 4);
        keep_pool_memory();
        e = cudaMallocAsync(&scr, bk + bc + bo, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(HNSW_ENOMEM, "hnsw_search: scheduling scratch");
        }
        uint64_t* keys = static_cast<uint64_t*>(scr);
        uint32_t* cnt = reinterpret_cast<uint32_t*>(static_cast<char*>(scr) + bk);
        uint32_t* ord = reinterpret_cast<uint32_t*>(static_cast<char*>(scr) + bk + bc);
        r = launch_search_mode(ix, *p, q, uint32_t(n), ids, dists, st, s, work, smp, 1, keys, cnt, nullptr, nullptr,
                               nullptr, &snap);
        if (r == HNSW_OK) {
            const unsigned chunks = unsigned((uint64_t(n) + kSortChunk - 1) / kSortChunk);
            order_by_descent<<<chunks, 1024, 0, s>>>(keys, uint32_t(n), ord);
            e = cudaGetLastError();
            if (e != cudaSuccess) r = fail(HNSW_ECUDA, std::string("hnsw_search: order: ") + cudaGetErrorString(e));
        }
        if (r == HNSW_OK)
            r = launch_search_mode(ix, *p, q, uint32_t(n), ids, dists, st, s, work + 1, smp, 2, keys, cnt, ord,
                                   nullptr, nullptr, &snap);
        cudaFreeAsync(scr, s);
        if (r != HNSW_OK) return r;
    }
    if (!di || !dd || !ds) {
        if ((!di && (e = cudaMemcpyAsync(out_ids, ids, ob, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
            (!dd && (e = cudaMemcpyAsync(out_dists, dists, ob, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
            (!ds && (e = cudaMemcpyAsync(stats, st, sb, cudaMemcpyDeviceToHost, s)) != cudaSuccess))
            return fail(HNSW_ECUDA, std::string("hnsw_search: D2H: ") + cudaGetErrorString(e));
    }
    if (!dq || !di || !dd || !ds) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search: ") + cudaGetErrorString(e));
        if (take_device_error(ix))
            return fail(HNSW_ETIMEOUT, "hnsw_search: a bounded device-side wait ran out (this or an earlier call)");
    }
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_debug_hold_decisions(hnsw_index* ix, int32_t on) {
    if (!ix) return fail(HNSW_EINVAL, "hnsw_debug_hold_decisions: null index");
    ix->hold_decisions.store(on ? 1 : 0);
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_search(hnsw_index* ix, const float* queries, int64_t n, int32_t k, int32_t ef,
                                   uint32_t* out_ids, float* out_dists, void* stream) {
    hnsw_search_params p{};
    p.k = k;
    p.ef = ef;
    p.stop_threshold = 2.0f;
    return hnsw_search_ex(ix, &p, queries, n, out_ids, out_dists, nullptr, stream);
}

extern "C" hnsw_status hnsw_search_trace(hnsw_index* ix, const hnsw_search_params* p, const float* queries,
                                         int64_t n, int32_t max_checks, float* feats, uint32_t* topk,
                                         float* logits, int32_t* n_checks, uint32_t* out_ids, float* out_dists,
                                         hnsw_query_stats* stats, void* stream) {
    if (!ix || !p) return fail(HNSW_EINVAL, "hnsw_search_trace: null index or params");
    if (n < 0 || n >= (int64_t(1) << 31) || max_checks < 1) return fail(HNSW_EINVAL, "hnsw_search_trace: n or max_checks");
    if (p->k < 1 || p->k > kMaxK || p->ef < 1 || (p->ef > p->k ? p->ef : p->k) > kMaxEf)
        return fail(HNSW_EINVAL, "hnsw_search_trace: k or ef out of range");
    if (p->rerank && !ix->dev.vec32) return fail(HNSW_EINVAL, "hnsw_search_trace: rerank needs the fp32 copy");
    if (n == 0) return HNSW_OK;
    const void* ptrs[] = {queries, feats, topk, n_checks, out_ids, out_dists};
    for (const void* q : ptrs)
        if (!is_device_ptr(q)) return fail(HNSW_EINVAL, "hnsw_search_trace: buffers must be device memory");
    if ((logits && !is_device_ptr(logits)) || (stats && !is_device_ptr(stats)))
        return fail(HNSW_EINVAL, "hnsw_search_trace: buffers must be device memory");
    if (p->stop_period > 65535) return fail(HNSW_EINVAL, "hnsw_search_trace: stop_period above 65535");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StopModel sm{};
    sm.stop = logits ? ix->d_stop : nullptr;
    sm.logit_threshold = 0.0f;
    sm.period = p->stop_period > 0 ? p->stop_period : 4;
    sm.tr_feat = feats;
    sm.tr_topk = topk;
    sm.tr_logit = ix->d_stop ? logits : nullptr;
    sm.tr_count = n_checks;
    sm.tr_max = max_checks;
    uint32_t* work = ix->d_work + take_work_slots(ix);
    cudaError_t e = cudaMemsetAsync(work, 0, 8, s);
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search_trace: memset: ") + cudaGetErrorString(e));
    hnsw_search_params q = *p;
    return launch_search(ix, q, queries, uint32_t(n), out_ids, out_dists, stats, s, work, &sm);
}
