// gpu_build.cu -- bulk construction of the graph with the insertions of
// layer-0 elements done on the GPU in batches (Alg. 1 with Alg. 4 as
// SELECT-NEIGHBORS; parallel construction, Section 4.1).
//
// Decomposition.  On layers >= 1, Alg. 1 only involves elements whose level
// is >= 1: a search on layer lc >= 1 visits only elements present there, and
// only they receive links there.  So the graph is built in two parts:
//  1. a seed set -- every element of level >= 1 plus the first elements of
//     the data -- inserted in id order on the host (hnsw_build), which gives
//     the upper layers and the seed's layer-0 links;
//  2. the remaining elements (all of level 0) inserted into layer 0 on the
//     GPU in batches, in id order: for a batch, every element searches the
//     graph as it stands before the batch (Alg. 5's descent through the upper
//     layers, then SEARCH-LAYER with ef = efConstruction on layer 0, run by the
//     library's search kernel), selects its M links (Alg. 4's selection), and
//     the reverse links are added per target element, which shrinks its list
//     with Alg. 4 when it exceeds Mmax0 (Alg. 1's reverse links and shrink).
// Elements of one batch do not see one another (they are linked only through
// the elements they link to); a batch is at most 1/16 of the elements already
// inserted, so each element searches a graph that already holds at least 94%
// of what precedes it.  The insertion order is a permutation of Alg. 1's (seed
// first) with batch-parallel semantics, so the graph is not the sequential
// one; it is deterministic, and on integer data equal byte for byte to the
// oracle's batch form of Alg. 1 (which batches of one element reduce to
// Alg. 1 itself).
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.hpp"
#include "index.cuh"

namespace hnswgb {
// defined in search.cu
hnsw_status launch_search_view(hnsw_index* ix, const DevIndex& view, const hnsw_search_params& p, const float* q,
                               uint32_t n, uint32_t* ids, float* dists, cudaStream_t s, uint32_t* work);
}  // namespace hnswgb

namespace {

using namespace hnswgb;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxDW = 8;      // coordinates per lane: d <= 256
constexpr int kKeep = 256;     // shrink candidates examined per chunk (ascending key order)
constexpr int kKeyBuf = 512;   // candidate keys sorted at once in a shrink
constexpr int kMaxOld = 64;    // members of a layer-0 list (Mmax0 <= 64)
constexpr int kWarps = 4;      // most warps per block of the selection kernels

__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Per-warp shared-memory layout of the selection kernels.
struct WarpSmem {
    float* Rv;       // [cap][dp] vectors of the accepted elements
    uint32_t* Rid;   // [cap]
    float* Rd;       // [cap] their distances to the base element
    uint32_t* Did;   // [cap] the first discarded candidates, in order (keepPrunedConnections)
    float* Dd;       // [cap]
    uint64_t* keys;  // [kKeyBuf] shrink candidates, (ordered distance, id)
    uint64_t* okeys; // [kMaxOld] keys of a list's current members
    uint32_t* cid;   // [kKeep] sorted shrink candidates
    float* cd;       // [kKeep]
};

__host__ __device__ inline size_t warp_smem_bytes(int cap, uint32_t dp) {
    size_t b = size_t(kKeyBuf) * 8 + size_t(kMaxOld) * 8;
    b += size_t(cap) * dp * 4 + size_t(cap) * 16;
    b += size_t(kKeep) * 8;
    return (b + 15) & ~size_t(15);
}

__device__ inline WarpSmem carve(uint8_t* base, int cap, uint32_t dp) {
    WarpSmem w;
    uint8_t* p = base;
    w.keys = reinterpret_cast<uint64_t*>(p);
    p += size_t(kKeyBuf) * 8;
    w.okeys = reinterpret_cast<uint64_t*>(p);
    p += size_t(kMaxOld) * 8;
    w.Rv = reinterpret_cast<float*>(p);
    p += size_t(cap) * dp * 4;
    w.Rid = reinterpret_cast<uint32_t*>(p);
    p += size_t(cap) * 4;
    w.Rd = reinterpret_cast<float*>(p);
    p += size_t(cap) * 4;
    w.Did = reinterpret_cast<uint32_t*>(p);
    p += size_t(cap) * 4;
    w.Dd = reinterpret_cast<float*>(p);
    p += size_t(cap) * 4;
    w.cid = reinterpret_cast<uint32_t*>(p);
    p += size_t(kKeep) * 4;
    w.cd = reinterpret_cast<float*>(p);
    return w;
}

// The warp's copy of row `id`: lane l holds coordinates l, l + 32, ...
__device__ __forceinline__ void load_vec(const float* rows, uint32_t stride, uint32_t d, uint32_t id,
                                         float (&x)[kMaxDW], int lane) {
    const float* r = rows + uint64_t(id) * stride;
#pragma unroll
    for (int k = 0; k < kMaxDW; ++k) {
        const uint32_t c = uint32_t(lane + 32 * k);
        x[k] = c < d ? __ldg(r + c) : 0.0f;
    }
}

// Distance between the warp's vector x and v (shared memory, dp floats);
// every lane returns the same value.
__device__ __forceinline__ float dist_sm(const float (&x)[kMaxDW], const float* v, uint32_t d, int metric,
                                         int lane) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxDW; ++k) {
        const uint32_t c = uint32_t(lane + 32 * k);
        if (c < d) {
            if (metric == HNSW_L2SQ) {
                const float t = x[k] - v[c];
                s = fmaf(t, t, s);
            } else {
                s = fmaf(x[k], v[c], s);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return metric == HNSW_L2SQ ? s : 1.0f - s;
}

// SELECT-NEIGHBORS, resumable: takes the candidates (cid[i], cd[i]), i < nc,
// sorted by (distance to the base, id) and following every candidate of
// earlier calls, into R (w.Rid/Rd/Rv; nr entries so far), at most cap.
// heuristic: Alg. 4's acceptance loop without extendCandidates (a candidate is
// accepted when it is closer to the base than to every element accepted
// before it, strictly); the discarded ones are recorded in order (nd so far,
// the first cap of them: keepPrunedConnections never takes more).  Otherwise Alg. 3
// (the cap nearest).
__device__ void select_more(const float* rows, uint32_t stride, uint32_t d, uint32_t dp, int metric,
                            const uint32_t* cid, const float* cd, int nc, int cap, bool heuristic,
                            const WarpSmem& w, int& nr, int& nd, int lane) {
    for (int i = 0; i < nc && nr < cap; ++i) {
        const uint32_t e = cid[i];
        const float de = cd[i];
        bool good = true;
        float x[kMaxDW];
        if (heuristic) {
            load_vec(rows, stride, d, e, x, lane);
            for (int j = 0; j < nr; ++j)
                if (!(de < dist_sm(x, w.Rv + size_t(j) * dp, d, metric, lane))) {
                    good = false;
                    break;
                }
        }
        if (!good) {
            if (nd < cap && lane == 0) {
                w.Did[nd] = e;
                w.Dd[nd] = de;
            }
            nd += nd < cap;
        }
        if (good) {
            if (heuristic) {
#pragma unroll
                for (int k = 0; k < kMaxDW; ++k) {
                    const uint32_t c = uint32_t(lane + 32 * k);
                    if (c < dp) w.Rv[size_t(nr) * dp + c] = x[k];
                }
            }
            if (lane == 0) {
                w.Rid[nr] = e;
                w.Rd[nr] = de;
            }
            ++nr;
        }
        __syncwarp();
    }
}

// Alg. 4's last step (keepPrunedConnections): the nearest discarded
// candidates fill R up to cap.
__device__ void append_pruned(const WarpSmem& w, int cap, int& nr, int nd, int lane) {
    for (int i = 0; i < nd && nr < cap; ++i) {
        if (lane == 0) {
            w.Rid[nr] = w.Did[i];
            w.Rd[nr] = w.Dd[i];
        }
        ++nr;
    }
    __syncwarp();
}

// SELECT-NEIGHBORS over one sorted candidate list; returns |R|.
__device__ int select_links(const float* rows, uint32_t stride, uint32_t d, uint32_t dp, int metric,
                            const uint32_t* cid, const float* cd, int nc, int cap, bool heuristic,
                            bool keep_pruned, const WarpSmem& w, int lane) {
    int nr = 0, nd = 0;
    select_more(rows, stride, d, dp, metric, cid, cd, nc, cap, heuristic, w, nr, nd, lane);
    __syncwarp();
    if (heuristic && keep_pruned) append_pruned(w, cap, nr, nd, lane);
    return nr;
}

__global__ void gather_rows(const float* __restrict__ rows, uint32_t stride, uint32_t d,
                            const uint32_t* __restrict__ ids, uint32_t n, float* __restrict__ out) {
    const uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= uint64_t(n) * d) return;
    const uint32_t j = uint32_t(t / d), c = uint32_t(t % d);
    out[t] = rows[uint64_t(ids[j]) * stride + c];
}

// One warp per new element b: its M links from its search result (sorted
// (dist, id), kNone-padded), written to its layer-0 row, and one reverse
// pair per link: key = the linked element, value = the new element and their
// distance (pairs of unused slots get key kNone).
__global__ void __launch_bounds__(kWarps * 32) select_forward(
    const float* __restrict__ rows, uint32_t stride, uint32_t d, uint32_t dp, int metric,
    const uint32_t* __restrict__ bids, uint32_t B, const uint32_t* __restrict__ res_id,
    const float* __restrict__ res_d, int efc, int M, int heuristic, int keep_pruned, uint32_t* __restrict__ nbr0,
    uint32_t s0, uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval, float* __restrict__ pdist) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t b = blockIdx.x * nw + wib;
    if (b >= B) return;
    const WarpSmem w = carve(smem + wib * warp_smem_bytes(M, dp), M, dp);
    const uint32_t q = bids[b];
    const uint32_t* cid = res_id + uint64_t(b) * efc;
    const float* cd = res_d + uint64_t(b) * efc;
    int nc = 0;
    for (int i = lane; i < efc; i += 32) nc += cid[i] != kNone && cid[i] != q;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nc += __shfl_xor_sync(kFull, nc, o);
    // results are sorted with the kNone padding last; q itself is never reachable
    const int nr = select_links(rows, stride, d, dp, metric, cid, cd, nc, M, heuristic != 0, keep_pruned != 0, w,
                                lane);
    for (int j = lane; j < M; j += 32) {
        const uint64_t o = uint64_t(b) * M + j;
        if (j < nr) {
            nbr0[uint64_t(q) * s0 + j] = w.Rid[j];
            pkey[o] = w.Rid[j];
            pval[o] = q;
            pdist[o] = w.Rd[j];
        } else {
            pkey[o] = kNone;
            pval[o] = kNone;
            pdist[o] = 0.0f;
        }
    }
}

__global__ void mark_segments(const uint32_t* __restrict__ skey, uint32_t n, uint32_t* __restrict__ seg,
                              uint32_t* __restrict__ nseg) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = skey[i];
    if (k != kNone && (i == 0 || skey[i - 1] != k)) seg[atomicAdd(nseg, 1u)] = i;
}

// warp bitonic sort of n keys (power of two) in shared memory, ascending
__device__ void sort_keys(uint64_t* a, int n, int lane) {
    for (int kk = 2; kk <= n; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                const int p = i ^ j;
                if (p > i) {
                    const uint64_t x = a[i], y = a[p];
                    if ((x > y) == ((i & kk) == 0)) {
                        a[i] = y;
                        a[p] = x;
                    }
                }
            }
            __syncwarp();
        }
}

__device__ __forceinline__ unsigned lanes_below(int lane) { return (1u << lane) - 1u; }

// One warp per target element e (a segment of the sorted pairs): the new
// elements linking to e join neighbourhood(e); when the list then exceeds
// Mmax0 it becomes SELECT-NEIGHBORS(e, eConn, Mmax0) over all of eConn, the
// current members and the new ones (Alg. 1's reverse links and shrink).  Alg. 4 takes eConn
// in ascending (distance, id) order and stops once Mmax0 are accepted; here
// that order is walked in chunks of kKeep: each chunk is the kKeep smallest
// keys above the previous chunk's last one (keys are distinct: ids are),
// found by one pass over the candidates that sorts kKeyBuf keys at a time.
__global__ void __launch_bounds__(kWarps * 32) link_reverse(
    const float* __restrict__ rows, uint32_t stride, uint32_t d, uint32_t dp, int metric,
    const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx, uint32_t npairs,
    const uint32_t* __restrict__ seg, const uint32_t* __restrict__ nseg, const uint32_t* __restrict__ pval,
    const float* __restrict__ pdist, uint32_t* __restrict__ nbr0, uint32_t s0, int Mmax0, int heuristic,
    int keep_pruned) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const WarpSmem w = carve(smem + wib * warp_smem_bytes(Mmax0, dp), Mmax0, dp);
    const uint32_t nsegs = *nseg;
    for (uint32_t s = blockIdx.x * nw + wib; s < nsegs; s += gridDim.x * nw) {
        const uint32_t i0 = seg[s];
        const uint32_t e = skey[i0];
        uint32_t i1 = i0 + 1;
        while (i1 < npairs && skey[i1] == e) ++i1;  // segments are short
        uint32_t* row = nbr0 + uint64_t(e) * s0;
        int n0 = 0;
        for (int j = lane; j < Mmax0; j += 32) n0 += row[j] != kNone;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(kFull, n0, o);
        const int nin = int(i1 - i0);
        if (n0 + nin <= Mmax0) {  // room: append in insertion order
            for (int t = lane; t < nin; t += 32) row[n0 + t] = pval[sidx[i0 + t]];
            __syncwarp();
            continue;
        }
        // keys of the current members (their distances to e recomputed)
        float x[kMaxDW];
        load_vec(rows, stride, d, e, x, lane);
        for (int j = 0; j < n0; ++j) {
            const uint32_t c = row[j];
            float y[kMaxDW];
            load_vec(rows, stride, d, c, y, lane);
            float sacc = 0.0f;
#pragma unroll
            for (int k = 0; k < kMaxDW; ++k) {
                if (uint32_t(lane + 32 * k) < d) {
                    if (metric == HNSW_L2SQ) {
                        const float t = x[k] - y[k];
                        sacc = fmaf(t, t, sacc);
                    } else {
                        sacc = fmaf(x[k], y[k], sacc);
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(kFull, sacc, o);
            const float dc = metric == HNSW_L2SQ ? sacc : 1.0f - sacc;
            if (lane == 0) w.okeys[j] = (uint64_t(f2ord(dc)) << 32) | c;
        }
        __syncwarp();
        const int total = n0 + nin;
        int nr = 0, nd = 0, seen = 0;
        uint64_t last = 0;  // keys of the next chunk are above it (all keys in the first chunk)
        bool first = true;
        for (;;) {
            // the kKeep smallest candidate keys above `last`
            int nk = 0;
            for (int b0 = 0; b0 < total; b0 += 32) {
                const int j = b0 + lane;
                uint64_t k = ~0ull;
                if (j < n0) {
                    k = w.okeys[j];
                } else if (j < total) {
                    const uint32_t pi = sidx[i0 + uint32_t(j - n0)];
                    k = (uint64_t(f2ord(pdist[pi])) << 32) | pval[pi];
                }
                const bool ok = j < total && (first || k > last);
                const unsigned m = __ballot_sync(kFull, ok);
                if (ok) w.keys[nk + __popc(m & lanes_below(lane))] = k;
                nk += __popc(m);
                if (nk > kKeyBuf - 32) {  // full: keep the kKeep smallest
                    for (int u = nk + lane; u < kKeyBuf; u += 32) w.keys[u] = ~0ull;
                    __syncwarp();
                    sort_keys(w.keys, kKeyBuf, lane);
                    nk = kKeep;
                }
                __syncwarp();
            }
            int n2 = 32;
            while (n2 < nk) n2 <<= 1;
            for (int u = nk + lane; u < n2; u += 32) w.keys[u] = ~0ull;
            __syncwarp();
            sort_keys(w.keys, n2, lane);
            nk = min(nk, kKeep);
            if (nk == 0) break;
            for (int u = lane; u < nk; u += 32) {
                w.cid[u] = uint32_t(w.keys[u] & 0xffffffffu);
                w.cd[u] = ord2f(uint32_t(w.keys[u] >> 32));
            }
            __syncwarp();
            select_more(rows, stride, d, dp, metric, w.cid, w.cd, nk, Mmax0, heuristic != 0, w, nr, nd, lane);
            __syncwarp();
            seen += nk;
            if (nr >= Mmax0 || seen >= total) break;
            last = w.keys[nk - 1];
            first = false;
            __syncwarp();
        }
        if (heuristic && keep_pruned) append_pruned(w, Mmax0, nr, nd, lane);
        for (int j = lane; j < Mmax0; j += 32) row[j] = j < nr ? w.Rid[j] : kNone;
        __syncwarp();
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

hnsw_status cuda_fail(cudaError_t e, const char* what) {
    return fail(HNSW_ECUDA, std::string("hnsw_build_gpu: ") + what + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace hnswgb {

// Inserts the elements `ids` (in order, all of level 0 or already linked on
// their upper layers) into layer 0 of `view` in batches of at most 1/16 of
// the elements inserted so far (`inserted` before the first batch), on
// stream s.  The view's rows must be fp32 (storage F32) and its nbr0 is the
// adjacency written; asynchronous, buffers freed at return (cudaFree waits
// for the stream's work).
hnsw_status insert_layer0(hnsw_index* ix, const DevIndex& view, const std::vector<uint32_t>& ids, uint64_t inserted,
                          int metric, int M, int Mmax0, int efc, int heuristic, int keep_pruned, cudaStream_t s) {
    if (ids.empty()) return HNSW_OK;
    const DevIndex& D = view;
    const float* drows = reinterpret_cast<const float*>(D.vec);
    const uint32_t d = D.d, stride = D.row_chunks * 4, dp = D.row_chunks * 4, s0 = D.s0;
    uint32_t* nbr0 = const_cast<uint32_t*>(D.nbr0);
    const uint32_t Bmax = uint32_t(std::min<uint64_t>(32768, std::max<uint64_t>(64, ids.size())));
    DevBuf dbid, dq, rid, rdist, pkey, pval, pdist, skey, sidx, idx, seg, nseg, work, tmp;
    size_t tmp_bytes = 0;
    const uint32_t npair_max = Bmax * uint32_t(M);
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, static_cast<uint32_t*>(nullptr),
                                    static_cast<uint32_t*>(nullptr), static_cast<uint32_t*>(nullptr),
                                    static_cast<uint32_t*>(nullptr), int(npair_max), 0, 32, s);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](DevBuf& x, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(&x.p, bytes ? bytes : 16);
    };
    alloc(dbid, size_t(ids.size()) * 4);
    alloc(dq, size_t(Bmax) * d * 4);
    alloc(rid, size_t(Bmax) * efc * 4);
    alloc(rdist, size_t(Bmax) * efc * 4);
    alloc(pkey, size_t(npair_max) * 4);
    alloc(pval, size_t(npair_max) * 4);
    alloc(pdist, size_t(npair_max) * 4);
    alloc(skey, size_t(npair_max) * 4);
    alloc(sidx, size_t(npair_max) * 4);
    alloc(idx, size_t(npair_max) * 4);
    alloc(seg, size_t(npair_max) * 4);
    alloc(nseg, 16);
    alloc(work, 16);
    alloc(tmp, tmp_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HNSW_ENOMEM, "layer-0 insertion: device buffers");
    }
    std::vector<uint32_t> iota(npair_max);
    for (uint32_t i = 0; i < npair_max; ++i) iota[i] = i;
    // pageable sources: the copies complete before cudaMemcpyAsync returns
    if ((e = cudaMemcpyAsync(idx.p, iota.data(), size_t(npair_max) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dbid.p, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "copy");
    // warps per block: as many (up to kWarps) as the shared memory allows
    auto warps_for = [](size_t per_warp) {
        int nw = kWarps;
        while (nw > 1 && size_t(nw) * per_warp > 227 * 1024) --nw;
        return nw;
    };
    const int fw_w = warps_for(warp_smem_bytes(M, dp)), rv_w = warps_for(warp_smem_bytes(Mmax0, dp));
    const size_t fw_smem = size_t(fw_w) * warp_smem_bytes(M, dp);
    const size_t rv_smem = size_t(rv_w) * warp_smem_bytes(Mmax0, dp);
    if (fw_smem > 227 * 1024 || rv_smem > 227 * 1024)
        return fail(HNSW_EINVAL, "layer-0 insertion: dimension too large for the selection kernels");
    {
        hnsw_status r = raise_smem_limit(reinterpret_cast<const void*>(select_forward), fw_smem, "layer-0 insertion");
        if (r == HNSW_OK)
            r = raise_smem_limit(reinterpret_cast<const void*>(link_reverse), rv_smem, "layer-0 insertion");
        if (r != HNSW_OK) return r;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    hnsw_search_params sp{};
    sp.k = efc;
    sp.ef = efc;
    hnsw_status st = HNSW_OK;
    for (size_t pos = 0; pos < ids.size();) {
        const uint32_t B = uint32_t(std::min<uint64_t>(
            {uint64_t(Bmax), uint64_t(ids.size() - pos), std::max<uint64_t>(64, inserted / 16)}));
        const uint32_t* bids = static_cast<const uint32_t*>(dbid.p) + pos;
        const uint64_t nq = uint64_t(B) * d;
        gather_rows<<<unsigned((nq + 255) / 256), 256, 0, s>>>(drows, stride, d, bids, B, static_cast<float*>(dq.p));
        if ((e = cudaMemsetAsync(work.p, 0, 8, s)) != cudaSuccess) break;
        st = launch_search_view(ix, view, sp, static_cast<const float*>(dq.p), B, static_cast<uint32_t*>(rid.p),
                                static_cast<float*>(rdist.p), s, static_cast<uint32_t*>(work.p));
        if (st != HNSW_OK) break;
        select_forward<<<(B + fw_w - 1) / fw_w, fw_w * 32, fw_smem, s>>>(
            drows, stride, d, dp, metric, bids, B, static_cast<const uint32_t*>(rid.p),
            static_cast<const float*>(rdist.p), efc, M, heuristic, keep_pruned, nbr0, s0,
            static_cast<uint32_t*>(pkey.p), static_cast<uint32_t*>(pval.p), static_cast<float*>(pdist.p));
        const uint32_t np = B * uint32_t(M);
        size_t tb = tmp_bytes;
        if ((e = cub::DeviceRadixSort::SortPairs(tmp.p, tb, static_cast<const uint32_t*>(pkey.p),
                                                 static_cast<uint32_t*>(skey.p), static_cast<const uint32_t*>(idx.p),
                                                 static_cast<uint32_t*>(sidx.p), int(np), 0, 32, s)) != cudaSuccess)
            break;
        if ((e = cudaMemsetAsync(nseg.p, 0, 4, s)) != cudaSuccess) break;
        mark_segments<<<(np + 255) / 256, 256, 0, s>>>(static_cast<const uint32_t*>(skey.p), np,
                                                      static_cast<uint32_t*>(seg.p), static_cast<uint32_t*>(nseg.p));
        link_reverse<<<unsigned(sms) * 4, rv_w * 32, rv_smem, s>>>(
            drows, stride, d, dp, metric, static_cast<const uint32_t*>(skey.p), static_cast<const uint32_t*>(sidx.p),
            np, static_cast<const uint32_t*>(seg.p), static_cast<const uint32_t*>(nseg.p),
            static_cast<const uint32_t*>(pval.p), static_cast<const float*>(pdist.p), nbr0, s0, Mmax0, heuristic,
            keep_pruned);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        pos += B;
        inserted += B;
    }
    if (st != HNSW_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batch");
    return HNSW_OK;
}

}  // namespace hnswgb

extern "C" hnsw_status hnsw_build_gpu(const float* data, uint64_t N, uint32_t d, hnsw_metric metric,
                                      const hnsw_build_params* params, const double* level_u, void* stream,
                                      void** out_blob, uint64_t* out_bytes) {
    if (!params || !out_blob || !out_bytes || (N > 0 && (!data || !level_u)))
        return fail(HNSW_EINVAL, "hnsw_build_gpu: null pointer");
    const hnsw_build_params& p = *params;
    if (d == 0 || d > 32u * kMaxDW || N >= (1ull << 31) || p.M == 0 || p.M > p.Mmax || p.M > p.Mmax0 ||
        p.Mmax0 > 64 || p.Mmax > 64 || !(p.mL > 0) || p.ef_construction == 0 || p.ef_construction > 1024 ||
        p.extend_candidates || (metric != HNSW_L2SQ && metric != HNSW_COSINE))
        return fail(HNSW_EINVAL, "hnsw_build_gpu: invalid parameters (d <= 256, efConstruction <= 1024, "
                                 "no extendCandidates)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // levels (the level draw of Alg. 1) and the seed: the first elements and every
    // element of level >= 1, in id order
    std::vector<uint8_t> level(N);
    uint64_t rows = 0;
    for (uint64_t i = 0; i < N; ++i) {
        const double u = level_u[i];
        if (!(u > 0.0 && u <= 1.0)) return fail(HNSW_EINVAL, "hnsw_build_gpu: level_u outside (0,1]");
        const double lv = std::floor(-std::log(u) * p.mL);
        if (lv > 255) return fail(HNSW_EINVAL, "hnsw_build_gpu: level above 255");
        level[i] = uint8_t(lv);
        rows += level[i];
    }
    const uint64_t n_first = std::min<uint64_t>(N, 4096);
    std::vector<uint32_t> seed, rest;
    for (uint64_t i = 0; i < N; ++i) (i < n_first || level[i] > 0 ? seed : rest).push_back(uint32_t(i));
    if (rest.empty()) return hnsw_build(data, N, d, metric, params, level_u, out_blob, out_bytes);
    // 1. the seed on the host
    std::vector<float> sdata(seed.size() * size_t(d));
    std::vector<double> su(seed.size());
    for (size_t j = 0; j < seed.size(); ++j) {
        std::memcpy(&sdata[j * d], data + uint64_t(seed[j]) * d, d * 4ull);
        su[j] = level_u[seed[j]];
    }
    void* sblob = nullptr;
    uint64_t sbytes = 0;
    hnsw_status st = hnsw_build(sdata.data(), seed.size(), d, metric, params, su.data(), &sblob, &sbytes);
    if (st != HNSW_OK) return st;
    BlobHeader sh{};
    read_header(static_cast<const uint8_t*>(sblob), sbytes, sh);
    const BlobLayout sl = BlobLayout::of(seed.size(), d, p.Mmax0, p.Mmax, sh.n_upper_rows);
    // the full blob: all vectors and levels, the seed's links in original ids
    const BlobLayout lay = BlobLayout::of(N, d, p.Mmax0, p.Mmax, rows);
    uint8_t* b = static_cast<uint8_t*>(std::calloc(lay.total, 1));
    if (!b) {
        hnsw_free_blob(sblob);
        return fail(HNSW_ENOMEM, "hnsw_build_gpu: blob allocation failed");
    }
    const uint8_t* sb = static_cast<const uint8_t*>(sblob);
    std::memcpy(b + lay.data, data, N * d * 4ull);
    std::memcpy(b + lay.level, level.data(), N);
    std::memset(b + lay.nbr0, 0xFF, N * p.Mmax0 * 4ull);  // every slot kNone
    auto map = [&](uint32_t v) { return v == kNone ? kNone : seed[v]; };
    for (size_t j = 0; j < seed.size(); ++j)
        for (uint32_t c = 0; c < p.Mmax0; ++c)
            wr<uint32_t>(b + lay.nbr0 + (uint64_t(seed[j]) * p.Mmax0 + c) * 4,
                         map(rd<uint32_t>(sb + sl.nbr0 + (uint64_t(j) * p.Mmax0 + c) * 4)));
    // upper rows are element-major; the seed holds every element of level >= 1
    // in id order, so its rows are already in the full graph's order
    for (uint64_t r = 0; r < sh.n_upper_rows * p.Mmax; ++r)
        wr<uint32_t>(b + lay.nbrU + r * 4, map(rd<uint32_t>(sb + sl.nbrU + r * 4)));
    BlobHeader h = sh;
    h.N = N;
    h.ep = map(sh.ep);
    h.n_upper_rows = rows;
    hnsw_free_blob(sblob);
    auto finish_header = [&]() {
        h.checksum = fnv1a64(b + 128, lay.total - 128);
        write_header(b, h);
    };
    // 2. layer-0 insertion of the rest on the GPU (the intermediate blob is
    // uploaded without its checksum or per-list checks: written just above)
    h.checksum = 0;
    write_header(b, h);
    hnsw_index* ix = nullptr;
    st = upload_index(b, lay.total, HNSW_F32, 0, stream, &ix, true);
    if (st != HNSW_OK) {
        std::free(b);
        return st;
    }
    struct IxGuard {
        hnsw_index* ix;
        ~IxGuard() { hnsw_free_index(ix); }
    } ixg{ix};
    st = insert_layer0(ix, ix->dev, rest, seed.size(), int(metric), int(p.M), int(p.Mmax0),
                       int(p.ef_construction), p.heuristic, p.keep_pruned, s);
    if (st != HNSW_OK) {
        std::free(b);
        return st;
    }
    uint32_t* nbr0 = static_cast<uint32_t*>(ix->d_nbr0);
    const uint32_t s0 = ix->dev.s0;
    cudaError_t e = cudaSuccess;
    // 3. the final layer 0 back into the blob
    std::vector<uint32_t> h0(N * size_t(s0));
    if ((e = cudaMemcpyAsync(h0.data(), nbr0, h0.size() * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        std::free(b);
        return cuda_fail(e, "layer 0 copy");
    }
    for (uint64_t i = 0; i < N; ++i)
        for (uint32_t c = 0; c < p.Mmax0; ++c) wr<uint32_t>(b + lay.nbr0 + (i * p.Mmax0 + c) * 4, h0[i * s0 + c]);
    finish_header();
    *out_blob = b;
    *out_bytes = lay.total;
    return HNSW_OK;
}

// ---------------------------------------------------------------------------
// Incremental insertion into a resident index
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ uint64_t mkkey(float d, uint32_t id) { return (uint64_t(f2ord(d)) << 32) | id; }
__device__ __forceinline__ uint32_t kid(uint64_t k) { return uint32_t(k & 0xffffffffu); }
__device__ __forceinline__ float kdist(uint64_t k) { return ord2f(uint32_t(k >> 32)); }

// distance from the warp's vector x to row `id` (every lane returns it)
__device__ __forceinline__ float dist_id(const float (&x)[kMaxDW], const float* rows, uint32_t stride, uint32_t d,
                                         uint32_t id, int metric, int lane) {
    float y[kMaxDW];
    load_vec(rows, stride, d, id, y, lane);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxDW; ++k) {
        if (uint32_t(lane + 32 * k) < d) {
            if (metric == HNSW_L2SQ) {
                const float t = x[k] - y[k];
                s = fmaf(t, t, s);
            } else {
                s = fmaf(x[k], y[k], s);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return metric == HNSW_L2SQ ? s : 1.0f - s;
}

// distance from the vector a (shared memory, 16-byte aligned, d floats) to
// row `id`, computed by one lane
__device__ __forceinline__ float dist_lane(const float* a, const float* rows, uint32_t stride, uint32_t d,
                                           uint32_t id, int metric) {
    const float* r = rows + uint64_t(id) * stride;
    float s = 0.0f;
    uint32_t c = 0;
    for (; c + 4 <= d; c += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(r + c));
        const float4 q = *reinterpret_cast<const float4*>(a + c);
        if (metric == HNSW_L2SQ) {
            const float t0 = q.x - v.x, t1 = q.y - v.y, t2 = q.z - v.z, t3 = q.w - v.w;
            s = fmaf(t0, t0, s);
            s = fmaf(t1, t1, s);
            s = fmaf(t2, t2, s);
            s = fmaf(t3, t3, s);
        } else {
            s = fmaf(q.x, v.x, s);
            s = fmaf(q.y, v.y, s);
            s = fmaf(q.z, v.z, s);
            s = fmaf(q.w, v.w, s);
        }
    }
    for (; c < d; ++c) {
        const float v = __ldg(r + c);
        if (metric == HNSW_L2SQ) {
            const float t = a[c] - v;
            s = fmaf(t, t, s);
        } else {
            s = fmaf(a[c], v, s);
        }
    }
    return metric == HNSW_L2SQ ? s : 1.0f - s;
}

// keys of the single-list search: (ordered distance, id, expanded bit)
__device__ __forceinline__ uint64_t lkey(uint64_t k) { return (k & 0xffffffff00000000ull) | (uint64_t(kid(k)) << 1); }
__device__ __forceinline__ uint32_t lid(uint64_t k) { return uint32_t(k >> 1) & 0x7fffffffu; }

// ascending bitonic sort of one key per lane across the warp
__device__ __forceinline__ uint64_t warp_sort_u64(uint64_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint64_t o = __shfl_xor_sync(kFull, v, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            v = (lower == up) ? (v < o ? v : o) : (v > o ? v : o);
        }
    return v;
}

struct UpperArgs {
    DevIndex v;                 // fp32 view; nbrU / upoff of the version being written
    const uint32_t* ids;        // new elements of level >= 1, in id order
    const uint8_t* lv;          // their levels
    uint32_t n;
    int efc, M, Mmax, heuristic, keep_pruned;
    uint32_t* visited;          // [capacity] epoch tags
    int* state;                 // {enter point, top level}
};

// the W buffer: a power of two >= ef (>= 32) for the final bitonic sort
__host__ __device__ inline int wcap_of(int efc) {
    int n = 32;
    while (n < efc) n <<= 1;
    return n;
}

__device__ __forceinline__ uint32_t* upper_row(const UpperArgs& a, uint32_t e, int lc) {
    return const_cast<uint32_t*>(a.v.nbrU) + (uint64_t(a.v.upoff[e]) + uint32_t(lc - 1)) * a.v.sU;
}

// Alg. 1's descent and layer insertion on layers >= 1 for each new element in turn (one warp):
// greedy descent above the element's level, then on each of its layers
// SEARCH-LAYER with efConstruction, SELECT-NEIGHBORS for its list and the
// reverse links, shrunk with the same selection beyond Mmax; a new top level
// makes the element the enter point (as in Alg. 1).
__global__ void __launch_bounds__(32) insert_upper(const UpperArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const DevIndex& V = a.v;
    const float* rows = reinterpret_cast<const float*>(V.vec);
    const uint32_t d = V.d, stride = V.row_chunks * 4, dp = V.row_chunks * 4;
    const WarpSmem w = carve(smem, a.Mmax, dp);
    uint8_t* p = smem + warp_smem_bytes(a.Mmax, dp);
    float* qs = reinterpret_cast<float*>(p);  // [dp] the element being inserted
    p += size_t(dp) * 4;
    float* rs = reinterpret_cast<float*>(p);  // [dp] a reverse-link target
    p += size_t(dp) * 4;
    uint64_t* Wk = reinterpret_cast<uint64_t*>(p);  // [pow2 >= efc] W: a max-heap, then sorted
    p += size_t(wcap_of(a.efc)) * 8;
    uint64_t* Ek = reinterpret_cast<uint64_t*>(p);  // [efc] enter points of the next layer
    p += size_t(a.efc) * 8;
    uint32_t* Wid = reinterpret_cast<uint32_t*>(p);  // [efc] decoded W
    p += size_t(a.efc) * 4;
    float* Wd = reinterpret_cast<float*>(p);  // [efc]
    p += size_t(a.efc) * 4;
    uint32_t* qR = reinterpret_cast<uint32_t*>(p);  // [64]
    p += 64 * 4;
    int* LB = reinterpret_cast<int*>(p);  // [32] insertion points of a merge
    p += 32 * 4;
    uint64_t* W2 = reinterpret_cast<uint64_t*>(p);  // [pow2 >= efc] merge target
    uint32_t epoch = 0;
    for (uint32_t u = 0; u < a.n; ++u) {
        const uint32_t q = a.ids[u];
        const int l = a.lv[u];
        __syncwarp();
        const uint32_t ep = uint32_t(((volatile int*)a.state)[0]);
        const int L = ((volatile int*)a.state)[1];
        float xq[kMaxDW];
        load_vec(rows, stride, d, q, xq, lane);
#pragma unroll
        for (int k = 0; k < kMaxDW; ++k)
            if (uint32_t(lane + 32 * k) < dp) qs[lane + 32 * k] = xq[k];
        __syncwarp();
        uint32_t cur = ep;
        float dcur = dist_id(xq, rows, stride, d, ep, V.metric, lane);
        for (int lc = L; lc > l; --lc) {  // descent above the level, ef = 1 (steepest descent)
            for (;;) {
                // every neighbour's distance at once (a lane each), then the
                // smallest key over the warp
                const uint32_t* row = upper_row(a, cur, lc);
                uint64_t best = mkkey(dcur, cur);
                for (uint32_t j0 = 0; j0 < V.Mmax; j0 += 32) {
                    const uint32_t j = j0 + lane;
                    const uint32_t e = j < V.Mmax ? row[j] : kNone;
                    if (e != kNone) {
                        const uint64_t k = mkkey(dist_lane(qs, rows, stride, d, e, V.metric), e);
                        best = k < best ? k : best;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t other = __shfl_xor_sync(kFull, best, o);
                    best = other < best ? other : best;
                }
                if (kid(best) == cur) break;
                cur = kid(best);
                dcur = kdist(best);
            }
        }
        int n_ep = 1;
        if (lane == 0) Ek[0] = mkkey(dcur, cur);
        __syncwarp();
        for (int lc = l < L ? l : L; lc >= 1; --lc) {
            // SEARCH-LAYER(q, ep, efc, lc), in the single-list
            // form: W sorted by key with an 'expanded' bit below the id; its
            // unexpanded entries are C (an element that left W can never be
            // expanded: it lies beyond W's furthest when reached), the next
            // to expand is the first unexpanded; an expansion's new
            // neighbours are merged at once (taking them one at a time keeps
            // W = the ef smallest of W and the ones taken, in any order)
            ++epoch;
            uint64_t* Wa = Wk;
            uint64_t* Wb = W2;
            int wn = n_ep;  // n_ep <= efc (the previous layer's W)
            for (int i = lane; i < wn; i += 32) {
                const uint64_t k = Ek[i];
                a.visited[kid(k)] = epoch;
                Wa[i] = lkey(k);
            }
            __syncwarp();
            int scan = 0;
            for (;;) {
                int pos = -1;
                for (int s0 = scan; s0 < wn; s0 += 32) {
                    const int i = s0 + lane;
                    const bool un = i < wn && !(Wa[i] & 1ull);
                    const unsigned m = __ballot_sync(kFull, un);
                    if (m) {
                        pos = s0 + __ffs(m) - 1;
                        break;
                    }
                }
                if (pos < 0) break;  // every entry of W expanded (Alg. 2 stops)
                const uint64_t c = Wa[pos];
                __syncwarp();
                if (lane == 0) Wa[pos] = c | 1ull;
                scan = pos + 1;
                const uint32_t* row = upper_row(a, lid(c), lc);
                for (uint32_t j0 = 0; j0 < V.Mmax; j0 += 32) {
                    // each neighbour's visited test and distance at once, a lane each
                    const uint32_t j = j0 + lane;
                    const uint32_t e = j < V.Mmax ? row[j] : kNone;
                    const bool fresh = e != kNone && a.visited[e] != epoch;
                    uint64_t k = ~0ull;
                    if (fresh) {
                        a.visited[e] = epoch;
                        k = (uint64_t(f2ord(dist_lane(qs, rows, stride, d, e, V.metric))) << 32) | (uint64_t(e) << 1);
                    }
                    // admission: with W full only keys below its furthest enter
                    const bool pass = fresh && (wn < a.efc || k < (Wa[wn - 1] & ~1ull));
                    const unsigned m = __ballot_sync(kFull, pass);
                    if (!m) continue;
                    const int nb = __popc(m);
                    const uint64_t key = warp_sort_u64(pass ? k : ~0ull, lane);  // lane j: j-th smallest
                    int lb = 0;
                    if (lane < nb) {  // old entries below the key
                        int lo = 0, hi = wn;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if ((Wa[mid] & ~1ull) < key)
                                lo = mid + 1;
                            else
                                hi = mid;
                        }
                        lb = lo;
                        LB[lane] = lb;
                    }
                    __syncwarp();
                    const int nn = wn + nb < a.efc ? wn + nb : a.efc;
                    for (int i = lane; i < wn; i += 32) {  // old entry i moves up by the new keys below it
                        int lo = 0, hi = nb;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (LB[mid] <= i)
                                lo = mid + 1;
                            else
                                hi = mid;
                        }
                        if (i + lo < nn) Wb[i + lo] = Wa[i];
                    }
                    if (lane < nb && lb + lane < nn) Wb[lb + lane] = key;
                    __syncwarp();
                    if (LB[0] < scan) scan = LB[0];  // the smallest new key may precede the scan
                    uint64_t* t = Wa;
                    Wa = Wb;
                    Wb = t;
                    wn = nn;
                    __syncwarp();
                }
            }
            for (int i = lane; i < wn; i += 32) {
                const uint64_t k = Wa[i];
                Wid[i] = lid(k);
                Wd[i] = kdist(k);
                Ek[i] = (k & 0xffffffff00000000ull) | lid(k);
            }
            n_ep = int(wn);
            __syncwarp();
            // neighbourhood(q) at lc: SELECT-NEIGHBORS(q, W, M)
            const int nr = select_links(rows, stride, d, dp, V.metric, Wid, Wd, int(wn), a.M, a.heuristic != 0,
                                        a.keep_pruned != 0, w, lane);
            for (int j = lane; j < nr; j += 32) qR[j] = w.Rid[j];
            __syncwarp();
            uint32_t* rq = upper_row(a, q, lc);
            for (uint32_t j = lane; j < V.Mmax; j += 32) rq[j] = int(j) < nr ? qR[j] : kNone;
            __syncwarp();
            // reverse links and their shrink
            for (int t = 0; t < nr; ++t) {
                const uint32_t r = qR[t];
                uint32_t* rr = upper_row(a, r, lc);
                int n0 = 0;
                for (uint32_t j = lane; j < V.Mmax; j += 32) n0 += rr[j] != kNone;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) n0 += __shfl_xor_sync(kFull, n0, o);
                if (n0 < int(V.Mmax)) {
                    if (lane == 0) rr[n0] = q;
                    __syncwarp();
                    continue;
                }
                float xr[kMaxDW];
                load_vec(rows, stride, d, r, xr, lane);
#pragma unroll
                for (int k = 0; k < kMaxDW; ++k)
                    if (uint32_t(lane + 32 * k) < dp) rs[lane + 32 * k] = xr[k];
                __syncwarp();
                for (int j = lane; j <= n0; j += 32) {  // the members and q, a lane each
                    const uint32_t c2 = j < n0 ? rr[j] : q;
                    w.keys[j] = mkkey(dist_lane(rs, rows, stride, d, c2, V.metric), c2);
                }
                int n2 = 32;
                while (n2 < n0 + 1) n2 <<= 1;
                for (int j = n0 + 1 + lane; j < n2; j += 32) w.keys[j] = ~0ull;
                __syncwarp();
                sort_keys(w.keys, n2, lane);
                for (int j = lane; j <= n0; j += 32) {
                    w.cid[j] = kid(w.keys[j]);
                    w.cd[j] = kdist(w.keys[j]);
                }
                __syncwarp();
                const int nr2 = select_links(rows, stride, d, dp, V.metric, w.cid, w.cd, n0 + 1, int(V.Mmax),
                                             a.heuristic != 0, a.keep_pruned != 0, w, lane);
                for (uint32_t j = lane; j < V.Mmax; j += 32) rr[j] = int(j) < nr2 ? w.Rid[j] : kNone;
                __syncwarp();
            }
        }
        if (l > L && lane == 0) {  // a new top level moves the enter point
            a.state[0] = int(q);
            a.state[1] = l;
        }
        __threadfence_block();
        __syncwarp();
    }
}

size_t upper_smem_bytes(int Mmax, uint32_t dp, int efc) {
    return warp_smem_bytes(Mmax, dp) + size_t(dp) * 8 + size_t(wcap_of(efc)) * 8 + size_t(efc) * 8 +
           size_t(efc) * 8 + 64 * 4 + 32 * 4 + size_t(wcap_of(efc)) * 8;
}

hnsw_status ins_fail(hnsw_status st, const std::string& m) { return fail(st, "hnsw_insert: " + m); }

}  // namespace

extern "C" hnsw_status hnsw_reserve(hnsw_index* ix, uint64_t capacity, void* stream) {
    if (!ix) return fail(HNSW_EINVAL, "hnsw_reserve: null index");
    std::lock_guard<std::mutex> lk(ix->insert_mu);
    const DevIndex D = dev_snapshot(ix);
    if (capacity < D.N || capacity >= (1ull << 31)) return fail(HNSW_EINVAL, "hnsw_reserve: capacity out of range");
    if (capacity <= ix->capacity && ix->v_nbr0[1 - ix->active]) return HNSW_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_reserve: ") + cudaGetErrorString(e));
    const hnsw_index_info& I = ix->info;
    const uint64_t N = D.N;
    const uint32_t d_pad32 = D.row_chunks32 * 4;
    const uint64_t Mm1 = ix->build_M > 1 ? ix->build_M - 1 : 1;
    const uint64_t ucap = ix->upper_rows + (capacity - N) * 2 / Mm1 + 1024;
    const bool alias32 = ix->d_vec32 && ix->d_vec32 == ix->d_vec;
    std::vector<void*> fresh;
    auto get = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e == cudaSuccess) fresh.push_back(p);
        return p;
    };
    void* vec = get(capacity * I.row_bytes);
    void* scale = ix->d_scale ? get(capacity * 4) : nullptr;
    void* vec32 = ix->d_vec32 && !alias32 ? get(capacity * d_pad32 * 4ull) : nullptr;
    void* n0[2] = {get(capacity * D.s0 * 4ull), get(capacity * D.s0 * 4ull)};
    void* uo[2] = {get(capacity * 4), get(capacity * 4)};
    void* nu[2] = {get(ucap * D.sU * 4ull), get(ucap * D.sU * 4ull)};
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (void* p : fresh) cudaFree(p);
        return fail(HNSW_ENOMEM, "hnsw_reserve: device memory");
    }
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
    };
    auto ff = [&](void* dst, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemsetAsync(dst, 0xFF, bytes, s);
    };
    cp(vec, ix->d_vec, N * I.row_bytes);
    if (scale) cp(scale, ix->d_scale, N * 4);
    if (vec32) cp(vec32, ix->d_vec32, N * d_pad32 * 4ull);
    for (int v = 0; v < 2; ++v) {
        ff(n0[v], capacity * D.s0 * 4ull);
        ff(uo[v], capacity * 4);
        ff(nu[v], ucap * D.sU * 4ull);
    }
    cp(n0[0], ix->dev.nbr0, N * D.s0 * 4ull);
    cp(uo[0], ix->dev.upoff, N * 4);
    cp(nu[0], ix->dev.nbrU, ix->upper_rows * D.sU * 4ull);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        for (void* p : fresh) cudaFree(p);
        return fail(HNSW_ECUDA, std::string("hnsw_reserve: copy: ") + cudaGetErrorString(e));
    }
    // release the old arrays (both adjacency versions)
    std::vector<void*> old = {ix->d_vec, ix->d_scale};
    if (ix->d_vec32 && !alias32) old.push_back(ix->d_vec32);
    for (int v = 0; v < 2; ++v)
        for (void* p : {ix->v_nbr0[v], ix->v_upoff[v], ix->v_nbrU[v]}) old.push_back(p);
    for (void* p : old)
        if (p) cudaFree(p);
    ix->d_vec = vec;
    ix->d_scale = scale;
    ix->d_vec32 = alias32 ? vec : vec32;
    for (int v = 0; v < 2; ++v) {
        ix->v_nbr0[v] = n0[v];
        ix->v_upoff[v] = uo[v];
        ix->v_nbrU[v] = nu[v];
    }
    ix->active = 0;
    ix->d_nbr0 = n0[0];
    ix->d_upoff = uo[0];
    ix->d_nbrU = nu[0];
    ix->capacity = capacity;
    ix->upper_capacity = ucap;
    {
        std::lock_guard<std::mutex> dl(ix->dev_mu);
        ix->dev.vec = static_cast<const uint4*>(vec);
        ix->dev.scale = static_cast<const float*>(scale);
        ix->dev.vec32 = static_cast<const uint4*>(ix->d_vec32);
        ix->dev.nbr0 = static_cast<const uint32_t*>(n0[0]);
        ix->dev.upoff = static_cast<const uint32_t*>(uo[0]);
        ix->dev.urows = uint32_t(ucap);
        ix->dev.nbrU = static_cast<const uint32_t*>(nu[0]);
    }
    std::lock_guard<std::mutex> il(ix->dev_mu);
    ix->info.device_bytes = capacity * I.row_bytes + (scale ? capacity * 4 : 0) + (vec32 ? capacity * d_pad32 * 4ull : 0) +
                            2 * (capacity * D.s0 * 4ull + capacity * 4 + ucap * D.sU * 4ull) + kWorkSlots * 4;
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_insert(hnsw_index* ix, const float* data, uint64_t n, const double* level_u, void* stream) {
    if (!ix) return ins_fail(HNSW_EINVAL, "null index");
    if (n == 0) return HNSW_OK;
    if (!data || !level_u) return ins_fail(HNSW_EINVAL, "null data or level_u");
    std::lock_guard<std::mutex> lk(ix->insert_mu);
    DevIndex V = dev_snapshot(ix);
    const uint64_t N0 = V.N;
    if (!ix->v_nbr0[1 - ix->active]) return ins_fail(HNSW_EINVAL, "no capacity reserved (hnsw_reserve)");
    if (N0 + n > ix->capacity) return ins_fail(HNSW_EINVAL, "beyond the reserved capacity");
    if (V.storage != HNSW_F32 && !V.vec32)
        return ins_fail(HNSW_EINVAL, "needs the fp32 vectors (F32 storage or keep_fp32_for_rerank)");
    if (N0 == 0) return ins_fail(HNSW_EINVAL, "the index is empty (build its first elements with hnsw_build)");
    if (V.d > 32u * kMaxDW) return ins_fail(HNSW_EINVAL, "d above 256");
    const int efc = int(ix->build_efC), M = int(ix->build_M), Mmax = int(V.Mmax), Mmax0 = int(V.Mmax0);
    const int heur = (ix->build_flags & 1u) ? 1 : 0, keep = (ix->build_flags & 4u) ? 1 : 0;
    if ((ix->build_flags & 2u) != 0) return ins_fail(HNSW_EINVAL, "graphs built with extendCandidates");
    if (efc < 1 || efc > 1024) return ins_fail(HNSW_EINVAL, "efConstruction of the graph outside 1..1024");
    // levels (the level draw of Alg. 1) and the new upper rows, in id order
    std::vector<uint8_t> lv(n);
    std::vector<uint32_t> up(n, kNone), U, Z;
    std::vector<uint8_t> Ul;
    uint64_t rows = ix->upper_rows;
    for (uint64_t i = 0; i < n; ++i) {
        const double u = level_u[i];
        if (!(u > 0.0 && u <= 1.0)) return ins_fail(HNSW_EINVAL, "level_u outside (0,1]");
        const double l = std::floor(-std::log(u) * ix->build_mL);
        if (l > 255) return ins_fail(HNSW_EINVAL, "level above 255");
        lv[i] = uint8_t(l);
        if (lv[i] > 0) {
            up[i] = uint32_t(rows);
            rows += lv[i];
            U.push_back(uint32_t(N0 + i));
            Ul.push_back(lv[i]);
        } else {
            Z.push_back(uint32_t(N0 + i));
        }
    }
    if (rows > ix->upper_capacity) return ins_fail(HNSW_EINVAL, "upper-layer rows beyond the reserved capacity");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // searches still reading the version about to be overwritten finish first
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return ins_fail(HNSW_ECUDA, cudaGetErrorString(e));
    const int act = ix->active, ina = 1 - act;
    const uint32_t d = V.d, d_pad32 = V.row_chunks32 * 4;
    DevBuf stage, dU, dUl, visited, state;
    auto alloc = [&](DevBuf& x, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(&x.p, bytes ? bytes : 16);
    };
    alloc(stage, n * d_pad32 * 4ull);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ins_fail(HNSW_ENOMEM, "staging");
    }
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    // the version to write: a copy of the published one, with the new rows empty
    step(cudaMemcpyAsync(ix->v_nbr0[ina], ix->v_nbr0[act], N0 * V.s0 * 4ull, cudaMemcpyDeviceToDevice, s));
    step(cudaMemcpyAsync(ix->v_upoff[ina], ix->v_upoff[act], N0 * 4, cudaMemcpyDeviceToDevice, s));
    step(cudaMemcpyAsync(ix->v_nbrU[ina], ix->v_nbrU[act], ix->upper_rows * V.sU * 4ull, cudaMemcpyDeviceToDevice, s));
    step(cudaMemsetAsync(static_cast<uint32_t*>(ix->v_nbr0[ina]) + N0 * V.s0, 0xFF, n * V.s0 * 4ull, s));
    step(cudaMemsetAsync(static_cast<uint32_t*>(ix->v_nbrU[ina]) + ix->upper_rows * V.sU, 0xFF,
                         (rows - ix->upper_rows) * V.sU * 4ull, s));
    step(cudaMemcpyAsync(static_cast<uint32_t*>(ix->v_upoff[ina]) + N0, up.data(), n * 4, cudaMemcpyHostToDevice, s));
    // the vectors: fp32 rows d_pad32 apart, then the stored form
    step(cudaMemsetAsync(stage.p, 0, n * d_pad32 * 4ull, s));
    step(cudaMemcpy2DAsync(stage.p, d_pad32 * 4ull, data, d * 4ull, d * 4ull, n, cudaMemcpyDefault, s));
    if (e != cudaSuccess) return ins_fail(HNSW_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
    hnsw_status st = store_rows(ix, static_cast<const float*>(stage.p), N0, n, s);
    if (st != HNSW_OK) return st;
    // the fp32 view of the version being written
    V.nbr0 = static_cast<const uint32_t*>(ix->v_nbr0[ina]);
    V.upoff = static_cast<const uint32_t*>(ix->v_upoff[ina]);
    V.nbrU = static_cast<const uint32_t*>(ix->v_nbrU[ina]);
    V.urows = uint32_t(ix->upper_capacity);
    V.N = uint32_t(N0 + n);
    if (V.storage != HNSW_F32) {
        V.vec = V.vec32;
        V.row_chunks = V.row_chunks32;
        V.storage = HNSW_F32;
        V.scale = nullptr;
    }
    const int metric = V.metric;
    // 1. layer 0 of the new elements of level >= 1 (through the old upper layers)
    st = insert_layer0(ix, V, U, N0, metric, M, Mmax0, efc, heur, keep, s);
    if (st != HNSW_OK) return st;
    // 2. their upper layers, one at a time in id order
    if (!U.empty()) {
        alloc(dU, U.size() * 4);
        alloc(dUl, U.size());
        alloc(visited, (N0 + n) * 4);
        alloc(state, 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ins_fail(HNSW_ENOMEM, "upper-layer buffers");
        }
        const int st0[2] = {int(V.ep), V.maxlevel};
        step(cudaMemcpyAsync(dU.p, U.data(), U.size() * 4, cudaMemcpyHostToDevice, s));
        step(cudaMemcpyAsync(dUl.p, Ul.data(), U.size(), cudaMemcpyHostToDevice, s));
        step(cudaMemsetAsync(visited.p, 0, (N0 + n) * 4, s));
        step(cudaMemcpyAsync(state.p, st0, 8, cudaMemcpyHostToDevice, s));
        UpperArgs ua{};
        ua.v = V;
        ua.ids = static_cast<const uint32_t*>(dU.p);
        ua.lv = static_cast<const uint8_t*>(dUl.p);
        ua.n = uint32_t(U.size());
        ua.efc = efc;
        ua.M = M;
        ua.Mmax = Mmax;
        ua.heuristic = heur;
        ua.keep_pruned = keep;
        ua.visited = static_cast<uint32_t*>(visited.p);
        ua.state = static_cast<int*>(state.p);
        const size_t sm = upper_smem_bytes(Mmax, V.row_chunks * 4, efc);
        if (sm > 227 * 1024) return ins_fail(HNSW_EINVAL, "dimension too large for the upper-layer kernel");
        {
            const hnsw_status r = raise_smem_limit(reinterpret_cast<const void*>(insert_upper), sm, "hnsw_insert");
            if (r != HNSW_OK) return r;
        }
        if (e == cudaSuccess) {
            insert_upper<<<1, 32, sm, s>>>(ua);
            e = cudaGetLastError();
        }
        int st1[2] = {0, 0};
        step(cudaMemcpyAsync(st1, state.p, 8, cudaMemcpyDeviceToHost, s));
        step(cudaStreamSynchronize(s));
        if (e != cudaSuccess) return ins_fail(HNSW_ECUDA, std::string("upper layers: ") + cudaGetErrorString(e));
        V.ep = uint32_t(st1[0]);
        V.maxlevel = st1[1];
    }
    // 3. layer 0 of the new elements of level 0
    st = insert_layer0(ix, V, Z, N0 + U.size(), metric, M, Mmax0, efc, heur, keep, s);
    if (st != HNSW_OK) return st;
    step(cudaStreamSynchronize(s));
    if (e != cudaSuccess) return ins_fail(HNSW_ECUDA, cudaGetErrorString(e));
    // publish the new version
    {  // the device view and the info together (both read under dev_mu)
        std::lock_guard<std::mutex> dl(ix->dev_mu);
        ix->dev.nbr0 = V.nbr0;
        ix->dev.upoff = V.upoff;
        ix->dev.nbrU = V.nbrU;
        ix->dev.urows = V.urows;
        ix->dev.N = V.N;
        ix->dev.ep = V.ep;
        ix->dev.maxlevel = V.maxlevel;
        ix->info.N = V.N;
        ix->info.max_level = V.maxlevel;
        ix->info.enter_point = V.ep;
        ix->info.n_upper_rows = rows;
    }
    ix->active = ina;
    ix->d_nbr0 = ix->v_nbr0[ina];
    ix->d_upoff = ix->v_upoff[ina];
    ix->d_nbrU = ix->v_nbrU[ina];
    ix->upper_rows = rows;
    ix->levels.insert(ix->levels.end(), lv.begin(), lv.end());
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_index_to_blob(hnsw_index* ix, void** out_blob, uint64_t* out_bytes) {
    if (!ix || !out_blob || !out_bytes) return fail(HNSW_EINVAL, "hnsw_index_to_blob: null argument");
    std::lock_guard<std::mutex> lk(ix->insert_mu);
    const DevIndex D = dev_snapshot(ix);
    if (D.storage != HNSW_F32 && !D.vec32)
        return fail(HNSW_EINVAL, "hnsw_index_to_blob: needs the fp32 vectors (F32 storage or keep_fp32_for_rerank)");
    const uint64_t N = D.N;
    const uint32_t d = D.d, d_pad32 = D.row_chunks32 * 4;
    const BlobLayout lay = BlobLayout::of(N, d, D.Mmax0, D.Mmax, ix->upper_rows);
    uint8_t* b = static_cast<uint8_t*>(std::calloc(lay.total, 1));
    if (!b) return fail(HNSW_ENOMEM, "hnsw_index_to_blob: host memory");
    const void* src32 = D.storage == HNSW_F32 ? static_cast<const void*>(D.vec) : static_cast<const void*>(D.vec32);
    cudaError_t e = cudaMemcpy2D(b + lay.data, d * 4ull, src32, d_pad32 * 4ull, d * 4ull, N, cudaMemcpyDeviceToHost);
    std::vector<uint32_t> h0(N * size_t(D.s0)), hu(ix->upper_rows * size_t(D.sU));
    if (e == cudaSuccess && !h0.empty()) e = cudaMemcpy(h0.data(), D.nbr0, h0.size() * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && !hu.empty()) e = cudaMemcpy(hu.data(), D.nbrU, hu.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        std::free(b);
        return fail(HNSW_ECUDA, std::string("hnsw_index_to_blob: ") + cudaGetErrorString(e));
    }
    std::memcpy(b + lay.level, ix->levels.data(), N);
    for (uint64_t i = 0; i < N; ++i)
        for (uint32_t c = 0; c < D.Mmax0; ++c) wr<uint32_t>(b + lay.nbr0 + (i * D.Mmax0 + c) * 4, h0[i * D.s0 + c]);
    for (uint64_t r = 0; r < ix->upper_rows; ++r)
        for (uint32_t c = 0; c < D.Mmax; ++c) wr<uint32_t>(b + lay.nbrU + (r * D.Mmax + c) * 4, hu[r * D.sU + c]);
    BlobHeader h{};
    h.version = 1;
    h.metric = uint32_t(D.metric);
    h.N = N;
    h.d = d;
    h.M = ix->build_M;
    h.Mmax = D.Mmax;
    h.Mmax0 = D.Mmax0;
    h.maxlevel = N ? uint32_t(D.maxlevel) : 0;
    h.ep = N ? D.ep : kNone;
    h.flags = ix->build_flags;
    h.efC = ix->build_efC;
    h.mL = ix->build_mL;
    h.n_upper_rows = ix->upper_rows;
    h.checksum = fnv1a64(b + 128, lay.total - 128);
    write_header(b, h);
    *out_blob = b;
    *out_bytes = lay.total;
    return HNSW_OK;
}
