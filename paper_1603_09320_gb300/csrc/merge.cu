// merge.cu -- the exchange step of data-sharded search (Section 6 discusses
// distributing HNSW by partitioning the data): every shard holds its own
// graph over a disjoint range of element ids and answers every query with its
// own K nearest; the global answer is the K smallest keys (distance, global
// id) of the union of the shards' answers.
//
// One warp per query.  Lane s holds the head of shard s's list (each list is
// sorted by (distance, local id), and adding the shard's id base keeps that
// order); K times the warp takes the smallest head, lane 0 writes it, and the
// winning lane advances in its list.  Global ids are distinct across shards,
// so the smallest head is unique.  Padding entries (HNSW_NO_ID) end a list;
// when every list has ended the rest of the output is padded.
#include <cuda_runtime.h>

#include <string>

#include "common.hpp"
#include "index.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxShards = 32;

struct MergeArgs {
    const uint32_t* ids;    // [S][n][k]
    const float* dists;     // [S][n][k]
    uint32_t base[kMaxShards];
    int S;
    uint32_t n;
    int k;
    uint32_t* out_ids;      // [n][k]
    float* out_dists;       // [n][k]
};

__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// key of entry j of shard s's list for query q (~0: the list has ended)
__device__ __forceinline__ uint64_t head_key(const MergeArgs& a, int s, uint32_t q, int j) {
    if (j >= a.k) return ~0ull;
    const uint64_t o = (uint64_t(s) * a.n + q) * uint64_t(a.k) + uint64_t(j);
    const uint32_t id = __ldg(a.ids + o);
    if (id == hnswgb::kNoId) return ~0ull;
    return (uint64_t(f2ord(__ldg(a.dists + o))) << 32) | uint64_t(a.base[s] + id);
}

__global__ void __launch_bounds__(256) merge_topk(const MergeArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < a.n; q += warps) {
        int cur = 0;
        uint64_t head = lane < a.S ? head_key(a, lane, q, 0) : ~0ull;
        const uint64_t ob = uint64_t(q) * uint64_t(a.k);
        for (int i = 0; i < a.k; ++i) {
            const uint32_t hi = uint32_t(head >> 32), lo = uint32_t(head);
            const uint32_t mh = __reduce_min_sync(kFull, hi);
            const uint32_t ml = __reduce_min_sync(kFull, hi == mh ? lo : 0xffffffffu);
            const uint64_t m = (uint64_t(mh) << 32) | ml;
            if (m == ~0ull) {  // every list has ended: pad
                for (int j = i + lane; j < a.k; j += 32) {
                    a.out_ids[ob + j] = hnswgb::kNoId;
                    a.out_dists[ob + j] = __int_as_float(0x7f800000);
                }
                break;
            }
            if (lane == 0) {
                a.out_ids[ob + i] = ml;
                a.out_dists[ob + i] = ord2f(mh);
            }
            if (head == m) head = head_key(a, lane, q, ++cur);
        }
    }
}

}  // namespace

extern "C" hnsw_status hnsw_merge_topk(const uint32_t* shard_ids, const float* shard_dists, int32_t n_shards,
                                       const uint32_t* id_base, int64_t n, int32_t k, uint32_t* out_ids,
                                       float* out_dists, void* stream) {
    using hnswgb::fail;
    if (n_shards < 1 || n_shards > kMaxShards) return fail(HNSW_EINVAL, "hnsw_merge_topk: n_shards outside [1,32]");
    if (n < 0 || n >= (int64_t(1) << 31) || k < 1 || k > hnswgb::kMaxK)
        return fail(HNSW_EINVAL, "hnsw_merge_topk: n or k out of range");
    if (!id_base) return fail(HNSW_EINVAL, "hnsw_merge_topk: null id_base");
    if (n == 0) return HNSW_OK;
    if (!shard_ids || !shard_dists || !out_ids || !out_dists) return fail(HNSW_EINVAL, "hnsw_merge_topk: null buffer");
    for (const void* p : {static_cast<const void*>(shard_ids), static_cast<const void*>(shard_dists),
                          static_cast<const void*>(out_ids), static_cast<const void*>(out_dists)}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(HNSW_EINVAL, "hnsw_merge_topk: buffers must be device memory");
        }
    }
    MergeArgs a{};
    a.ids = shard_ids;
    a.dists = shard_dists;
    a.S = n_shards;
    a.n = uint32_t(n);
    a.k = k;
    a.out_ids = out_ids;
    a.out_dists = out_dists;
    for (int s = 0; s < n_shards; ++s) a.base[s] = id_base[s];
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t blocks_needed = (uint64_t(n) + 7) / 8;
    const uint64_t cap = uint64_t(sms) * 8;
    merge_topk<<<unsigned(blocks_needed < cap ? blocks_needed : cap), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_merge_topk: ") + cudaGetErrorString(e));
    return HNSW_OK;
}
