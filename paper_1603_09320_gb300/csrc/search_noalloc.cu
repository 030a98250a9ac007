// search_noalloc.cu -- hnsw_search_noalloc: batched K-NN search that performs
// no device allocation of its own.
//
// Who needs it: callers that cannot call cudaMalloc on the search path, for
// example a process whose device memory has been handed in full to another
// allocator (a framework's caching allocator or a serving runtime that
// reserves all memory at start-up, so a new cudaMalloc fails), or a latency
// critical path that must not take cudaMalloc/cudaFree, which synchronise the
// device.  hnsw_search itself allocates a staging buffer the first time it is
// given host pointers; this entry point uses a fixed device array instead.
//
// The scratch is one file-scope device array of kScratchBytes (16 MiB).  Every
// GPU that loads the library holds it until the process exits.  Host code
// never uses the array's name as an address: the first call on each device
// (with that device current) looks the address up with cudaGetSymbolAddress,
// checks the result and caches it; later calls reuse it.  Make that first
// call before any stream capture.
//
// Layout of the array per call: bytes [0, 256) hold the work-queue counter of
// the search kernel, cleared to zero on the stream before each launch; the
// rest stages the host-memory buffers of the call (queries, ids, distances),
// each 256-byte aligned.  All calls share the array and it keeps the last
// call's contents, so calls whose work overlaps on the GPU (concurrent
// streams, other threads) race on it: issue them one after another.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "common.hpp"
#include "index.cuh"

namespace hnswgb {
// defined in search.cu
hnsw_status launch_search(hnsw_index* ix, const hnsw_search_params& p, const float* q, uint32_t n,
                          uint32_t* ids, float* dists, hnsw_query_stats* stats, cudaStream_t s,
                          uint32_t* work, const StopModel* stop);
}  // namespace hnswgb

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_search_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_search_scratch on the current device (looked up once).
hnsw_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hnswgb::fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return hnswgb::fail(HNSW_EINVAL, "hnsw_search_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_search_scratch);
        if (e != cudaSuccess || !p)
            return hnswgb::fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: scratch lookup: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HNSW_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" hnsw_status hnsw_search_noalloc(hnsw_index* ix, const float* queries, int64_t n, int32_t k,
                                           int32_t ef, uint32_t* out_ids, float* out_dists, void* stream) {
    using hnswgb::fail;
    if (!ix) return fail(HNSW_EINVAL, "hnsw_search_noalloc: null index");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(HNSW_EINVAL, "hnsw_search_noalloc: n out of range");
    if (k < 1 || k > hnswgb::kMaxK || ef < 1) return fail(HNSW_EINVAL, "hnsw_search_noalloc: k or ef out of range");
    if ((ef > k ? ef : k) > hnswgb::kMaxEf) return fail(HNSW_EINVAL, "hnsw_search_noalloc: ef' above 1024");
    if (n == 0) return HNSW_OK;
    if (!queries || !out_ids || !out_dists) return fail(HNSW_EINVAL, "hnsw_search_noalloc: null buffer");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ix->device) return fail(HNSW_EINVAL, "hnsw_search_noalloc: index lives on another device");
    void* base = nullptr;
    hnsw_status st = scratch_address(&base);
    if (st != HNSW_OK) return st;

    const bool dq = on_device(queries), di = on_device(out_ids), dd = on_device(out_dists);
    const size_t qb = size_t(n) * ix->dev.d * 4, ob = size_t(n) * size_t(k) * 4;
    const size_t need = 256 + (dq ? 0 : up256(qb)) + (di ? 0 : up256(ob)) + (dd ? 0 : up256(ob));
    if (need > kScratchBytes)
        return fail(HNSW_EINVAL, "hnsw_search_noalloc: the batch needs " + std::to_string(need) +
                                     " bytes of staging but the fixed scratch holds " + std::to_string(kScratchBytes) +
                                     " bytes; pass device buffers or split the batch");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* p = static_cast<uint8_t*>(base);
    uint32_t* work = reinterpret_cast<uint32_t*>(p);
    p += 256;
    const float* q = queries;
    uint32_t* ids = out_ids;
    float* dists = out_dists;
    cudaError_t e;
    if (!dq) {
        e = cudaMemcpyAsync(p, queries, qb, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: H2D: ") + cudaGetErrorString(e));
        q = reinterpret_cast<const float*>(p);
        p += up256(qb);
    }
    if (!di) {
        ids = reinterpret_cast<uint32_t*>(p);
        p += up256(ob);
    }
    if (!dd) dists = reinterpret_cast<float*>(p);
    e = cudaMemsetAsync(work, 0, sizeof(uint32_t), s);  // the work counter starts at zero
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: clear: ") + cudaGetErrorString(e));
    hnsw_search_params prm{};
    prm.k = k;
    prm.ef = ef;
    prm.stop_threshold = 2.0f;
    st = hnswgb::launch_search(ix, prm, q, uint32_t(n), ids, dists, nullptr, s, work, nullptr);
    if (st != HNSW_OK) return st;
    if (!di && (e = cudaMemcpyAsync(out_ids, ids, ob, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: D2H ids: ") + cudaGetErrorString(e));
    if (!dd && (e = cudaMemcpyAsync(out_dists, dists, ob, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: D2H distances: ") + cudaGetErrorString(e));
    if (!dq || !di || !dd) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("hnsw_search_noalloc: ") + cudaGetErrorString(e));
    }
    return HNSW_OK;
}
