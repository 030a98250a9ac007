// index.cuh -- the device-resident layout of one HNSW index and the host
// object that owns it.
//
// Device layout (Section 4.2.3 sizes the links at (Mmax0 + mL*Mmax) * 4 bytes
// per element; ids are 4-byte unsigned integers):
//   vec    [N][row_chunks]  16-byte chunks; storage dtype, row zero padded
//   scale  [N]              fp32 per-row scale (FP8E4M3 storage only)
//   vec32  [N][row_chunks32] fp32 copy for the exact rerank (optional)
//   nbr0   [N][s0]          layer-0 neighbour ids, s0 = Mmax0 rounded up to 4,
//                           valid ids first, then 0xFFFFFFFF
//   upoff  [N]              first upper-layer row of an element (0xFFFFFFFF at level 0)
//   nbrU   [rows][sU]       upper rows; element i's row for layer lc >= 1 is
//                           upoff[i] + lc - 1; sU = Mmax rounded up to 4
//   work   [kWorkSlots]     work-queue counters of the persistent search kernel
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/hnsw.h"

namespace hnswgb {

constexpr int kWorkSlots = 1024;
constexpr int kMaxStages = 16;  // streams with their own host-memory staging buffer
constexpr int kMaxEf = 1024;   // ef' limit of the search kernel
constexpr int kMaxK = 1024;
constexpr uint32_t kNone = 0xFFFFFFFFu;

struct DevIndex {
    const uint4* vec;
    const float* scale;
    const uint4* vec32;
    const uint32_t* nbr0;
    const uint32_t* upoff;
    const uint32_t* nbrU;
    uint32_t N, d;
    uint32_t urows;  // upper-layer rows allocated (bound of upoff[i] + lc - 1)
    uint32_t row_chunks, row_chunks32;
    uint32_t s0, sU, Mmax0, Mmax;
    uint32_t ep;
    int32_t maxlevel;
    int32_t metric;
    int32_t storage;
};

// Optional parts of one search launch: the learned early stop and the trace
// recording used to train it (all null/zero: the plain search).
struct StopModel {
    const void* stop;       // device StopDev, or null
    float logit_threshold;  // stop when the network's logit exceeds this
    int period;             // check every `period` layer-0 expansions
    float* tr_feat;         // trace buffers (device), tr_count == null: no trace
    uint32_t* tr_topk;
    float* tr_logit;
    int32_t* tr_count;
    int tr_max;
};

}  // namespace hnswgb

struct hnsw_index {
    hnswgb::DevIndex dev{};
    hnsw_index_info info{};
    // owned device allocations
    void* d_vec = nullptr;
    void* d_scale = nullptr;
    void* d_vec32 = nullptr;
    void* d_nbr0 = nullptr;
    void* d_upoff = nullptr;
    void* d_nbrU = nullptr;
    uint32_t* d_work = nullptr;
    void* d_stop = nullptr;  // learned-stop weights (fp16), or null
    std::atomic<uint32_t> work_next{0};
    // staging for host-memory queries/results: one device buffer per stream
    // (grown on demand, at most kMaxStages streams; the oldest idle one is
    // dropped to make room)
    struct Stage {
        void* stream;
        void* buf;
        size_t bytes;
        int in_use;  // calls between taking the buffer and their final synchronisation
    };
    std::mutex stage_mu;
    std::vector<Stage> stages;
    // `dev` is read by every launch and replaced by an incremental insertion
    // when it publishes a new adjacency version: both under dev_mu
    std::mutex dev_mu;
    // construction parameters of the graph (from its header) and the levels
    uint32_t build_M = 0, build_efC = 0, build_flags = 0;
    double build_mL = 0.0;
    std::vector<uint8_t> levels;
    uint64_t upper_rows = 0;  // upper-layer rows in use
    // incremental insertion (hnsw_reserve / hnsw_insert): rows allocated, and
    // two versions of the adjacency -- the published one (index `active`) and
    // the one the next insertion writes
    uint64_t capacity = 0, upper_capacity = 0;
    void* v_nbr0[2] = {nullptr, nullptr};
    void* v_upoff[2] = {nullptr, nullptr};
    void* v_nbrU[2] = {nullptr, nullptr};
    int active = 0;
    std::mutex insert_mu;
    int device = 0;
    // a search kernel whose bounded wait ran out sets this word (host memory
    // mapped into the device's address space: h_err on the host, d_err on
    // the device); the next search call that synchronises reads and clears it
    uint32_t* h_err = nullptr;
    uint32_t* d_err = nullptr;
    // test hook (hnsw_debug_hold_decisions): searches withhold one decision
    // of the deferral, so that its claims wait until their limit runs out
    std::atomic<int> hold_decisions{0};
};

namespace hnswgb {
// The index's published device view (a consistent snapshot for one launch).
inline DevIndex dev_snapshot(hnsw_index* ix) {
    std::lock_guard<std::mutex> lk(ix->dev_mu);
    return ix->dev;
}
// hnsw_upload_index; trusted: skip the checksum and per-list validation of a
// blob the library has just written itself.
hnsw_status upload_index(const void* graph_blob, uint64_t blob_bytes, hnsw_dtype storage, int keep_fp32_for_rerank,
                         void* stream, hnsw_index** out, bool trusted);
// Writes stored rows [first, first + n) (and the fp32 copy when kept) from
// fp32 rows in device memory, d_pad32 floats apart; asynchronous on s.
hnsw_status store_rows(hnsw_index* ix, const float* rows32, uint64_t first, uint64_t n, cudaStream_t s);

// Raises kernel `fn`'s dynamic shared-memory limit on the current device to
// at least `bytes`.  The limit is per device and is never lowered: a launch
// issued by another thread after it raised the limit may still rely on it.
hnsw_status raise_smem_limit(const void* fn, size_t bytes, const char* who);
}  // namespace hnswgb
