// index.cu -- hnsw_upload_index / hnsw_free_index / hnsw_get_index_info and
// the quantiser that writes the stored vector rows on the device.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "common.hpp"
#include "index.cuh"

namespace hnswgb {
namespace {

// One warp per row: reads the fp32 row (d values, zero padded to d_pad32),
// writes the stored row (zero padded) and, for FP8E4M3, the row scale
// s = max|x| / 448 with codes RNE(x / s) saturated to the e4m3 range.
__global__ void quantize_rows(const float* __restrict__ src, uint32_t d_pad32, uint64_t N, uint32_t d,
                              int storage, uint8_t* __restrict__ dst, uint32_t row_bytes,
                              float* __restrict__ scale) {
    const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const float* x = src + warp * d_pad32;
    uint8_t* y = dst + warp * row_bytes;
    if (storage == HNSW_BF16 || storage == HNSW_F16) {
        const uint32_t n = row_bytes / 2;
        for (uint32_t i = lane; i < n; i += 32) {
            const float v = i < d ? x[i] : 0.0f;
            if (storage == HNSW_BF16) {
                __nv_bfloat16 b = __float2bfloat16_rn(v);
                reinterpret_cast<__nv_bfloat16*>(y)[i] = b;
            } else {
                __half h = __float2half_rn(v);
                reinterpret_cast<__half*>(y)[i] = h;
            }
        }
        return;
    }
    // FP8E4M3
    float m = 0.0f;
    for (uint32_t i = lane; i < d; i += 32) m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float s = m > 0.0f ? m / 448.0f : 1.0f;
    if (lane == 0) scale[warp] = s;
    for (uint32_t i = lane; i < row_bytes; i += 32) {
        const float v = i < d ? x[i] / s : 0.0f;
        y[i] = static_cast<uint8_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
    }
}

uint32_t round_up(uint32_t x, uint32_t m) { return (x + m - 1) / m * m; }

struct Guard {  // frees every registered device pointer unless released
    std::vector<void*> ptrs;
    bool keep = false;
    ~Guard() {
        if (!keep)
            for (void* p : ptrs) cudaFree(p);
    }
};

hnsw_status cuda_fail(cudaError_t e, const char* what) {
    return fail(HNSW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace
}  // namespace hnswgb

using namespace hnswgb;

#define HNSW_CUDA_TRY(expr, what)                              \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);     \
    } while (0)

extern "C" hnsw_status hnsw_upload_index(const void* graph_blob, uint64_t blob_bytes, hnsw_dtype storage,
                                         int keep_fp32_for_rerank, void* stream, hnsw_index** out) {
    return upload_index(graph_blob, blob_bytes, storage, keep_fp32_for_rerank, stream, out, false);
}

namespace hnswgb {

// hnsw_upload_index; trusted: a blob the library has just written (no
// checksum or per-list validation)
hnsw_status upload_index(const void* graph_blob, uint64_t blob_bytes, hnsw_dtype storage, int keep_fp32_for_rerank,
                         void* stream, hnsw_index** out, bool trusted) {
    if (!out) return fail(HNSW_EINVAL, "hnsw_upload_index: out is null");
    *out = nullptr;
    if (storage < HNSW_F32 || storage > HNSW_F16) return fail(HNSW_EINVAL, "hnsw_upload_index: bad storage");
    const uint8_t* b = static_cast<const uint8_t*>(graph_blob);
    BlobHeader h{};
    BlobLayout lay{};
    std::vector<uint32_t> upoff;
    hnsw_status st = validate_blob(b, blob_bytes, h, lay, upoff, !trusted);
    if (st != HNSW_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t N = h.N;
    const uint32_t d = h.d;
    const uint32_t d_pad32 = round_up(d, 4);
    uint32_t coords_per_chunk = storage == HNSW_F32 ? 4 : (storage == HNSW_FP8E4M3 ? 16 : 8);
    const uint32_t d_pad = round_up(d, coords_per_chunk);
    const uint32_t elem = storage == HNSW_F32 ? 4 : (storage == HNSW_FP8E4M3 ? 1 : 2);
    const uint32_t row_bytes = d_pad * elem;
    if (d_pad32 > 512 || row_bytes > 2048)
        return fail(HNSW_EINVAL, "hnsw_upload_index: dimension above 512 is not supported");
    const uint32_t s0 = round_up(h.Mmax0, 4), sU = round_up(h.Mmax, 4);

    std::unique_ptr<hnsw_index> holder(new (std::nothrow) hnsw_index());
    hnsw_index* ix = holder.get();
    if (!ix) return fail(HNSW_ENOMEM, "hnsw_upload_index: host allocation");
    Guard g;
    auto dalloc = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) g.ptrs.push_back(*p);
        return e;
    };
    cudaGetDevice(&ix->device);
    try {
        // fp32 rows, padded to d_pad32 (host repack only when d is not a multiple of 4)
        const float* data = reinterpret_cast<const float*>(b + lay.data);
        std::vector<float> padded;
        if (d_pad32 != d) {
            padded.assign(N * d_pad32, 0.0f);
            for (uint64_t i = 0; i < N; ++i) std::memcpy(&padded[i * d_pad32], data + i * d, d * 4ull);
            data = padded.data();
        }
        void* d32 = nullptr;
        cudaError_t e = dalloc(&d32, N * d_pad32 * 4ull);
        if (e != cudaSuccess) { return fail(HNSW_ENOMEM, "hnsw_upload_index: device vectors"); }
        HNSW_CUDA_TRY(cudaMemcpyAsync(d32, data, N * d_pad32 * 4ull, cudaMemcpyHostToDevice, s), "copy vectors");
        if (storage == HNSW_F32) {
            ix->d_vec = d32;
        } else {
            if (dalloc(&ix->d_vec, N * row_bytes) != cudaSuccess) { return fail(HNSW_ENOMEM, "device rows"); }
            if (storage == HNSW_FP8E4M3 && dalloc(&ix->d_scale, N * 4ull) != cudaSuccess) {
                return fail(HNSW_ENOMEM, "device scales");
            }
            if (N > 0) {
                const uint64_t threads = N * 32ull;
                const unsigned blocks = unsigned((threads + 255) / 256);
                quantize_rows<<<blocks, 256, 0, s>>>(static_cast<const float*>(d32), d_pad32, N, d, int(storage),
                                                     static_cast<uint8_t*>(ix->d_vec), row_bytes,
                                                     static_cast<float*>(ix->d_scale));
                HNSW_CUDA_TRY(cudaGetLastError(), "quantize launch");
            }
            if (keep_fp32_for_rerank) {
                ix->d_vec32 = d32;
            } else {
                HNSW_CUDA_TRY(cudaStreamSynchronize(s), "quantize");
                cudaFree(d32);
                g.ptrs.erase(std::find(g.ptrs.begin(), g.ptrs.end(), d32));
            }
        }
        if (storage == HNSW_F32 && keep_fp32_for_rerank) ix->d_vec32 = d32;
        // adjacency, repacked to 4-id strides
        std::vector<uint32_t> nbr0(N * s0, kNone), nbrU(h.n_upper_rows * sU, kNone);
        for (uint64_t i = 0; i < N; ++i)
            std::memcpy(&nbr0[i * s0], b + lay.nbr0 + i * h.Mmax0 * 4ull, h.Mmax0 * 4ull);
        for (uint64_t r = 0; r < h.n_upper_rows; ++r)
            std::memcpy(&nbrU[r * sU], b + lay.nbrU + r * h.Mmax * 4ull, h.Mmax * 4ull);
        if (dalloc(&ix->d_nbr0, nbr0.size() * 4) != cudaSuccess || dalloc(&ix->d_upoff, N * 4) != cudaSuccess ||
            dalloc(&ix->d_nbrU, nbrU.size() * 4) != cudaSuccess ||
            dalloc(reinterpret_cast<void**>(&ix->d_work), kWorkSlots * 4) != cudaSuccess) {
            return fail(HNSW_ENOMEM, "hnsw_upload_index: device adjacency");
        }
        if (cudaHostAlloc(reinterpret_cast<void**>(&ix->h_err), 4, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&ix->d_err), ix->h_err, 0) != cudaSuccess) {
            cudaGetLastError();
            return fail(HNSW_ENOMEM, "hnsw_upload_index: error word");
        }
        *reinterpret_cast<volatile uint32_t*>(ix->h_err) = 0u;
        HNSW_CUDA_TRY(cudaMemcpyAsync(ix->d_nbr0, nbr0.data(), nbr0.size() * 4, cudaMemcpyHostToDevice, s), "copy nbr0");
        HNSW_CUDA_TRY(cudaMemcpyAsync(ix->d_upoff, upoff.data(), N * 4, cudaMemcpyHostToDevice, s), "copy upoff");
        HNSW_CUDA_TRY(cudaMemcpyAsync(ix->d_nbrU, nbrU.data(), nbrU.size() * 4, cudaMemcpyHostToDevice, s), "copy nbrU");
        HNSW_CUDA_TRY(cudaMemsetAsync(ix->d_work, 0, kWorkSlots * 4, s), "clear work");
        HNSW_CUDA_TRY(cudaStreamSynchronize(s), "upload");
    } catch (const std::bad_alloc&) {
        return fail(HNSW_ENOMEM, "hnsw_upload_index: host allocation");
    }
    DevIndex& D = ix->dev;
    D.vec = static_cast<const uint4*>(ix->d_vec);
    D.scale = static_cast<const float*>(ix->d_scale);
    D.vec32 = static_cast<const uint4*>(ix->d_vec32);
    D.nbr0 = static_cast<const uint32_t*>(ix->d_nbr0);
    D.upoff = static_cast<const uint32_t*>(ix->d_upoff);
    D.nbrU = static_cast<const uint32_t*>(ix->d_nbrU);
    D.N = uint32_t(N);
    D.urows = uint32_t(h.n_upper_rows);
    D.d = d;
    D.row_chunks = row_bytes / 16;
    D.row_chunks32 = d_pad32 / 4;
    D.s0 = s0;
    D.sU = sU;
    D.Mmax0 = h.Mmax0;
    D.Mmax = h.Mmax;
    D.ep = N ? h.ep : kNone;
    D.maxlevel = N ? int32_t(h.maxlevel) : -1;
    D.metric = int32_t(h.metric);
    D.storage = int32_t(storage);
    hnsw_index_info& I = ix->info;
    I.N = N;
    I.d = d;
    I.d_pad = d_pad;
    I.row_bytes = row_bytes;
    I.metric = int32_t(h.metric);
    I.storage = int32_t(storage);
    I.has_fp32 = ix->d_vec32 != nullptr;
    I.M = h.M;
    I.Mmax = h.Mmax;
    I.Mmax0 = h.Mmax0;
    I.max_level = D.maxlevel;
    I.enter_point = D.ep;
    I.n_upper_rows = h.n_upper_rows;
    ix->build_M = h.M;
    ix->build_efC = h.efC;
    ix->build_flags = h.flags;
    ix->build_mL = h.mL;
    ix->levels.assign(b + lay.level, b + lay.level + N);
    ix->upper_rows = h.n_upper_rows;
    ix->capacity = N;
    ix->upper_capacity = h.n_upper_rows;
    ix->v_nbr0[0] = ix->d_nbr0;
    ix->v_upoff[0] = ix->d_upoff;
    ix->v_nbrU[0] = ix->d_nbrU;
    I.device_bytes = N * row_bytes + (ix->d_scale ? N * 4 : 0) + (ix->d_vec32 && storage != HNSW_F32 ? N * d_pad32 * 4ull : 0) +
                     N * s0 * 4ull + N * 4ull + h.n_upper_rows * sU * 4ull + kWorkSlots * 4;
    g.keep = true;
    *out = holder.release();
    return HNSW_OK;
}

}  // namespace hnswgb

extern "C" hnsw_status hnsw_free_index(hnsw_index* ix) {
    if (!ix) return HNSW_OK;
    void* ptrs[] = {ix->d_vec, ix->d_scale, ix->d_nbr0, ix->d_upoff, ix->d_nbrU, ix->d_work, ix->d_stop};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    // the unpublished adjacency version, when an insertion capacity was reserved
    const int o = 1 - ix->active;
    for (void* p : {ix->v_nbr0[o], ix->v_upoff[o], ix->v_nbrU[o]})
        if (p) cudaFree(p);
    for (auto& st : ix->stages)
        if (st.buf) cudaFree(st.buf);
    if (ix->d_vec32 && ix->d_vec32 != ix->d_vec) cudaFree(ix->d_vec32);
    if (ix->h_err) cudaFreeHost(ix->h_err);
    delete ix;
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_get_index_info(const hnsw_index* ix, hnsw_index_info* out) {
    if (!ix || !out) return fail(HNSW_EINVAL, "hnsw_get_index_info: null pointer");
    // an insertion publishes N, top level, enter point and rows under dev_mu
    hnsw_index* m = const_cast<hnsw_index*>(ix);
    {
        std::lock_guard<std::mutex> lk(m->dev_mu);
        *out = ix->info;
    }
    uint64_t sb = 0;
    {
        std::lock_guard<std::mutex> lk(m->stage_mu);
        for (const auto& st : m->stages) sb += st.bytes;
    }
    out->staging_bytes = sb;
    return HNSW_OK;
}

namespace hnswgb {

hnsw_status raise_smem_limit(const void* fn, size_t bytes, const char* who) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, fn}];
    if (cur >= bytes) return HNSW_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess)
        return fail(HNSW_ECUDA, std::string(who) + ": shared memory attribute: " + cudaGetErrorString(e));
    cur = bytes;
    return HNSW_OK;
}

hnsw_status store_rows(hnsw_index* ix, const float* rows32, uint64_t first, uint64_t n, cudaStream_t s) {
    if (n == 0) return HNSW_OK;
    const hnsw_index_info& I = ix->info;
    const uint32_t d_pad32 = round_up(I.d, 4);
    uint8_t* vec = static_cast<uint8_t*>(ix->d_vec) + first * I.row_bytes;
    cudaError_t e = cudaSuccess;
    if (I.storage == HNSW_F32) {
        e = cudaMemcpyAsync(vec, rows32, n * I.row_bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        const unsigned blocks = unsigned((n * 32ull + 255) / 256);
        quantize_rows<<<blocks, 256, 0, s>>>(rows32, d_pad32, n, I.d, I.storage, vec, I.row_bytes,
                                             ix->d_scale ? static_cast<float*>(ix->d_scale) + first : nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess && ix->d_vec32)
            e = cudaMemcpyAsync(static_cast<float*>(ix->d_vec32) + first * d_pad32, rows32, n * d_pad32 * 4ull,
                                cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) return fail(HNSW_ECUDA, std::string("store rows: ") + cudaGetErrorString(e));
    return HNSW_OK;
}

}  // namespace hnswgb

