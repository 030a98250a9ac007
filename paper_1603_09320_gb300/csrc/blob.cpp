// blob.cpp -- error reporting, validation of "HNSWGB01" graph blobs, and
// their files.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.hpp"

namespace hnswgb {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

hnsw_status fail(hnsw_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

hnsw_status validate_blob(const uint8_t* b, uint64_t bytes, BlobHeader& h, BlobLayout& lay,
                          std::vector<uint32_t>& upoff, bool full) {
    if (!b) return fail(HNSW_EINVAL, "blob: null pointer");
    if (!read_header(b, bytes, h)) return fail(HNSW_ECORRUPT, "blob: bad magic, version or size");
    if (h.metric > 1 || h.d == 0 || h.N >= (1ull << 31) || h.Mmax0 == 0 || h.Mmax == 0 || h.Mmax0 > 64 ||
        h.Mmax > 64)
        return fail(HNSW_ECORRUPT, "blob: header fields out of range");
    lay = BlobLayout::of(h.N, h.d, h.Mmax0, h.Mmax, h.n_upper_rows);
    if (lay.total != bytes) return fail(HNSW_ECORRUPT, "blob: size does not match header");
    if (full && fnv1a64(b + 128, bytes - 128) != h.checksum) return fail(HNSW_ECORRUPT, "blob: checksum mismatch");
    const uint64_t N = h.N;
    const uint8_t* level = b + lay.level;
    if (N > 0) {
        if (h.ep >= N || level[h.ep] != h.maxlevel) return fail(HNSW_ECORRUPT, "blob: bad enter point");
    }
    upoff.assign(N, kNoId);
    uint64_t rows = 0;
    for (uint64_t i = 0; i < N; ++i) {
        if (level[i] > h.maxlevel) return fail(HNSW_ECORRUPT, "blob: level above the top level");
        if (level[i] > 0) {
            upoff[i] = uint32_t(rows);
            rows += level[i];
        }
    }
    if (rows != h.n_upper_rows || rows >= kNoId) return fail(HNSW_ECORRUPT, "blob: upper row count mismatch");
    // lists: valid ids first, then padding; no self or duplicate links; the
    // target of a link on layer lc is present on layer lc.
    auto check_row = [&](const uint8_t* r, uint32_t cap, uint64_t self, int lc) -> bool {
        bool ended = false;
        for (uint32_t j = 0; j < cap; ++j) {
            uint32_t x = rd<uint32_t>(r + 4ull * j);
            if (x == kNoId) {
                ended = true;
                continue;
            }
            if (ended || x >= N || x == self || level[x] < lc) return false;
            for (uint32_t k = 0; k < j; ++k)
                if (rd<uint32_t>(r + 4ull * k) == x) return false;
        }
        return true;
    };
    if (!full) return HNSW_OK;
    for (uint64_t i = 0; i < N; ++i) {
        if (!check_row(b + lay.nbr0 + i * h.Mmax0 * 4ull, h.Mmax0, i, 0))
            return fail(HNSW_ECORRUPT, "blob: bad layer-0 list of element " + std::to_string(i));
        for (int lc = 1; lc <= level[i]; ++lc) {
            const uint64_t rr = uint64_t(upoff[i]) + uint64_t(lc - 1);
            if (!check_row(b + lay.nbrU + rr * h.Mmax * 4ull, h.Mmax, i, lc))
                return fail(HNSW_ECORRUPT, "blob: bad upper list of element " + std::to_string(i));
        }
    }
    return HNSW_OK;
}

}  // namespace hnswgb

extern "C" const char* hnsw_last_error(void) { return hnswgb::g_last_error.c_str(); }
extern "C" int hnsw_abi_version(void) { return HNSW_ABI_VERSION; }

using namespace hnswgb;

extern "C" hnsw_status hnsw_save_blob(const void* blob, uint64_t bytes, const char* path) {
    if (!blob || !path) return fail(HNSW_EINVAL, "hnsw_save_blob: null argument");
    BlobHeader h{};
    BlobLayout lay{};
    std::vector<uint32_t> upoff;
    hnsw_status st = validate_blob(static_cast<const uint8_t*>(blob), bytes, h, lay, upoff);
    if (st != HNSW_OK) return st;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(HNSW_EINVAL, "hnsw_save_blob: cannot create " + tmp + ": " + std::strerror(errno));
    const bool ok = std::fwrite(blob, 1, bytes, f) == bytes;
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(HNSW_EINVAL, std::string("hnsw_save_blob: write failed: ") + std::strerror(errno));
    }
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_load_blob(const char* path, void** out_blob, uint64_t* out_bytes) {
    if (!path || !out_blob || !out_bytes) return fail(HNSW_EINVAL, "hnsw_load_blob: null argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(HNSW_EINVAL, std::string("hnsw_load_blob: cannot open ") + path + ": " + std::strerror(errno));
    uint64_t bytes = 0;
    if (std::fseek(f, 0, SEEK_END) == 0) {
        const long n = std::ftell(f);
        bytes = n > 0 ? uint64_t(n) : 0;
    }
    std::rewind(f);
    uint8_t* b = bytes ? static_cast<uint8_t*>(std::malloc(bytes)) : nullptr;
    if (bytes && !b) {
        std::fclose(f);
        return fail(HNSW_ENOMEM, "hnsw_load_blob: out of host memory");
    }
    const bool ok = bytes > 0 && std::fread(b, 1, bytes, f) == bytes;
    std::fclose(f);
    if (!ok) {
        std::free(b);
        return fail(HNSW_ECORRUPT, std::string("hnsw_load_blob: short or empty file ") + path);
    }
    BlobHeader h{};
    BlobLayout lay{};
    std::vector<uint32_t> upoff;
    hnsw_status st = validate_blob(b, bytes, h, lay, upoff);
    if (st != HNSW_OK) {
        std::free(b);
        return st;
    }
    *out_blob = b;
    *out_bytes = bytes;
    return HNSW_OK;
}
