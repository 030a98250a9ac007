// common.hpp -- error reporting and the graph blob format ("HNSWGB01") as the
// library reads and writes it.  Host-only C++.
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hnsw.h"

namespace hnswgb {

// thread-local last-error message behind hnsw_last_error()
void set_error(const std::string& msg);
hnsw_status fail(hnsw_status st, const std::string& msg);

constexpr uint32_t kNoId = 0xFFFFFFFFu;

inline uint64_t align16(uint64_t x) { return (x + 15u) & ~uint64_t(15); }

// Offsets of the payload sections of a blob (header is 128 bytes).
struct BlobLayout {
    uint64_t data, level, nbr0, nbrU, total;
    static BlobLayout of(uint64_t N, uint32_t d, uint32_t Mmax0, uint32_t Mmax, uint64_t rows) {
        BlobLayout o;
        o.data = 128;
        o.level = align16(o.data + N * d * 4ull);
        o.nbr0 = align16(o.level + N);
        o.nbrU = align16(o.nbr0 + N * Mmax0 * 4ull);
        o.total = o.nbrU + rows * Mmax * 4ull;
        return o;
    }
};

// 64-bit FNV-1a over a byte range, 8 bytes per step of the outer loop.
inline uint64_t fnv1a64(const uint8_t* p, uint64_t n) {
    uint64_t h = 0xcbf29ce484222325ull;
    const uint64_t prime = 0x100000001b3ull;
    for (uint64_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= prime;
    }
    return h;
}

struct BlobHeader {
    uint32_t version, metric;
    uint64_t N;
    uint32_t d, M, Mmax, Mmax0, maxlevel, ep, flags, efC;
    double mL;
    uint64_t n_upper_rows, checksum;
};

template <class T>
inline T rd(const uint8_t* p) {
    T v;
    std::memcpy(&v, p, sizeof(T));
    return v;
}
template <class T>
inline void wr(uint8_t* p, T v) {
    std::memcpy(p, &v, sizeof(T));
}

inline void write_header(uint8_t* b, const BlobHeader& h) {
    std::memset(b, 0, 128);
    std::memcpy(b, "HNSWGB01", 8);
    wr<uint32_t>(b + 8, h.version);
    wr<uint32_t>(b + 12, h.metric);
    wr<uint64_t>(b + 16, h.N);
    wr<uint32_t>(b + 24, h.d);
    wr<uint32_t>(b + 28, h.M);
    wr<uint32_t>(b + 32, h.Mmax);
    wr<uint32_t>(b + 36, h.Mmax0);
    wr<uint32_t>(b + 40, h.maxlevel);
    wr<uint32_t>(b + 44, h.ep);
    wr<uint32_t>(b + 48, h.flags);
    wr<uint32_t>(b + 52, h.efC);
    wr<double>(b + 56, h.mL);
    wr<uint64_t>(b + 64, h.n_upper_rows);
    wr<uint64_t>(b + 72, h.checksum);
}

inline bool read_header(const uint8_t* b, uint64_t bytes, BlobHeader& h) {
    if (bytes < 128 || std::memcmp(b, "HNSWGB01", 8) != 0) return false;
    h.version = rd<uint32_t>(b + 8);
    h.metric = rd<uint32_t>(b + 12);
    h.N = rd<uint64_t>(b + 16);
    h.d = rd<uint32_t>(b + 24);
    h.M = rd<uint32_t>(b + 28);
    h.Mmax = rd<uint32_t>(b + 32);
    h.Mmax0 = rd<uint32_t>(b + 36);
    h.maxlevel = rd<uint32_t>(b + 40);
    h.ep = rd<uint32_t>(b + 44);
    h.flags = rd<uint32_t>(b + 48);
    h.efC = rd<uint32_t>(b + 52);
    h.mL = rd<double>(b + 56);
    h.n_upper_rows = rd<uint64_t>(b + 64);
    h.checksum = rd<uint64_t>(b + 72);
    return h.version == 1;
}

// Full structural validation of a blob; on success fills `h`, the layout and
// the per-element first-upper-row offsets (kNoId for level-0 elements).
// full = false (a blob the library has just written itself): header, sizes
// and offsets only -- no checksum, no per-list checks.
hnsw_status validate_blob(const uint8_t* b, uint64_t bytes, BlobHeader& h, BlobLayout& lay,
                          std::vector<uint32_t>& upoff, bool full = true);

}  // namespace hnswgb
