// Host-side driver for the sanitizer builds of the graph builder and the
// graph-file code (builder.cpp, blob.cpp), run by test_host_sanitizers.py
// under ThreadSanitizer and under AddressSanitizer + UBSan: concurrent
// construction (Alg. 1 with Alg. 3 / Alg. 4, Section 4.1's parallel build)
// on small seeded inputs, then the blob checks, file round trip and the
// rejection paths.  Exit status 0 when every call returned what it should.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "hnsw.h"

static uint64_t g_state = 0x9E3779B97F4A7C15ull;
static double next_unit() {  // (0, 1]
    g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double((g_state >> 11) & ((1ull << 53) - 1)) + 1.0) / 9007199254740992.0;
}

static int check(bool ok, const char* what) {
    if (!ok) std::fprintf(stderr, "FAILED: %s (%s)\n", what, hnsw_last_error());
    return ok ? 0 : 1;
}

int main(int argc, char** argv) {
    const uint64_t N = argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 3000;
    const int threads = argc > 2 ? std::atoi(argv[2]) : 8;
    const char* dir = argc > 3 ? argv[3] : ".";
    const uint32_t d = 12;  // not a multiple of 8: the distance tails run too
    std::vector<float> X(N * d);
    for (auto& x : X) x = float(std::floor(next_unit() * 64.0));  // many equal distances
    std::vector<float> Xn(X);
    for (uint64_t i = 0; i < N; ++i) {
        double s = 0;
        for (uint32_t j = 0; j < d; ++j) s += double(X[i * d + j]) * X[i * d + j] + 1e-3;
        for (uint32_t j = 0; j < d; ++j) Xn[i * d + j] = float((X[i * d + j] + 0.03) / std::sqrt(s));
    }
    std::vector<double> u(N);
    for (auto& v : u) v = next_unit();

    int bad = 0;
    struct Case {
        hnsw_metric metric;
        int heuristic, keep;
    } cases[] = {{HNSW_L2SQ, 1, 0}, {HNSW_L2SQ, 0, 0}, {HNSW_L2SQ, 1, 1}, {HNSW_COSINE, 1, 0}};
    for (const Case& c : cases) {
        hnsw_build_params p{};
        p.M = 6;
        p.Mmax = 6;
        p.Mmax0 = 12;
        p.ef_construction = 32;
        p.mL = 1.0 / std::log(6.0);
        p.heuristic = c.heuristic;
        p.keep_pruned = c.keep;
        p.n_threads = threads;
        void* blob = nullptr;
        uint64_t bytes = 0;
        const float* data = c.metric == HNSW_COSINE ? Xn.data() : X.data();
        bad += check(hnsw_build(data, N, d, c.metric, &p, u.data(), &blob, &bytes) == HNSW_OK, "hnsw_build");
        if (!blob) continue;
        const std::string path = std::string(dir) + "/graph.hnsw";
        bad += check(hnsw_save_blob(blob, bytes, path.c_str()) == HNSW_OK, "hnsw_save_blob");
        void* back = nullptr;
        uint64_t back_bytes = 0;
        bad += check(hnsw_load_blob(path.c_str(), &back, &back_bytes) == HNSW_OK, "hnsw_load_blob");
        bad += check(back && back_bytes == bytes && std::memcmp(back, blob, bytes) == 0, "file round trip");
        hnsw_free_blob(back);
        // a flipped payload byte fails the checksum; a short blob fails the header
        std::vector<unsigned char> bent(static_cast<unsigned char*>(blob), static_cast<unsigned char*>(blob) + bytes);
        bent[bytes / 2] ^= 0x5A;
        bad += check(hnsw_save_blob(bent.data(), bytes, path.c_str()) == HNSW_ECORRUPT, "corrupt blob rejected");
        bad += check(hnsw_save_blob(blob, 64, path.c_str()) != HNSW_OK, "short blob rejected");
        hnsw_free_blob(blob);
    }
    // argument checks
    hnsw_build_params p{};
    p.M = 8;
    p.Mmax = 4;  // M > Mmax
    p.Mmax0 = 16;
    p.ef_construction = 32;
    p.mL = 0.5;
    void* blob = nullptr;
    uint64_t bytes = 0;
    bad += check(hnsw_build(X.data(), N, d, HNSW_L2SQ, &p, u.data(), &blob, &bytes) == HNSW_EINVAL, "M > Mmax");
    bad += check(hnsw_build(nullptr, N, d, HNSW_L2SQ, &p, u.data(), &blob, &bytes) == HNSW_EINVAL, "null data");
    void* none = nullptr;
    bad += check(hnsw_load_blob((std::string(dir) + "/missing.hnsw").c_str(), &none, &bytes) != HNSW_OK,
                 "missing file");
    std::printf("%s\n", bad ? "sanitize driver: failures" : "sanitize driver: ok");
    return bad ? 1 : 0;
}
