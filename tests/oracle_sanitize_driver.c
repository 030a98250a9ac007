/* Driver for the AddressSanitizer + UBSan build of the oracle
 * (oracle/hnsw_oracle.c), run by test_host_sanitizers.py: construction
 * (Alg. 1 with Alg. 3 / Alg. 4, both flags, sequential and in batches), the searches (Alg. 2, Alg. 5,
 * the traced form), the selection routines, brute force and the blob format
 * with its rejections, on small seeded inputs including the degenerate ones
 * (one element, K above N, ef = 1).  Exit status 0 when every call returned
 * what it should. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hnsw_oracle.h"

static uint64_t g_state = 0x243F6A8885A308D3ull;
static double next_unit(void) { /* (0, 1] */
    g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
    return ((double)((g_state >> 11) & ((1ull << 53) - 1)) + 1.0) / 9007199254740992.0;
}

static int bad = 0;
static void check(int ok, const char* what) {
    if (!ok) {
        fprintf(stderr, "FAILED: %s\n", what);
        ++bad;
    }
}

static void run(uint64_t N, uint32_t d, int metric, int heuristic, int extend, int keep) {
    float* X = (float*)malloc(sizeof(float) * (N * d + 1));
    double* u = (double*)malloc(sizeof(double) * (N + 1));
    for (uint64_t i = 0; i < N * d; ++i) X[i] = (float)floor(next_unit() * 16.0);
    if (metric == 1)
        for (uint64_t i = 0; i < N; ++i) {
            double s = 1e-3;
            for (uint32_t j = 0; j < d; ++j) s += (double)X[i * d + j] * X[i * d + j];
            for (uint32_t j = 0; j < d; ++j) X[i * d + j] = (float)(X[i * d + j] / sqrt(s));
        }
    for (uint64_t i = 0; i < N; ++i) u[i] = next_unit();
    orc_graph* g = orc_new(X, N, d, metric, 4, 4, 8, 24, 1.0 / log(4.0), heuristic, extend, keep);
    check(g != NULL, "orc_new");
    if (!g) goto out;
    check(orc_build(g, u) == 0, "orc_build");
    float q[64];
    uint32_t ids[80];
    double ds[80];
    orc_stats st;
    for (int t = 0; t < 20; ++t) {
        for (uint32_t j = 0; j < d; ++j) q[j] = (float)(next_unit() * 16.0);
        const int K = t % 4 == 0 ? 70 : 10;          /* K above N for the small graphs */
        const int ef = t % 3 == 0 ? 1 : 5 + 7 * t;   /* ef' = max(ef, K) */
        check(orc_knn_search(g, q, K, ef, ids, ds, &st) == 0, "orc_knn_search");
        uint32_t bid[80];
        double bd[80];
        orc_brute_force(X, N, d, metric, q, K, bid, bd);
        for (int k = 1; k < K; ++k) check(ds[k] >= ds[k - 1], "sorted result");
        double raw[64 * 6];
        uint32_t topk[64 * 10];
        int nc = 0;
        check(orc_knn_search_trace(g, q, 10, 40, 2, 64, raw, topk, &nc) == 0 && nc <= 64, "trace");
        if (N > 0) {
            uint32_t ep = orc_enter_point(g);
            uint32_t w[48];
            double wd[48];
            const int n = orc_search_layer(g, q, &ep, 1, 40, 0, w, wd, &st);
            check(n >= 1 && n <= 40, "orc_search_layer");
            const uint32_t m = orc_greedy_layer(g, q, ep, 0, &st);
            check(m < N, "orc_greedy_layer");
            uint32_t sel[8];
            const int ns = orc_select_heuristic(g, q, ORC_NONE, w, n, 6, 0, 1, 1, sel);
            check(ns >= 0 && ns <= 6, "orc_select_heuristic");
            check(orc_select_simple(g, q, w, n, 6, sel) == (n < 6 ? n : 6), "orc_select_simple");
        }
    }
    const uint64_t bytes = orc_blob_size(g);
    unsigned char* blob = (unsigned char*)malloc(bytes);
    check(orc_save_blob(g, blob, bytes) == 0, "orc_save_blob");
    check(orc_save_blob(g, blob, bytes - 1) != 0, "orc_save_blob short buffer");
    int err = 0;
    orc_graph* h = orc_load_blob(blob, bytes, &err);
    check(h != NULL, "orc_load_blob");
    if (h) {
        check(orc_n(h) == N && orc_enter_point(h) == orc_enter_point(g), "round trip");
        check(orc_set_data(h, X) == 0, "orc_set_data");
        orc_free(h);
    }
    blob[bytes - 1] ^= 0x11;
    h = orc_load_blob(blob, bytes, &err);
    check(h == NULL && err == 2, "checksum rejection");
    check(orc_load_blob(blob, 100, &err) == NULL, "short blob rejection");
    free(blob);
    orc_free(g);
    if (!extend) { /* the batched construction, growing and fixed batches */
        for (uint32_t batch = 0; batch < 8; batch += 7) {
            orc_graph* b = orc_new(X, N, d, metric, 4, 4, 8, 24, 1.0 / log(4.0), heuristic, 0, keep);
            check(b != NULL && orc_build_batched(b, u, N / 4, batch) == 0, "orc_build_batched");
            if (b && N > 0) check(orc_knn_search(b, q, 10, 20, ids, ds, &st) == 0, "search of the batched graph");
            orc_free(b);
            /* incremental: the first half in sequence, the rest in two insertions */
            if (N >= 4) {
                orc_graph* c = orc_new(X, N, d, metric, 4, 4, 8, 24, 1.0 / log(4.0), heuristic, 0, keep);
                check(c != NULL, "orc_new (incremental)");
                if (!c) continue;
                const uint64_t h = N / 2, m = h + (N - h) / 2;
                for (uint64_t i = 0; i < h; ++i) check(orc_insert(c, (uint32_t)i, orc_level_from_u(u[i], 1.0 / log(4.0))) == 0, "seed");
                check(orc_insert_batched(c, u + h, h, m - h, batch) == 0, "orc_insert_batched");
                check(orc_insert_batched(c, u + m, m, N - m, batch) == 0, "orc_insert_batched (second)");
                check(orc_insert_batched(c, u, 1, 1, batch) != 0, "insertion of present elements rejected");
                orc_free(c);
            }
        }
    }
out:
    free(X);
    free(u);
}

int main(void) {
    run(1, 5, 0, 1, 0, 0);  /* a single element: enter point, no links */
    run(9, 3, 0, 1, 0, 0);
    run(600, 7, 0, 1, 0, 0);
    run(600, 7, 0, 0, 0, 0);
    run(600, 7, 0, 1, 1, 1);
    run(600, 9, 1, 1, 0, 0);
    check(orc_new(NULL, 0, 0, 0, 4, 4, 8, 24, 1.0, 1, 0, 0) == NULL, "d = 0 rejected");
    printf("%s\n", bad ? "oracle sanitize driver: failures" : "oracle sanitize driver: ok");
    return bad ? 1 : 0;
}
