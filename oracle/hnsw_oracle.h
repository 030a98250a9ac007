/*
 * hnsw_oracle.h -- the ORACLE: a plain, slow, single-threaded CPU restatement of
 * Hierarchical NSW (Malkov & Yashunin, arXiv:1603.09320), Algorithms 1-5.
 *
 * This is TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call it.  It shares no
 * code, header, table or helper with the CUDA library under
 * paper_1603_09320_gb300/; the only interface the two have in common is the
 * serialised graph format described below, which each side reads and writes
 * with its own code.
 *
 * Precision: distances are accumulated in fp64 from the fp32 coordinates
 * (the paper fixes no precision).
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *  - Ties: every "nearest"/"furthest" comparison orders elements by the key
 *    (distance, id), lexicographically.  Alg. 2's break test is key(c) > key(f)
 *    and its insertion test is key(e) < key(f) or |W| < ef.
 *  - Alg. 4, the acceptance test ("e is closer to q compared to any element
 *    from R"): accept e iff dist(e,q) < dist(e,r) for every r in R (strict;
 *    R empty accepts).
 *  - keepPrunedConnections defaults to false, extendCandidates to false
 *    (Section 4, text after Alg. 5).
 *  - Levels: l = floor(-ln(u) * mL) with u in (0,1] supplied by the caller,
 *    one u per element in id order (the level draw of Alg. 1).
 *  - The first element becomes the enter point with its drawn level and no
 *    links.  The enter point changes only when l > L (Alg. 1, strictly).
 *  - Alg. 1's "ep <- W" between layers: all elements of W seed the next layer's search.
 *  - No self links and no duplicate links are ever stored.
 *  - Alg. 5 with ef < K runs the layer-0 search with ef' = max(ef, K); missing
 *    results (fewer than K reachable elements) are reported as id 0xFFFFFFFF
 *    and distance +inf.
 *  - Cosine distance is 1 - <q,x>; vectors are expected unit-normalised
 *    ("equivalent to L2 after normalization", Section 5.2).
 *
 * Serialised graph format "HNSWGB01" (little-endian), shared with the
 * library's own reader/writer:
 *   header, 128 bytes:
 *     0  char[8] magic "HNSWGB01"   8  u32 version (1)      12 u32 metric (0 L2SQ, 1 COSINE)
 *     16 u64 N                      24 u32 d                 28 u32 M
 *     32 u32 Mmax                   36 u32 Mmax0             40 u32 maxlevel (level of ep)
 *     44 u32 ep (0xFFFFFFFF if N=0) 48 u32 flags (bit0 heuristic, bit1 extendCandidates,
 *                                                bit2 keepPrunedConnections)
 *     52 u32 efConstruction         56 f64 mL                64 u64 n_upper_rows
 *     72 u64 checksum (64-bit FNV-1a over every payload byte)  80..127 zero
 *   payload, in this order, each section starting on a 16-byte boundary
 *   (zero padding between sections):
 *     f32 data[N][d]
 *     u8  level[N]
 *     u32 nbr0[N][Mmax0]             layer-0 lists, valid ids first, then 0xFFFFFFFF
 *     u32 nbrU[n_upper_rows][Mmax]   for each element in id order, one row per
 *                                    layer 1..level[i]; same padding rule
 */
#ifndef HNSW_ORACLE_H
#define HNSW_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NONE 0xFFFFFFFFu

typedef struct orc_graph orc_graph;

typedef struct {
    uint64_t n_dist;   /* distance evaluations (every call of the distance function) */
    uint64_t n_hops0;  /* elements extracted from C and expanded on layer 0 */
    uint64_t n_hopsU;  /* elements expanded on layers >= 1 */
} orc_stats;

/* New empty graph over N elements of dimension d (data copied, fp32 row-major).
 * metric 0 = squared L2, 1 = cosine (1 - <q,x>). Returns NULL on bad args. */
orc_graph* orc_new(const float* data, uint64_t N, uint32_t d, int metric,
                   uint32_t M, uint32_t Mmax, uint32_t Mmax0, uint32_t efC, double mL,
                   int heuristic, int extend_candidates, int keep_pruned);
void orc_free(orc_graph* g);

/* Alg. 1, the level draw: l = floor(-ln(u) * mL). */
int orc_level_from_u(double u, double mL);

/* Alg. 1: insert element `id` (its vector is row `id` of the data) at level l. */
int orc_insert(orc_graph* g, uint32_t id, int level);

/* Inserts elements 0..N-1 in order, element i at level orc_level_from_u(u[i], mL). */
int orc_build(orc_graph* g, const double* u);

/* Alg. 1 with the layer-0 insertions grouped in batches (the parallel
 * construction of Section 4.1 in batch form).  Levels come from u as in
 * orc_build.  The seed -- every element of level >= 1 and the elements with
 * id < max(n_first, 1) -- is inserted first, in id order, by orc_insert.  The other
 * elements (all of level 0) follow in id order, in batches of `batch`
 * elements, or with batch = 0 of min(32768, max(64, remaining count at the
 * start), remaining, max(64, inserted / 16)) elements.  For a batch:
 *  1. every element q searches the graph as it stands before the batch:
 *     Alg. 5 with K = ef = efConstruction (Alg. 1's descent and layer search, on layer 0);
 *  2. q's layer-0 list becomes SELECT-NEIGHBORS(q, W, M) (Alg. 1's own links
 *     11's forward half), in selection order;
 *  3. each element e selected by batch elements takes them into its list,
 *     in ascending id: appended when they fit within Mmax0, otherwise the list
 *     becomes SELECT-NEIGHBORS(e, eConn, Mmax0) over all of eConn, the old
 *     members and every new one (Alg. 1's reverse links and shrink).
 * Elements of one batch do not see one another; batch = 1 is Alg. 1 applied
 * in the order seed, then the rest.  The batch sizes are a free parameter of
 * this form (the paper's parallel construction fixes none); the growing
 * schedule keeps each batch at most 1/16 of the elements already present.
 * extendCandidates must be off. */
int orc_build_batched(orc_graph* g, const double* u, uint64_t n_first, uint32_t batch);

/* orc_build_batched with explicit batch sizes: batch j holds sizes[j]
 * elements (the last size repeats; every size clipped to what remains; a
 * zero size is an error). */
int orc_build_batched_sizes(orc_graph* g, const double* u, uint64_t n_first, const uint32_t* sizes,
                            uint64_t n_sizes);

/* Incremental insertion of elements first..first+n-1 (rows of the data, not
 * inserted yet) into a graph holding exactly elements 0..first-1, levels
 * from u[0..n): 1. the new elements of level >= 1 take their layer-0 links
 * in batches as in orc_build_batched, searching through the upper layers as
 * they stand; 2. their upper layers follow one at a time in id order (Alg. 1
 * on layers >= 1, enter point updated as Alg. 1 does); 3. the new elements of
 * level 0 are inserted on layer 0 in batches.  Batches as in
 * orc_build_batched (0: the growing schedule, starting from the elements
 * present). */
int orc_insert_batched(orc_graph* g, const double* u, uint64_t first, uint64_t n, uint32_t batch);

/* Alg. 5: K nearest of q; ids/dists have K slots; missing -> ORC_NONE/+inf. */
int orc_knn_search(const orc_graph* g, const float* q, int K, int ef,
                   uint32_t* ids, double* dists, orc_stats* st);

/* Alg. 5 recording the layer-0 search state after every T-th expansion once
 * |W| >= K (up to max_checks records): raw[c][6] = nearest, furthest and K-th
 * nearest distance of W, layer-0 distance evaluations so far, the layer-0
 * enter point's distance, expansions since the K-th nearest last improved;
 * topk[c][K] = ids of the K nearest.  Used to check the learned-stop
 * features; the search itself is unchanged. */
int orc_knn_search_trace(const orc_graph* g, const float* q, int K, int ef, int T, int max_checks,
                         double* raw, uint32_t* topk, int* n_checks);

/* Alg. 2 on layer lc from enter points ep[0..n_ep); returns |W| and writes W
 * sorted ascending by key into out_ids/out_dists (capacity >= ef). */
int orc_search_layer(const orc_graph* g, const float* q, const uint32_t* ep, int n_ep,
                     int ef, int lc, uint32_t* out_ids, double* out_dists, orc_stats* st);

/* Steepest-descent form of Alg. 2 with ef = 1 (used to check the lemma that the
 * two coincide under key order): returns the local minimum reached from ep. */
uint32_t orc_greedy_layer(const orc_graph* g, const float* q, uint32_t ep, int lc, orc_stats* st);

/* Alg. 3 / Alg. 4 as standalone routines over candidate lists (base is a vector
 * `base` with optional element id base_id to exclude; cand ids refer to data rows).
 * Writes at most M selected ids (in selection order) and returns their number. */
int orc_select_simple(const orc_graph* g, const float* base, const uint32_t* cand,
                      int n_cand, int M, uint32_t* out);
int orc_select_heuristic(const orc_graph* g, const float* base, uint32_t base_id,
                         const uint32_t* cand, int n_cand, int M, int lc,
                         int extend_candidates, int keep_pruned, uint32_t* out);

/* Distance between a vector and data row i (fp64). */
double orc_dist_to(const orc_graph* g, const float* q, uint32_t i);

/* Replaces the N x d stored vectors, keeping every link: the same
 * multilayer graph, searched over other coordinates (e.g. the dequantised
 * rows of a lossy storage form).  Returns 0, or -1 for a null argument. */
int orc_set_data(orc_graph* g, const float* data);

/* Inspection. */
uint64_t orc_n(const orc_graph* g);
int orc_level(const orc_graph* g, uint32_t i);
uint32_t orc_enter_point(const orc_graph* g);
int orc_max_level(const orc_graph* g);
int orc_neighbors(const orc_graph* g, uint32_t i, int lc, uint32_t* out, int cap);

/* Serialisation (format above). orc_blob_size gives the exact byte count. */
uint64_t orc_blob_size(const orc_graph* g);
int orc_save_blob(const orc_graph* g, void* out, uint64_t cap);
orc_graph* orc_load_blob(const void* blob, uint64_t bytes, int* err);

/* Exact k-NN by scanning all N rows (fp64 distances, key order). */
void orc_brute_force(const float* data, uint64_t N, uint32_t d, int metric,
                     const float* q, int K, uint32_t* ids, double* dists);

#ifdef __cplusplus
}
#endif
#endif
