/*
 * hnsw.h -- C ABI of the GB300 batched HNSW search library (libhnsw_gb300.so).
 *
 * Hierarchical Navigable Small World graphs (Malkov & Yashunin,
 * arXiv:1603.09320).  The library builds the multilayer graph on the host
 * (Alg. 1 INSERT with Alg. 4 SELECT-NEIGHBORS-HEURISTIC, multi-threaded as in
 * Section 4.1) or with its layer-0 insertions on the GPU, answers batches of
 * K-NN queries on one GPU (Alg. 5 K-NN-SEARCH: greedy ef=1 descent through
 * layers L..1 followed by the ef-bounded SEARCH-LAYER of Alg. 2 on layer 0),
 * and inserts new elements into a resident index while it serves searches,
 * in hand-written sm_103a CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Return an hnsw_status; no C++ exception crosses the ABI.  On failure,
 *    hnsw_last_error() gives a message for the calling thread.
 *  - The caller owns query and output buffers; the library owns the memory of
 *    an index (device memory allocated by hnsw_upload_index and
 *    hnsw_reserve, freed by hnsw_free_index) and of blobs it returns (freed
 *    by hnsw_free_blob).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *  - Element ids are uint32; 0xFFFFFFFF (HNSW_NO_ID) marks "no element".
 *  - Distances are squared L2, or cosine distance 1 - <q,x> on unit vectors
 *    (Section 5.2: cosine similarity is L2 after normalisation).
 *  - Keys (distance, id) order every comparison, lexicographically; this makes
 *    a result a deterministic function of the graph and the distances.
 */
#ifndef HNSW_GB300_H
#define HNSW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HNSW_ABI_VERSION 2
#define HNSW_NO_ID 0xFFFFFFFFu

typedef enum {
    HNSW_OK = 0,
    HNSW_EINVAL = 1,   /* bad argument: null pointer, k <= 0, ef < 1, n < 0, size limits */
    HNSW_ENOMEM = 2,   /* host or device allocation failed */
    HNSW_ECUDA = 3,    /* a CUDA call or kernel launch failed (message has the CUDA error) */
    HNSW_ECORRUPT = 4, /* a graph blob failed validation (magic, checksum, links, levels) */
    HNSW_ETIMEOUT = 5, /* a bounded device-side wait ran out */
    HNSW_EBUSY = 6,    /* resource in use (e.g. server queue full, request already on the device) */
    HNSW_ECANCELED = 7 /* the request was cancelled before it reached the device */
} hnsw_status;

typedef enum { HNSW_L2SQ = 0, HNSW_COSINE = 1 } hnsw_metric;

/* Storage type of the vectors on the device.  F32 is exact.  BF16 and F16
 * are round-to-nearest-even from fp32; FP8E4M3 stores code = RNE(x / s_x)
 * with a per-vector fp32 scale s_x = max_i |x_i| / 448 (saturating).
 * Distances are always accumulated in fp32 from the dequantised values. */
typedef enum { HNSW_F32 = 0, HNSW_BF16 = 1, HNSW_FP8E4M3 = 2, HNSW_F16 = 3 } hnsw_dtype;

typedef struct hnsw_index hnsw_index;

/* ------------------------------------------------------------------------ */
/* Host-side graph construction                                              */
/* ------------------------------------------------------------------------ */

/* Construction parameters (Alg. 1 inputs; Mmax0 from Section 4.1, where 2*M is
 * recommended).  mL is the level normalisation (1/ln M recommended). */
typedef struct {
    uint32_t M;                 /* links made per inserted element (Alg. 1) */
    uint32_t Mmax;              /* cap on links per element on layers >= 1 */
    uint32_t Mmax0;             /* cap on layer 0 */
    uint32_t ef_construction;   /* beam width of SEARCH-LAYER during insertion */
    double mL;                  /* level normalisation factor */
    int32_t heuristic;          /* 1: Alg. 4, 0: Alg. 3 */
    int32_t extend_candidates;  /* Alg. 4 flag */
    int32_t keep_pruned;        /* Alg. 4 flag */
    int32_t n_threads;          /* <= 0: all hardware threads */
} hnsw_build_params;

/* Builds the HNSW graph of `data` (fp32 row-major [N][d], host memory) by
 * concurrent insertion of elements 0..N-1 (Alg. 1; Section 4.1: parallel
 * construction with per-element locks and one lock for the enter point).
 * Element i gets level floor(-ln(level_u[i]) * mL) (the level draw of Alg. 1); level_u
 * holds N host doubles in (0,1].  With n_threads = 1 elements are inserted in
 * id order, which is exactly Alg. 1 applied sequentially.
 * On success *out_blob receives a library-allocated graph blob in the
 * "HNSWGB01" format (below) of *out_bytes bytes; free it with hnsw_free_blob.
 * Errors: HNSW_EINVAL (null pointers, d = 0, N >= 2^31, M > Mmax or Mmax0,
 * Mmax0 > 64, mL <= 0), HNSW_ENOMEM. */
hnsw_status hnsw_build(const float* data, uint64_t N, uint32_t d, hnsw_metric metric,
                       const hnsw_build_params* params, const double* level_u,
                       void** out_blob, uint64_t* out_bytes);
void hnsw_free_blob(void* blob);

/* Bulk construction with the layer-0 insertions on the GPU (Alg. 1 with Alg.
 * 4 or Alg. 3 as SELECT-NEIGHBORS; parallel construction, Section 4.1).  On
 * layers >= 1 Alg. 1 involves only the elements of level >= 1, so a seed --
 * every element of level >= 1 and the first min(N, 4096) elements, in id
 * order -- is built by hnsw_build (same parameters, n_threads as given; with
 * n_threads = 1 its upper layers are exactly Alg. 1 applied to the seed).
 * The other elements (all of level 0) are then inserted into layer 0 on the
 * current device in id order, in batches of at most 1/16 of the elements
 * already inserted (64..32768): each element of a batch searches the graph as
 * it stood before the batch (SEARCH-LAYER with ef = efConstruction on layer
 * 0 after the upper-layer descent), links to the M neighbours its selection
 * keeps, and each element it links to takes it into its list, shrinking the
 * list with the same selection over all its old and new members when it
 * exceeds Mmax0 (Alg. 1's shrink).  Elements of one batch do not search one
 * another, so the graph differs from sequential insertion; it has the same
 * structure and format as hnsw_build's (validated the same way on upload).
 * data and level_u are host memory as for hnsw_build; device memory of about
 * the index size (fp32) plus per-batch buffers is allocated and freed inside
 * the call; work is issued on `stream`, which is synchronised before return.
 * Errors: those of hnsw_build; HNSW_EINVAL also for d > 256,
 * ef_construction > 1024 or extend_candidates set; HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_build_gpu(const float* data, uint64_t N, uint32_t d, hnsw_metric metric,
                           const hnsw_build_params* params, const double* level_u, void* stream,
                           void** out_blob, uint64_t* out_bytes);

/* Graph blob format "HNSWGB01" (little-endian), the interface shared with
 * other producers of graphs (e.g. test tools):
 *   header, 128 bytes:
 *     0 char[8] "HNSWGB01"  8 u32 version=1  12 u32 metric  16 u64 N  24 u32 d
 *     28 u32 M  32 u32 Mmax  36 u32 Mmax0  40 u32 maxlevel  44 u32 enter point
 *     48 u32 flags (bit0 heuristic, bit1 extendCandidates, bit2 keepPruned)
 *     52 u32 efConstruction  56 f64 mL  64 u64 n_upper_rows
 *     72 u64 FNV-1a-64 of all payload bytes   80..127 zero
 *   payload, each section 16-byte aligned (zero padded):
 *     f32 data[N][d]; u8 level[N]; u32 nbr0[N][Mmax0];
 *     u32 nbrU[n_upper_rows][Mmax] (element-major, layers 1..level[i]);
 *   lists hold their valid ids first, then 0xFFFFFFFF. */

/* Graph files.  hnsw_save_blob validates the blob (as hnsw_upload_index does)
 * and writes its bytes to `path` through a temporary file `path`.tmp renamed
 * over `path`, so that an interrupted save leaves no partial graph under that
 * name.  hnsw_load_blob reads and validates a file; on success *out_blob is a
 * library-allocated blob of *out_bytes bytes, freed with hnsw_free_blob.
 * Errors: HNSW_EINVAL (null arguments, the file cannot be opened, created
 * or written), HNSW_ECORRUPT (failed validation, short or empty file),
 * HNSW_ENOMEM. */
hnsw_status hnsw_save_blob(const void* blob, uint64_t blob_bytes, const char* path);
hnsw_status hnsw_load_blob(const char* path, void** out_blob, uint64_t* out_bytes);

/* ------------------------------------------------------------------------ */
/* Device index                                                              */
/* ------------------------------------------------------------------------ */

/* Validates a graph blob (host memory) and packs it into device memory:
 * vectors as `storage` rows padded to a multiple of 16 bytes, the layer-0
 * adjacency [N][Mmax0], the upper-layer rows with a per-element offset, and
 * the enter point and top level.  keep_fp32_for_rerank additionally keeps
 * an fp32 copy of the vectors for hnsw_search_ex's exact rerank.
 * The copy is issued on `stream`; the call synchronises it before returning.
 * Errors: HNSW_EINVAL, HNSW_ECORRUPT (blob fails validation: magic, version,
 * size, checksum, ids out of range, self or duplicate links, links to
 * elements absent from a layer, enter point not on the top level),
 * HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_upload_index(const void* graph_blob, uint64_t blob_bytes, hnsw_dtype storage,
                              int keep_fp32_for_rerank, void* stream, hnsw_index** out);

hnsw_status hnsw_free_index(hnsw_index* index);

/* ------------------------------------------------------------------------ */
/* Incremental insertion into a resident index (continuous indexing; Alg. 1) */
/* ------------------------------------------------------------------------ */
/* Reserves room for `capacity` elements (>= the current count, < 2^31) and
 * the upper-layer rows they will need (expected 1/(M-1) per element, twice
 * that reserved, plus 1,024): the device arrays are reallocated and the
 * adjacency is kept in two versions from then on.  Synchronises the device;
 * not to be called while other calls on the index are running.
 * Errors: HNSW_EINVAL, HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_reserve(hnsw_index* index, uint64_t capacity, void* stream);

/* Inserts n elements into a resident index as Alg. 1 does, with the graph's
 * own parameters (M, Mmax, Mmax0, efConstruction, mL, selection flags from
 * its header): ids count..count+n-1 in order, vectors data[n][d] (host or
 * device memory; unit-normalised for COSINE), level_u[n] host doubles in
 * (0,1] (level = floor(-ln u * mL)).  The new elements of level >= 1 are
 * linked into layer 0 first (searching through the existing upper layers),
 * then into their upper layers one at a time in id order (a new top level
 * makes the element the enter point), then the elements of level 0 are
 * linked into layer 0 in batches of at most 1/16 of the elements present;
 * elements of one batch do not search one another (see hnsw_build_gpu).
 * Concurrency: searches may be issued on other streams and host threads
 * during the call.  The call first synchronises the device (so that no
 * search still reads the adjacency version it is about to overwrite), writes
 * a copy of the adjacency, and publishes it when its work is done: a search
 * launched before the publication sees the graph without the new elements,
 * a search launched after it sees all of them.  Inserts on one index are
 * serialised.  Needs the fp32 vectors (F32 storage, or keep_fp32_for_rerank)
 * and a non-empty index built by hnsw_build or hnsw_build_gpu without
 * extendCandidates.  Work is issued on `stream`, synchronised before return;
 * issue it on a stream created non-blocking (not the legacy default stream,
 * which would serialise the searches of other streams behind the call).
 * Errors: HNSW_EINVAL (null pointers, no reserved capacity, capacity or
 * upper rows exceeded, level_u outside (0,1], d > 256, fp32 vectors absent),
 * HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_insert(hnsw_index* index, const float* data, uint64_t n, const double* level_u, void* stream);

/* The index's current graph as a library-allocated "HNSWGB01" blob (free
 * with hnsw_free_blob): fp32 vectors (needs F32 storage or the fp32 copy),
 * levels, both adjacencies and the enter point.  Serialised with inserts. */
hnsw_status hnsw_index_to_blob(hnsw_index* index, void** out_blob, uint64_t* out_bytes);

typedef struct {
    uint64_t N;
    uint32_t d, d_pad, row_bytes;
    int32_t metric, storage, has_fp32;
    uint32_t M, Mmax, Mmax0;
    int32_t max_level;
    uint32_t enter_point;
    uint64_t n_upper_rows;
    uint64_t device_bytes;   /* the index arrays */
    uint64_t staging_bytes;  /* device buffers hnsw_search_ex holds for calls with host
                              * pointers (one per stream); hnsw_search_noalloc never adds any */
} hnsw_index_info;

/* Copies the index's shape and sizes into *out (host).  Never touches the
 * device.  Errors: HNSW_EINVAL (null pointer). */
hnsw_status hnsw_get_index_info(const hnsw_index* index, hnsw_index_info* out);

/* ------------------------------------------------------------------------ */
/* Search                                                                    */
/* ------------------------------------------------------------------------ */

/* Alg. 5 K-NN-SEARCH for n queries (fp32 row-major [n][d]; for COSINE the
 * queries must be unit-normalised).  The layer-0 beam uses ef' = max(ef, k).
 * Writes out_ids[n][k] and out_dists[n][k] sorted ascending by (dist, id);
 * slots beyond the reachable elements hold HNSW_NO_ID / +inf.
 * Pointers may be host or device memory (detected per pointer).  With only
 * device pointers the call is asynchronous on `stream`; if any pointer is
 * host memory the call copies through a library-owned device buffer of that
 * stream (one per stream, for up to 16 streams per index) and synchronises
 * `stream` before returning.  Calls on different streams may run
 * concurrently from several host threads; concurrent host-memory calls on
 * one index and one stream are not supported.
 * Errors: HNSW_EINVAL (null index/pointers with n > 0, k < 1, ef < 1, n < 0,
 * k > 1024, ef' > the kernel limit 1024), HNSW_ECUDA. */
hnsw_status hnsw_search(hnsw_index* index, const float* queries, int64_t n, int32_t k, int32_t ef,
                        uint32_t* out_ids, float* out_dists, void* stream);

/* Per-query counters (the paper's cost measure is the number of distance
 * computations, Section 5.1). */
typedef struct {
    uint32_t n_eval;    /* distance evaluations on all layers */
    uint32_t n_exp0;    /* layer-0 expansions (elements taken from C) */
    uint32_t n_stepU;   /* elements expanded on layers >= 1 */
    uint32_t flags;     /* bit0: visited set overflowed (lossy, results unaffected);
                           bit1: stopped early by the learned stop;
                           bit2: the bounds-checked search met an element id, upper-row
                           index or work index out of range and left this query's
                           search there (its results are what W held) */
} hnsw_query_stats;

typedef struct {
    int32_t k;
    int32_t ef;
    int32_t rerank;          /* 1: recompute fp32 distances of all ef' final candidates
                                from the fp32 copy and return the top k of those */
    int32_t visited_log2;    /* log2 of visited-set slots per query; 0 = automatic: the
                                largest set from 2^8 up to 8-16 slots per beam entry
                                (at most 2^12) that keeps as many warps resident as
                                2^8 slots do (the set may forget elements, which only
                                repeats evaluations; results are the same at any size) */
    float stop_threshold;    /* learned stop: in (0,1) stop the layer-0 beam when the stop
                                network's sigmoid exceeds it (needs hnsw_set_stop_model);
                                <= 0 or >= 1: off, the plain search */
    int32_t stop_period;     /* learned stop / trace: check every stop_period layer-0
                                expansions (<= 0: 8 for the stop, 4 for traces;
                                above 65535: HNSW_EINVAL) */
    int32_t schedule;        /* order of the work (results and counters unchanged; both
                                scheduled forms take stream-ordered scratch, 16 bytes per
                                query):
                                0: automatic -- deferral (3) for batches of 33 to 2^24
                                queries, else one pass;
                                1: one pass in input order;
                                2: two passes -- the upper-layer descent of all queries
                                first, then the layer-0 beams in order of decreasing
                                descent distance;
                                3: deferral -- one pass in which a query whose descent
                                ends nearer than the mean of the descents before it is set
                                aside and its layer-0 beam run once the input queue is
                                drained, so that the long searches start first.  Its
                                device-side wait is bounded: a wait that runs out (never
                                in normal operation) leaves that claim and is reported as
                                HNSW_ETIMEOUT by this call, when it synchronises (host
                                buffers), else by the next call on the index that does.
                                Other values: HNSW_EINVAL */
    int32_t check_bounds;    /* 1: the bounds-checked search -- every element id read from
                                the graph is checked against N and every upper-row index
                                against the rows allocated before it is used; a query
                                that meets a bad one leaves its search and sets stats
                                flag bit 2 (no device fault).  Slower; for diagnosing a
                                suspect index.  Built for f32 rows of up to 32 chunks and
                                bf16 rows of up to 16 (d <= 128); other storage, or with
                                the learned stop: HNSW_EINVAL */
} hnsw_search_params;

/* hnsw_search with the options above and optional per-query counters
 * (stats may be NULL; host or device memory, [n]).  Same memory and stream
 * rules as hnsw_search.  Errors: those of hnsw_search; HNSW_EINVAL also for a
 * null params, visited_log2 outside [5,15] (when not 0), rerank without the
 * fp32 copy, stop_period above 65535. */
hnsw_status hnsw_search_ex(hnsw_index* index, const hnsw_search_params* params,
                           const float* queries, int64_t n, uint32_t* out_ids, float* out_dists,
                           hnsw_query_stats* stats, void* stream);

/* Test hook for the bounded wait of the deferral (schedule 3): while `on` is
 * non-zero, searches on this index withhold the decision of query 0, so that
 * claims waiting for the final count of deferred queries run into their limit
 * (2^20 polls, 0.1 to 1 s), leave, and the call reports HNSW_ETIMEOUT; every query is
 * still searched and its results are complete.  No device fault and no trap.
 * Not for production use.  Errors: HNSW_EINVAL (null index). */
hnsw_status hnsw_debug_hold_decisions(hnsw_index* index, int32_t on);

/* ------------------------------------------------------------------------ */
/* Learned early stop of the layer-0 beam (an addition: the paper has none)  */
/* ------------------------------------------------------------------------ */
/* A network 6 -> 64 -> 64 -> 1 (ReLU, fp16 weights, fp32 arithmetic) reads
 * the search state every stop_period layer-0 expansions and predicts whether
 * the current top-k of W is already final.  Features (d1 = distance of the
 * element where the upper-layer descent ended, clamped below by 1e-12):
 * log1p(best/d1), log1p(worst/d1), log1p(layer-0 distance evaluations),
 * log1p(d1), log1p(expansions since the k-th best entry last improved,
 * saturating at 65535),
 * log1p(kth/d1), where best/worst/kth are distances of W's entries.
 * Weights: 4,673 fp16 values in the order W1 (64x6, row-major out x in), b1,
 * W2 (64x64), b2, w3 (64), b3; normalisation: mean[6] then std[6], applied as
 * (x - mean) / std before the first layer. */
#define HNSW_STOP_NPARAM 4673

/* Installs (or replaces) the index's stop network; host arrays, copied.
 * Errors: HNSW_EINVAL (null argument, a std <= 0), HNSW_ENOMEM, HNSW_ECUDA.
 * hnsw_clear_stop_model removes it (searches with a threshold then run the
 * plain search); HNSW_EINVAL for a null index. */
hnsw_status hnsw_set_stop_model(hnsw_index* index, const float* norm12, const uint16_t* w_fp16);
hnsw_status hnsw_clear_stop_model(hnsw_index* index);

/* Runs the search of hnsw_search_ex without stopping early and records, at
 * every check (every stop_period layer-0 expansions once W holds k entries),
 * the six features into feats[n][max_checks][6], the ids of W's current top
 * k into topk[n][max_checks][k] and, when logits is not NULL and the index
 * has a stop network, its logit into logits[n][max_checks]; n_checks[n]
 * receives the number of checks recorded (at most max_checks).  All buffers
 * are device memory; asynchronous on stream.  Errors: HNSW_EINVAL (null
 * index or params, n < 0, max_checks < 1, k or ef out of range as in
 * hnsw_search, host buffers, rerank without the fp32 copy, stop_period above
 * 65535), HNSW_ECUDA. */
hnsw_status hnsw_search_trace(hnsw_index* index, const hnsw_search_params* params, const float* queries,
                              int64_t n, int32_t max_checks, float* feats, uint32_t* topk, float* logits,
                              int32_t* n_checks, uint32_t* out_ids, float* out_dists,
                              hnsw_query_stats* stats, void* stream);

/* Gradient of the mean binary cross-entropy of the network over n samples
 * (x: device [n][6] raw features, y: device [n] labels in {0,1}) at the given
 * fp16 weights and normalisation (host); writes grad_out[4673] and the mean
 * loss (host).  Synchronous.  Errors: HNSW_EINVAL (null argument, n < 1, x or
 * y not device memory), HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_stop_grad(const float* x, const float* y, int64_t n, const float* norm12,
                           const uint16_t* w_fp16, float* grad_out, float* loss_out, void* stream);

typedef struct {
    int32_t epochs;       /* passes over the samples */
    int32_t batch;        /* samples per optimiser step, a multiple of 128 */
    float lr;             /* Adam step size */
    float beta1, beta2, eps;  /* Adam constants (0: 0.9, 0.999, 1e-8) */
    float weight_decay;   /* L2 coefficient added to the gradient */
    uint64_t seed;        /* sample visiting order */
} hnsw_stop_train_params;

/* Trains the network on the GPU from w_init (host fp16): normalisation from
 * the samples' mean and std, then epochs of Adam on fp32 master weights with
 * fp16 working weights.  Writes norm_out[12], w_out[4673] (host) and, when
 * not NULL, the mean loss of every epoch.  x, y: device memory as in
 * hnsw_stop_grad.  Synchronous.  Errors: HNSW_EINVAL (null argument, n < 1,
 * epochs < 1, batch not a positive multiple of 128, lr <= 0, x or y not
 * device memory), HNSW_ENOMEM, HNSW_ECUDA. */
hnsw_status hnsw_stop_train(const float* x, const float* y, int64_t n, const hnsw_stop_train_params* params,
                            const uint16_t* w_init, float* norm_out, uint16_t* w_out, float* loss_per_epoch,
                            void* stream);

/* hnsw_search without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc while
 * searching -- a process whose device memory is all reserved by another
 * allocator (e.g. a framework's caching allocator), or a latency-critical
 * path that must avoid cudaMalloc/cudaFree, which synchronise the device.
 * Same arguments and results as hnsw_search (ef' = max(ef, k)).  Host-memory
 * buffers are staged through one fixed 16 MiB device array that the library
 * holds on every GPU it is loaded on until exit; a batch whose host buffers
 * need more than that (queries n*d*4 bytes, ids and distances n*k*4 bytes
 * each, 256-byte aligned, plus 256 bytes for the kernel's work counter) is
 * rejected with HNSW_EINVAL -- pass device buffers or split the batch.  The
 * first call on each device looks up that array's address (make it before
 * any stream capture).  All calls share the array: calls whose GPU work
 * overlaps race, so issue them one after another.  The index must have been
 * uploaded (which allocates) beforehand, on the current device.
 * Errors: as hnsw_search, plus HNSW_EINVAL for the size limit. */
hnsw_status hnsw_search_noalloc(hnsw_index* index, const float* queries, int64_t n, int32_t k, int32_t ef,
                                uint32_t* out_ids, float* out_dists, void* stream);

/* ------------------------------------------------------------------------ */
/* Data-sharded search (Section 6 discusses distributing HNSW by partitioning */
/* the data)                                                                  */
/* ------------------------------------------------------------------------ */
/* The exchange step of data-sharded search.  Shard s holds its own graph over
 * the elements with global ids id_base[s] .. id_base[s] + N_s - 1 (disjoint
 * ranges) and has answered n queries with its own k nearest, in local ids:
 * shard_ids[s][q][j], shard_dists[s][q][j] ([n_shards][n][k] row-major,
 * each list sorted ascending by (distance, local id) and padded with
 * HNSW_NO_ID, as hnsw_search writes them).  Writes, per query, the k smallest
 * keys (distance, global id) over all shards' lists -- the answer of the
 * whole data set's shards taken together -- to out_ids[n][k] (global ids) and
 * out_dists[n][k], padded with HNSW_NO_ID / +inf when the shards hold fewer
 * than k.  id_base is host memory (n_shards values; every global id must be
 * below 2^32 - 1); the four buffers are device memory of the current device;
 * asynchronous on `stream`.
 * Errors: HNSW_EINVAL (n_shards outside [1, 32], n < 0, k outside [1, 1024],
 * null or non-device buffers), HNSW_ECUDA. */
hnsw_status hnsw_merge_topk(const uint32_t* shard_ids, const float* shard_dists, int32_t n_shards,
                            const uint32_t* id_base, int64_t n, int32_t k, uint32_t* out_ids, float* out_dists,
                            void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching over resident indexes (an addition; the      */
/* paper has no serving component)                                           */
/* ------------------------------------------------------------------------ */
/* A server owns `n_slots` CUDA streams ("slots") and one device arena of
 * `memory_budget` bytes (0: a quarter of the free device memory, at most
 * 4 GiB).  Submitted requests wait in a FIFO; the request at its head is
 * admitted as soon as a slot is free and its device buffers (queries n*d*4
 * bytes, ids and distances n*k*4 bytes each, 256-byte aligned) fit in the
 * arena.  Requests admitted while others are on the GPU run concurrently
 * with them.  Results go to the caller's host buffers, which must stay valid
 * until hnsw_server_wait returns for the ticket.  Indexes stay resident and
 * owned by the caller (free them after hnsw_server_destroy). */
typedef struct hnsw_server hnsw_server;

typedef struct {
    int32_t n_slots;          /* 1..64 concurrent requests on the device */
    uint64_t memory_budget;   /* device bytes for request buffers, 0: automatic */
} hnsw_server_params;

typedef struct {
    int32_t index;            /* id returned by hnsw_server_add_index */
    int64_t n;                /* queries in this request (>= 1) */
    int32_t k, ef, rerank;    /* as in hnsw_search_params */
    float stop_threshold;     /* learned stop, as in hnsw_search_params */
    int32_t stop_period;
    const float* queries;     /* host [n][d] */
    uint32_t* out_ids;        /* host [n][k] */
    float* out_dists;         /* host [n][k] */
} hnsw_request;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t queued, in_flight;          /* waiting for admission / on the device */
    uint64_t bytes_in_use, budget;       /* device arena */
    uint64_t cancelled;                  /* removed from the queue by hnsw_server_cancel */
} hnsw_server_stats;

hnsw_status hnsw_server_create(const hnsw_server_params* params, hnsw_server** out);
hnsw_status hnsw_server_add_index(hnsw_server* server, hnsw_index* index, int32_t* index_id);
/* Errors: HNSW_EINVAL (bad request, unknown index, larger than the whole
 * budget), HNSW_EBUSY (server stopping). */
hnsw_status hnsw_server_submit(hnsw_server* server, const hnsw_request* request, uint64_t* ticket);
hnsw_status hnsw_server_poll(hnsw_server* server, uint64_t ticket, int32_t* done);
/* Waits until the request's results are in the caller's buffers (timeout_ms
 * < 0: no limit; HNSW_ETIMEOUT when it runs out, the request continues).  On
 * return other than HNSW_ETIMEOUT the ticket is consumed; latency_ms (may be
 * NULL) receives submit-to-completion time.  A request that failed on the
 * device returns its error here. */
hnsw_status hnsw_server_wait(hnsw_server* server, uint64_t ticket, int32_t timeout_ms, double* latency_ms);
/* Cancels a request that is still waiting for admission: it leaves the queue,
 * its device work is never issued and its output buffers are not written;
 * hnsw_server_wait on its ticket then returns HNSW_ECANCELED (and consumes
 * the ticket).  A request already admitted (its launch may be on the device)
 * or complete is not cancelled: HNSW_EBUSY.  Errors: HNSW_EINVAL (null
 * server, unknown ticket), HNSW_EBUSY. */
hnsw_status hnsw_server_cancel(hnsw_server* server, uint64_t ticket);
hnsw_status hnsw_server_get_stats(hnsw_server* server, hnsw_server_stats* out);
/* Completes every submitted request, then releases the server's streams and
 * arena. */
hnsw_status hnsw_server_destroy(hnsw_server* server);

/* Replays a request trace: submits reqs[i] at arrival_s[i] seconds after the
 * call starts (busy-waiting between arrivals), then waits for all of them
 * (timeout_ms per request) and writes each submit-to-completion latency to
 * latency_ms[i] and, when submit_s is not NULL, the actual submit time.
 * Returns the first error of a request, if any. */
hnsw_status hnsw_server_replay(hnsw_server* server, const hnsw_request* reqs, const double* arrival_s, int64_t n,
                               int32_t timeout_ms, double* latency_ms, double* submit_s);

/* Thread-local message describing the last failure of this thread. */
const char* hnsw_last_error(void);

int hnsw_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
