/*
 * hnsw_oracle.c -- ORACLE (test infrastructure only): plain single-threaded C
 * restatement of Hierarchical NSW, arXiv:1603.09320, Section 4, Algorithms 1-5.
 * See hnsw_oracle.h for the readings of the paper that this file takes and
 * for the serialised graph format.
 *
 * Nothing here is tuned: binary heaps, a fresh byte array as visited set per
 * SEARCH-LAYER call, fp64 distances, linear scans.  The code follows the
 * paper's steps in the paper's order so it can be checked against it by eye.
 */
#include "hnsw_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* graph                                                                     */
/* ------------------------------------------------------------------------ */

struct orc_graph {
    uint64_t N;
    uint32_t d;
    int metric;
    uint32_t M, Mmax, Mmax0, efC;
    double mL;
    int heuristic, extend, keep;
    float* data;       /* N*d */
    int* level;        /* -1 while not inserted */
    /* neighbourhood(i) at layer lc: list[0] = count, list[1..] = ids.
     * Capacity cap+1 so that one extra link fits before the shrink of Alg. 1. */
    uint32_t* adj0;    /* N * (Mmax0 + 2) */
    uint32_t** adjU;   /* adjU[i]: level[i] lists of (Mmax + 2) words, layer lc at (lc-1) */
    uint32_t ep;
    int maxlevel;
    uint64_t n_inserted;
};

typedef struct {
    double d;
    uint32_t id;
} orc_item;

/* key order (distance, id), lexicographic */
static int key_less(orc_item a, orc_item b) {
    return a.d < b.d || (a.d == b.d && a.id < b.id);
}

static uint32_t* nbh(const orc_graph* g, uint32_t i, int lc) {
    if (lc == 0) return g->adj0 + (uint64_t)i * (g->Mmax0 + 2);
    return g->adjU[i] + (uint64_t)(lc - 1) * (g->Mmax + 2);
}

static uint32_t cap_of(const orc_graph* g, int lc) { return lc == 0 ? g->Mmax0 : g->Mmax; }

/* Distance functions (Section 5.2 / Table 1): squared L2, or cosine distance
 * 1 - <q,x> on unit-normalised vectors.  Accumulated in fp64. */
static double dist_vec(const orc_graph* g, const float* a, const float* b) {
    double s = 0.0;
    if (g->metric == 0) {
        for (uint32_t i = 0; i < g->d; ++i) {
            double t = (double)a[i] - (double)b[i];
            s += t * t;
        }
        return s;
    }
    for (uint32_t i = 0; i < g->d; ++i) s += (double)a[i] * (double)b[i];
    return 1.0 - s;
}

static const float* row(const orc_graph* g, uint32_t i) { return g->data + (uint64_t)i * g->d; }

double orc_dist_to(const orc_graph* g, const float* q, uint32_t i) { return dist_vec(g, q, row(g, i)); }

int orc_set_data(orc_graph* g, const float* data) {
    if (!g || !data) return -1;
    if (g->N && g->d) memcpy(g->data, data, sizeof(float) * g->N * g->d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* binary heap over orc_item; is_max selects a max-heap (furthest on top)    */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_item* a;
    int n, cap, is_max;
} orc_heap;

static int heap_init(orc_heap* h, int cap, int is_max) {
    h->a = (orc_item*)malloc(sizeof(orc_item) * (size_t)(cap > 4 ? cap : 4));
    h->n = 0;
    h->cap = cap > 4 ? cap : 4;
    h->is_max = is_max;
    return h->a != NULL;
}
static void heap_free(orc_heap* h) { free(h->a); h->a = NULL; }

/* does x belong above y */
static int heap_above(const orc_heap* h, orc_item x, orc_item y) {
    return h->is_max ? key_less(y, x) : key_less(x, y);
}

static int heap_push(orc_heap* h, orc_item x) {
    if (h->n == h->cap) {
        int nc = h->cap * 2;
        orc_item* na = (orc_item*)realloc(h->a, sizeof(orc_item) * (size_t)nc);
        if (!na) return 0;
        h->a = na;
        h->cap = nc;
    }
    int i = h->n++;
    h->a[i] = x;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!heap_above(h, h->a[i], h->a[p])) break;
        orc_item t = h->a[i]; h->a[i] = h->a[p]; h->a[p] = t;
        i = p;
    }
    return 1;
}

static orc_item heap_pop(orc_heap* h) {
    orc_item top = h->a[0];
    h->a[0] = h->a[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->n && heap_above(h, h->a[l], h->a[b])) b = l;
        if (r < h->n && heap_above(h, h->a[r], h->a[b])) b = r;
        if (b == i) break;
        orc_item t = h->a[i]; h->a[i] = h->a[b]; h->a[b] = t;
        i = b;
    }
    return top;
}

static int cmp_item(const void* x, const void* y) {
    orc_item a = *(const orc_item*)x, b = *(const orc_item*)y;
    if (key_less(a, b)) return -1;
    if (key_less(b, a)) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* construction of the empty graph                                           */
/* ------------------------------------------------------------------------ */

orc_graph* orc_new(const float* data, uint64_t N, uint32_t d, int metric,
                   uint32_t M, uint32_t Mmax, uint32_t Mmax0, uint32_t efC, double mL,
                   int heuristic, int extend_candidates, int keep_pruned) {
    if (d == 0 || (metric != 0 && metric != 1) || M == 0 || M > Mmax || M > Mmax0 ||
        N >= 0xFFFFFFFFull || efC == 0)
        return NULL;
    orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
    if (!g) return NULL;
    g->N = N; g->d = d; g->metric = metric;
    g->M = M; g->Mmax = Mmax; g->Mmax0 = Mmax0; g->efC = efC; g->mL = mL;
    g->heuristic = heuristic; g->extend = extend_candidates; g->keep = keep_pruned;
    g->data = (float*)malloc(sizeof(float) * (N * d > 0 ? N * d : 1));
    g->level = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    g->adj0 = (uint32_t*)calloc((N > 0 ? N : 1) * (Mmax0 + 2), sizeof(uint32_t));
    g->adjU = (uint32_t**)calloc(N > 0 ? N : 1, sizeof(uint32_t*));
    if (!g->data || !g->level || !g->adj0 || !g->adjU) { orc_free(g); return NULL; }
    if (N && d) memcpy(g->data, data, sizeof(float) * N * d);
    for (uint64_t i = 0; i < N; ++i) g->level[i] = -1;
    g->ep = ORC_NONE;
    g->maxlevel = -1;
    g->n_inserted = 0;
    return g;
}

void orc_free(orc_graph* g) {
    if (!g) return;
    if (g->adjU)
        for (uint64_t i = 0; i < g->N; ++i) free(g->adjU[i]);
    free(g->adjU);
    free(g->adj0);
    free(g->level);
    free(g->data);
    free(g);
}

/* Alg. 1, the level draw: l <- floor(-ln(unif(0..1)) * mL), u supplied in (0,1]. */
int orc_level_from_u(double u, double mL) { return (int)floor(-log(u) * mL); }

/* ------------------------------------------------------------------------ */
/* Alg. 2  SEARCH-LAYER(q, ep, ef, lc)                                       */
/* ------------------------------------------------------------------------ */

/* Optional recording of the search state on layer 0 (for the learned-stop
 * features): after every T-th expansion, once |W| >= K, the nearest,
 * furthest and K-th nearest distances of W, the layer-0 distance evaluations
 * so far, the enter point's distance d1, the expansions since the K-th
 * nearest last improved, and the ids of the K nearest. */
typedef struct {
    int K, T, max_checks, n_checks;
    double* raw;      /* [max_checks][6]: best, worst, kth, n_eval0, d1, stale */
    uint32_t* topk;   /* [max_checks][K] */
} orc_trace;

/* ep given as items (id with its distance to q already known).  Result W is
 * written sorted ascending by key; returns |W|, or -1 on allocation failure. */
static int search_layer_items_tr(const orc_graph* g, const float* q, const orc_item* ep, int n_ep,
                                 int ef, int lc, orc_item* out, orc_stats* st, orc_trace* tr) {
    unsigned char* v = (unsigned char*)calloc(g->N > 0 ? g->N : 1, 1);
    orc_heap C, W;
    if (!v || !heap_init(&C, 64, 0) || !heap_init(&W, ef + 2, 1)) { free(v); return -1; }
    /* start: v <- ep, C <- ep, W <- ep */
    for (int i = 0; i < n_ep; ++i) {
        if (v[ep[i].id]) continue;
        v[ep[i].id] = 1;
        heap_push(&C, ep[i]);
        heap_push(&W, ep[i]);
    }
    uint64_t n_eval0 = 0, n_exp = 0, stale = 0;
    orc_item last_kth = { INFINITY, ORC_NONE };
    orc_item* sorted = tr ? (orc_item*)malloc(sizeof(orc_item) * (size_t)(ef + n_ep + 2)) : NULL;
    /* while C is not empty */
    while (C.n > 0) {
        orc_item c = heap_pop(&C);              /* extract the nearest of C */
        orc_item f = W.a[0];                    /* the furthest of W */
        if (key_less(f, c)) break;              /* stop when key(c) > key(f) */
        if (st) { if (lc == 0) st->n_hops0++; else st->n_hopsU++; }
        const uint32_t* nb = nbh(g, c.id, lc);
        for (uint32_t j = 0; j < nb[0]; ++j) { /* each neighbour e of c at layer lc */
            uint32_t e = nb[1 + j];
            if (v[e]) continue;                 /* skip visited */
            v[e] = 1;                           /* mark visited */
            f = W.a[0];                         /* the furthest of W again */
            orc_item ei = { dist_vec(g, q, row(g, e)), e };
            if (st) st->n_dist++;
            n_eval0++;
            if (key_less(ei, f) || W.n < ef) {  /* admit e: closer than f, or W not full */
                heap_push(&C, ei);              /* into C */
                heap_push(&W, ei);              /* into W */
                if (W.n > ef) heap_pop(&W);     /* drop the furthest when W exceeds ef */
            }
        }
        if (tr && sorted) {   /* state after this expansion */
            n_exp++;
            int nw = W.n;
            for (int i = 0; i < nw; ++i) sorted[i] = W.a[i];
            qsort(sorted, (size_t)nw, sizeof(orc_item), cmp_item);
            if (nw >= tr->K && key_less(sorted[tr->K - 1], last_kth)) {
                last_kth = sorted[tr->K - 1];
                stale = 0;
            } else {
                stale++;
            }
            if (nw >= tr->K && n_exp % (uint64_t)tr->T == 0) {
                if (tr->n_checks < tr->max_checks) {
                    double* r = tr->raw + 6 * (size_t)tr->n_checks;
                    r[0] = sorted[0].d;
                    r[1] = sorted[nw - 1].d;
                    r[2] = sorted[tr->K - 1].d;
                    r[3] = (double)n_eval0;
                    r[4] = ep[0].d;
                    r[5] = (double)stale;
                    for (int i = 0; i < tr->K; ++i) tr->topk[(size_t)tr->n_checks * tr->K + i] = sorted[i].id;
                }
                tr->n_checks++;
            }
        }
    }
    free(sorted);
    int n = W.n;
    for (int i = 0; i < n; ++i) out[i] = W.a[i];
    qsort(out, (size_t)n, sizeof(orc_item), cmp_item);
    heap_free(&C);
    heap_free(&W);
    free(v);
    return n;
}

static int search_layer_items(const orc_graph* g, const float* q, const orc_item* ep, int n_ep,
                              int ef, int lc, orc_item* out, orc_stats* st) {
    return search_layer_items_tr(g, q, ep, n_ep, ef, lc, out, st, NULL);
}

int orc_search_layer(const orc_graph* g, const float* q, const uint32_t* ep, int n_ep,
                     int ef, int lc, uint32_t* out_ids, double* out_dists, orc_stats* st) {
    if (ef < 1 || n_ep < 1) return 0;
    orc_item* e = (orc_item*)malloc(sizeof(orc_item) * (size_t)n_ep);
    int cap = (ef > n_ep ? ef : n_ep) + 2;
    orc_item* w = (orc_item*)malloc(sizeof(orc_item) * (size_t)cap);
    if (!e || !w) { free(e); free(w); return -1; }
    for (int i = 0; i < n_ep; ++i) {
        e[i].id = ep[i];
        e[i].d = dist_vec(g, q, row(g, ep[i]));
        if (st) st->n_dist++;
    }
    int n = search_layer_items(g, q, e, n_ep, ef, lc, w, st);
    for (int i = 0; i < n; ++i) { out_ids[i] = w[i].id; out_dists[i] = w[i].d; }
    free(e);
    free(w);
    return n;
}

/* Steepest descent: cur <- ep; repeat b <- argmin_key({cur} u N_lc(cur));
 * stop when b == cur.  Equal to Alg. 2 with ef = 1 under key order. */
uint32_t orc_greedy_layer(const orc_graph* g, const float* q, uint32_t ep, int lc, orc_stats* st) {
    orc_item cur = { dist_vec(g, q, row(g, ep)), ep };
    if (st) st->n_dist++;
    for (;;) {
        orc_item b = cur;
        const uint32_t* nb = nbh(g, cur.id, lc);
        for (uint32_t j = 0; j < nb[0]; ++j) {
            orc_item e = { dist_vec(g, q, row(g, nb[1 + j])), nb[1 + j] };
            if (st) st->n_dist++;
            if (key_less(e, b)) b = e;
        }
        if (b.id == cur.id) return cur.id;
        if (st) st->n_hopsU++;
        cur = b;
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 and Alg. 4                                                         */
/* ------------------------------------------------------------------------ */

/* Alg. 3: the M nearest of C to the base (C given with distances). */
static int select_simple_items(orc_item* C, int n, int M, uint32_t* out) {
    qsort(C, (size_t)n, sizeof(orc_item), cmp_item);
    int m = n < M ? n : M;
    for (int i = 0; i < m; ++i) out[i] = C[i].id;
    return m;
}

/* Alg. 4: SELECT-NEIGHBORS-HEURISTIC(base, C, M, lc, extendCandidates,
 * keepPrunedConnections).  C given with distances to the base. */
static int select_heuristic_items(const orc_graph* g, const float* base, uint32_t base_id,
                                  const orc_item* C, int n, int M, int lc,
                                  int extend, int keep, uint32_t* out) {
    int nR = 0;
    orc_item* R = (orc_item*)malloc(sizeof(orc_item) * (size_t)(M > 0 ? M : 1));
    orc_heap Wq, Wd;
    unsigned char* inW = (unsigned char*)calloc(g->N > 0 ? g->N : 1, 1);
    if (!R || !inW || !heap_init(&Wq, n + 4, 0) || !heap_init(&Wd, n + 4, 0)) {
        free(R); free(inW); return -1;
    }
    /* the working queue W <- C */
    for (int i = 0; i < n; ++i) { heap_push(&Wq, C[i]); inW[C[i].id] = 1; }
    /* extendCandidates: add the candidates' neighbourhoods at layer lc */
    if (extend) {
        for (int i = 0; i < n; ++i) {
            const uint32_t* nb = nbh(g, C[i].id, lc);
            for (uint32_t j = 0; j < nb[0]; ++j) {
                uint32_t a = nb[1 + j];
                if (inW[a] || a == base_id) continue;
                inW[a] = 1;
                orc_item it = { dist_vec(g, base, row(g, a)), a };
                heap_push(&Wq, it);
            }
        }
    }
    /* accept e when it is closer to the base than to every element of R */
    while (Wq.n > 0 && nR < M) {
        orc_item e = heap_pop(&Wq);
        int good = 1;
        for (int r = 0; r < nR; ++r) {
            /* e is accepted only if it is closer to the base than to every r */
            if (!(e.d < dist_vec(g, row(g, e.id), row(g, R[r].id)))) { good = 0; break; }
        }
        if (good) R[nR++] = e;
        else heap_push(&Wd, e);
    }
    /* keepPrunedConnections: refill R from the discarded, nearest first */
    if (keep)
        while (Wd.n > 0 && nR < M) R[nR++] = heap_pop(&Wd);
    for (int i = 0; i < nR; ++i) out[i] = R[i].id;
    heap_free(&Wq);
    heap_free(&Wd);
    free(inW);
    free(R);
    return nR;
}

static int select_items(const orc_graph* g, const float* base, uint32_t base_id,
                        orc_item* C, int n, int M, int lc, uint32_t* out) {
    if (g->heuristic) return select_heuristic_items(g, base, base_id, C, n, M, lc, g->extend, g->keep, out);
    return select_simple_items(C, n, M, out);
}

int orc_select_simple(const orc_graph* g, const float* base, const uint32_t* cand,
                      int n_cand, int M, uint32_t* out) {
    orc_item* C = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n_cand > 0 ? n_cand : 1));
    if (!C) return -1;
    for (int i = 0; i < n_cand; ++i) { C[i].id = cand[i]; C[i].d = dist_vec(g, base, row(g, cand[i])); }
    int r = select_simple_items(C, n_cand, M, out);
    free(C);
    return r;
}

int orc_select_heuristic(const orc_graph* g, const float* base, uint32_t base_id,
                         const uint32_t* cand, int n_cand, int M, int lc,
                         int extend_candidates, int keep_pruned, uint32_t* out) {
    orc_item* C = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n_cand > 0 ? n_cand : 1));
    if (!C) return -1;
    for (int i = 0; i < n_cand; ++i) { C[i].id = cand[i]; C[i].d = dist_vec(g, base, row(g, cand[i])); }
    int r = select_heuristic_items(g, base, base_id, C, n_cand, M, lc, extend_candidates, keep_pruned, out);
    free(C);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1  INSERT(hnsw, q, M, Mmax, efConstruction, mL)                      */
/* ------------------------------------------------------------------------ */

static int has_link(const uint32_t* list, uint32_t x) {
    for (uint32_t j = 0; j < list[0]; ++j)
        if (list[1 + j] == x) return 1;
    return 0;
}

/* Alg. 1 (everything after the level draw) for element qid of level l (level and lists already
 * set up), on layers lc >= lc_min only: lc_min = 0 is the whole insertion,
 * lc_min = 1 the upper layers of an element already linked on layer 0. */
static int insert_layers(orc_graph* g, uint32_t qid, int l, int lc_min) {
    const float* q = row(g, qid);
    int cap_w = (int)g->efC + 2;
    orc_item* W = (orc_item*)malloc(sizeof(orc_item) * (size_t)cap_w);
    orc_item* ep = (orc_item*)malloc(sizeof(orc_item) * (size_t)cap_w);
    orc_item* cand = (orc_item*)malloc(sizeof(orc_item) * (size_t)(g->Mmax0 + 2 + cap_w));
    uint32_t* sel = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(g->Mmax0 + 2 + cap_w));
    if (!W || !ep || !cand || !sel) { free(W); free(ep); free(cand); free(sel); return -1; }

    /* enter point and top level */
    int n_ep = 1;
    ep[0].id = g->ep;
    ep[0].d = dist_vec(g, q, row(g, g->ep));
    int L = g->maxlevel;
    /* greedy ef = 1 descent through layers L .. l+1 */
    for (int lc = L; lc > l; --lc) {
        int n = search_layer_items(g, q, ep, n_ep, 1, lc, W, NULL);
        ep[0] = W[0];
        n_ep = 1;
        (void)n;
    }
    /* layers min(L, l) .. 0 */
    for (int lc = (L < l ? L : l); lc >= lc_min; --lc) {
        int nW = search_layer_items(g, q, ep, n_ep, (int)g->efC, lc, W, NULL);  /* SEARCH-LAYER with efConstruction */
        for (int i = 0; i < nW; ++i) cand[i] = W[i];
        int nsel = select_items(g, q, qid, cand, nW, (int)g->M, lc, sel);         /* SELECT-NEIGHBORS(q, W, M) */
        /* bidirectional connections */
        uint32_t* ql = nbh(g, qid, lc);
        for (int i = 0; i < nsel; ++i) {
            if (sel[i] == qid || has_link(ql, sel[i])) continue;
            ql[1 + ql[0]++] = sel[i];
            uint32_t* el = nbh(g, sel[i], lc);
            if (!has_link(el, qid)) el[1 + el[0]++] = qid;
        }
        /* shrink overfull neighbourhoods */
        uint32_t cap = cap_of(g, lc);
        for (int i = 0; i < nsel; ++i) {
            uint32_t e = sel[i];
            uint32_t* el = nbh(g, e, lc);
            if (el[0] > cap) {
                int ne = (int)el[0];
                for (int j = 0; j < ne; ++j) {
                    cand[j].id = el[1 + j];
                    cand[j].d = dist_vec(g, row(g, e), row(g, el[1 + j]));
                }
                uint32_t* tmp = sel + nsel;  /* spare room after the selection */
                int nn = select_items(g, row(g, e), e, cand, ne, (int)cap, lc, tmp);
                el[0] = (uint32_t)nn;
                for (int j = 0; j < nn; ++j) el[1 + j] = tmp[j];
            }
        }
        /* ep <- W */
        for (int i = 0; i < nW; ++i) ep[i] = W[i];
        n_ep = nW;
    }
    /* a new top level moves the enter point */
    if (l > L) {
        g->ep = qid;
        g->maxlevel = l;
    }
    free(W); free(ep); free(cand); free(sel);
    return 0;
}

static int alloc_upper(orc_graph* g, uint32_t qid, int l) {
    g->level[qid] = l;
    if (l > 0) {
        g->adjU[qid] = (uint32_t*)calloc((size_t)l * (g->Mmax + 2), sizeof(uint32_t));
        if (!g->adjU[qid]) return -1;
    }
    return 0;
}

int orc_insert(orc_graph* g, uint32_t qid, int l) {
    if (qid >= g->N || g->level[qid] >= 0 || l < 0 || l > 255) return -1;
    if (alloc_upper(g, qid, l)) return -1;
    /* the first element: it becomes the enter point, no links */
    if (g->n_inserted == 0) {
        g->ep = qid;
        g->maxlevel = l;
        g->n_inserted = 1;
        return 0;
    }
    if (insert_layers(g, qid, l, 0)) return -1;
    g->n_inserted++;
    return 0;
}

int orc_build(orc_graph* g, const double* u) {
    for (uint64_t i = 0; i < g->N; ++i) {
        int r = orc_insert(g, (uint32_t)i, orc_level_from_u(u[i], g->mL));
        if (r) return r;
    }
    return 0;
}

/* Alg. 1 with batched layer-0 insertions (see the header). */
typedef struct {
    uint32_t target, src, order;
    double d;
} orc_pair;

static int cmp_pair(const void* x, const void* y) {
    const orc_pair* a = (const orc_pair*)x;
    const orc_pair* b = (const orc_pair*)y;
    if (a->target != b->target) return a->target < b->target ? -1 : 1;
    return a->order < b->order ? -1 : (a->order > b->order ? 1 : 0);
}

/* Layer-0 insertion of ids[0..n_ids) (id order, none inserted yet) in
 * batches: `inserted` elements are in the graph before the first batch.
 * Batch sizes: sizes[0..n_sizes) when given (the last one repeated, each
 * clipped to what remains), else `batch`, else the growing schedule. */
static int layer0_batches(orc_graph* g, const uint32_t* ids, uint64_t n_ids, uint64_t inserted, uint32_t batch,
                          const uint32_t* sizes, uint64_t n_sizes) {
    const int efc = (int)g->efC, M = (int)g->M;
    const uint64_t bmax = n_ids < 64 ? 64 : (n_ids > 32768 ? 32768 : n_ids);
    uint64_t cap = batch ? batch : bmax;
    if (sizes && n_sizes) {
        cap = 1;
        for (uint64_t j = 0; j < n_sizes; ++j)
            if (sizes[j] > cap) cap = sizes[j];
    }
    uint32_t* rid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(cap * efc + 1));
    double* rd = (double*)malloc(sizeof(double) * (size_t)(cap * efc + 1));
    orc_pair* pairs = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(cap * M + 1));
    orc_item* C = (orc_item*)malloc(sizeof(orc_item) * (size_t)(efc + 1));
    uint32_t* sel = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(g->Mmax0 + M + 1));
    int rc = (rid && rd && pairs && C && sel) ? 0 : -1;
    for (uint64_t pos = 0, nb = 0; rc == 0 && pos < n_ids; ++nb) {
        uint64_t B = n_ids - pos;
        if (sizes && n_sizes) {
            const uint64_t want = sizes[nb < n_sizes ? nb : n_sizes - 1];
            if (want == 0) { rc = -1; break; }
            if (B > want) B = want;
        } else if (batch) {
            if (B > batch) B = batch;
        } else {
            const uint64_t grow = inserted / 16 > 64 ? inserted / 16 : 64;
            if (B > bmax) B = bmax;
            if (B > grow) B = grow;
        }
        /* 1. searches on the graph before the batch */
        for (uint64_t b = 0; b < B; ++b)
            if (orc_knn_search(g, row(g, ids[pos + b]), efc, efc, rid + b * efc, rd + b * efc, NULL)) rc = -1;
        /* 2. forward links */
        uint64_t np = 0;
        for (uint64_t b = 0; rc == 0 && b < B; ++b) {
            const uint32_t q = ids[pos + b];
            int n = 0;
            for (int i = 0; i < efc; ++i)
                if (rid[b * efc + i] != ORC_NONE && rid[b * efc + i] != q) {
                    C[n].id = rid[b * efc + i];
                    C[n].d = rd[b * efc + i];
                    ++n;
                }
            const int ns = select_items(g, row(g, q), q, C, n, M, 0, sel);
            g->level[q] = 0;
            g->n_inserted++;
            uint32_t* ql = nbh(g, q, 0);
            ql[0] = (uint32_t)ns;
            for (int j = 0; j < ns; ++j) {
                ql[1 + j] = sel[j];
                pairs[np].target = sel[j];
                pairs[np].src = q;
                pairs[np].order = (uint32_t)np;
                pairs[np].d = dist_vec(g, row(g, q), row(g, sel[j]));
                ++np;
            }
        }
        /* 3. reverse links, per target, new members in ascending id */
        qsort(pairs, (size_t)np, sizeof(orc_pair), cmp_pair);
        for (uint64_t i0 = 0; rc == 0 && i0 < np;) {
            uint64_t i1 = i0 + 1;
            while (i1 < np && pairs[i1].target == pairs[i0].target) ++i1;
            const uint32_t e = pairs[i0].target;
            uint32_t* el = nbh(g, e, 0);
            const uint32_t n0 = el[0], nin = (uint32_t)(i1 - i0);
            if (n0 + nin <= g->Mmax0) {
                for (uint32_t t = 0; t < nin; ++t) el[1 + n0 + t] = pairs[i0 + t].src;
                el[0] = n0 + nin;
            } else {
                orc_item* cand = (orc_item*)malloc(sizeof(orc_item) * (size_t)(n0 + nin));
                uint32_t* out = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(g->Mmax0 + 1));
                if (!cand || !out) {
                    rc = -1;
                } else {
                    for (uint32_t j = 0; j < n0; ++j) {
                        cand[j].id = el[1 + j];
                        cand[j].d = dist_vec(g, row(g, e), row(g, el[1 + j]));
                    }
                    for (uint32_t t = 0; t < nin; ++t) {
                        cand[n0 + t].id = pairs[i0 + t].src;
                        cand[n0 + t].d = pairs[i0 + t].d;
                    }
                    /* Alg. 1's shrink: SELECT-NEIGHBORS(e, eConn, Mmax0) over
                     * the whole of eConn, old members and new ones */
                    qsort(cand, (size_t)(n0 + nin), sizeof(orc_item), cmp_item);
                    const int nn = select_items(g, row(g, e), e, cand, (int)(n0 + nin), (int)g->Mmax0, 0, out);
                    el[0] = (uint32_t)nn;
                    for (int j = 0; j < nn; ++j) el[1 + j] = out[j];
                }
                free(cand);
                free(out);
            }
            i0 = i1;
        }
        pos += B;
        inserted += B;
    }
    free(rid); free(rd); free(pairs); free(C); free(sel);
    return rc;
}

static int build_batched(orc_graph* g, const double* u, uint64_t n_first, uint32_t batch, const uint32_t* sizes,
                         uint64_t n_sizes) {
    if (g->extend || g->n_inserted != 0) return -1;
    const uint64_t N = g->N;
    if (n_first < 1) n_first = 1;  /* the first element starts the graph (enter point) */
    int* lv = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    uint32_t* rest = (uint32_t*)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
    if (!lv || !rest) { free(lv); free(rest); return -1; }
    uint64_t n_rest = 0, inserted = 0;
    for (uint64_t i = 0; i < N; ++i) lv[i] = orc_level_from_u(u[i], g->mL);
    /* the seed, in id order */
    for (uint64_t i = 0; i < N; ++i) {
        if (i < n_first || lv[i] > 0) {
            if (orc_insert(g, (uint32_t)i, lv[i])) { free(lv); free(rest); return -1; }
            ++inserted;
        } else {
            rest[n_rest++] = (uint32_t)i;
        }
    }
    const int rc = layer0_batches(g, rest, n_rest, inserted, batch, sizes, n_sizes);
    free(lv); free(rest);
    return rc;
}

int orc_build_batched(orc_graph* g, const double* u, uint64_t n_first, uint32_t batch) {
    return build_batched(g, u, n_first, batch, NULL, 0);
}

int orc_build_batched_sizes(orc_graph* g, const double* u, uint64_t n_first, const uint32_t* sizes,
                            uint64_t n_sizes) {
    if (!sizes || n_sizes == 0) return -1;
    return build_batched(g, u, n_first, 0, sizes, n_sizes);
}

int orc_insert_batched(orc_graph* g, const double* u, uint64_t first, uint64_t n, uint32_t batch) {
    if (g->extend || g->n_inserted != first || first + n > g->N || first == 0) return -1;
    for (uint64_t i = first; i < first + n; ++i)
        if (g->level[i] >= 0) return -1;
    uint32_t* U = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t* Z = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    int* lv = (int*)malloc(sizeof(int) * (size_t)(n + 1));
    if (!U || !Z || !lv) { free(U); free(Z); free(lv); return -1; }
    uint64_t nu = 0, nz = 0;
    for (uint64_t i = 0; i < n; ++i) {
        lv[i] = orc_level_from_u(u[i], g->mL);
        if (lv[i] > 255) { free(U); free(Z); free(lv); return -1; }
        if (lv[i] > 0) U[nu++] = (uint32_t)(first + i);
        else Z[nz++] = (uint32_t)(first + i);
    }
    /* 1. layer 0 of the new elements of level >= 1, through the upper layers
     *    as they stand (the new elements are not on them yet) */
    int rc = layer0_batches(g, U, nu, first, batch, NULL, 0);
    /* 2. their upper layers, one at a time in id order (Alg. 1 on lc >= 1) */
    for (uint64_t j = 0; rc == 0 && j < nu; ++j) {
        const uint32_t q = U[j];
        const int l = lv[q - first];
        if (alloc_upper(g, q, l) || insert_layers(g, q, l, 1)) rc = -1;
    }
    /* 3. layer 0 of the new elements of level 0 */
    if (rc == 0) rc = layer0_batches(g, Z, nz, first + nu, batch, NULL, 0);
    free(U); free(Z); free(lv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg. 5  K-NN-SEARCH(hnsw, q, K, ef)                                       */
/* ------------------------------------------------------------------------ */

int orc_knn_search(const orc_graph* g, const float* q, int K, int ef,
                   uint32_t* ids, double* dists, orc_stats* st) {
    if (K < 1 || ef < 1) return -1;
    for (int i = 0; i < K; ++i) { ids[i] = ORC_NONE; dists[i] = INFINITY; }
    if (g->n_inserted == 0) return 0;
    int efp = ef > K ? ef : K;                         /* ef' = max(ef, K) */
    orc_item* W = (orc_item*)malloc(sizeof(orc_item) * (size_t)(efp + 2));
    if (!W) return -1;
    orc_item ep = { dist_vec(g, q, row(g, g->ep)), g->ep };   /* the enter point */
    if (st) st->n_dist++;
    int L = g->maxlevel;                                /* its level, the top one */
    for (int lc = L; lc >= 1; --lc) {                   /* greedy descent, ef = 1 */
        search_layer_items(g, q, &ep, 1, 1, lc, W, st);
        ep = W[0];
    }
    int n = search_layer_items(g, q, &ep, 1, efp, 0, W, st);   /* layer 0 with ef' */
    for (int i = 0; i < n && i < K; ++i) { ids[i] = W[i].id; dists[i] = W[i].d; }  /* the K nearest of W */
    free(W);
    return 0;
}

int orc_knn_search_trace(const orc_graph* g, const float* q, int K, int ef, int T, int max_checks,
                         double* raw, uint32_t* topk, int* n_checks) {
    if (K < 1 || ef < 1 || T < 1 || max_checks < 1) return -1;
    *n_checks = 0;
    if (g->n_inserted == 0) return 0;
    int efp = ef > K ? ef : K;
    orc_item* W = (orc_item*)malloc(sizeof(orc_item) * (size_t)(efp + 2));
    if (!W) return -1;
    orc_item ep = { dist_vec(g, q, row(g, g->ep)), g->ep };
    for (int lc = g->maxlevel; lc >= 1; --lc) {
        search_layer_items(g, q, &ep, 1, 1, lc, W, NULL);
        ep = W[0];
    }
    orc_trace tr = { K, T, max_checks, 0, raw, topk };
    search_layer_items_tr(g, q, &ep, 1, efp, 0, W, NULL, &tr);
    *n_checks = tr.n_checks < max_checks ? tr.n_checks : max_checks;
    free(W);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* inspection                                                                */
/* ------------------------------------------------------------------------ */

uint64_t orc_n(const orc_graph* g) { return g->N; }
int orc_level(const orc_graph* g, uint32_t i) { return i < g->N ? g->level[i] : -1; }
uint32_t orc_enter_point(const orc_graph* g) { return g->ep; }
int orc_max_level(const orc_graph* g) { return g->maxlevel; }

int orc_neighbors(const orc_graph* g, uint32_t i, int lc, uint32_t* out, int cap) {
    if (i >= g->N || lc < 0 || lc > g->level[i]) return -1;
    const uint32_t* nb = nbh(g, i, lc);
    int n = (int)nb[0];
    for (int j = 0; j < n && j < cap; ++j) out[j] = nb[1 + j];
    return n;
}

/* ------------------------------------------------------------------------ */
/* exact k-NN                                                                */
/* ------------------------------------------------------------------------ */

void orc_brute_force(const float* data, uint64_t N, uint32_t d, int metric,
                     const float* q, int K, uint32_t* ids, double* dists) {
    orc_graph tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.d = d;
    tmp.metric = metric;
    orc_item* best = (orc_item*)malloc(sizeof(orc_item) * (size_t)(K + 1));
    int nb = 0;
    for (uint64_t i = 0; i < N; ++i) {
        orc_item e = { dist_vec(&tmp, q, data + i * d), (uint32_t)i };
        /* keep the K smallest keys, sorted, by insertion */
        if (nb == K && !key_less(e, best[K - 1])) continue;
        int p = nb < K ? nb++ : K - 1;
        while (p > 0 && key_less(e, best[p - 1])) { best[p] = best[p - 1]; --p; }
        best[p] = e;
    }
    for (int i = 0; i < K; ++i) {
        ids[i] = i < nb ? best[i].id : ORC_NONE;
        dists[i] = i < nb ? best[i].d : INFINITY;
    }
    free(best);
}

/* ------------------------------------------------------------------------ */
/* serialisation, format "HNSWGB01"                                          */
/* ------------------------------------------------------------------------ */

static uint64_t al16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

typedef struct {
    uint64_t data, level, nbr0, nbrU, total;
} orc_layout;

static orc_layout layout_of(uint64_t N, uint32_t d, uint32_t Mmax0, uint32_t Mmax, uint64_t rows) {
    orc_layout o;
    o.data = 128;
    o.level = al16(o.data + N * d * 4u);
    o.nbr0 = al16(o.level + N);
    o.nbrU = al16(o.nbr0 + N * Mmax0 * 4u);
    o.total = o.nbrU + rows * Mmax * 4u;
    return o;
}

static uint64_t upper_rows(const orc_graph* g) {
    uint64_t r = 0;
    for (uint64_t i = 0; i < g->N; ++i) r += g->level[i] > 0 ? (uint64_t)g->level[i] : 0;
    return r;
}

static uint64_t fnv1a(const unsigned char* p, uint64_t n) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (uint64_t i = 0; i < n; ++i) { h ^= p[i]; h *= 0x100000001b3ull; }
    return h;
}

static void put32(unsigned char* p, uint32_t v) { memcpy(p, &v, 4); }
static void put64(unsigned char* p, uint64_t v) { memcpy(p, &v, 8); }
static uint32_t get32(const unsigned char* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t get64(const unsigned char* p) { uint64_t v; memcpy(&v, p, 8); return v; }

uint64_t orc_blob_size(const orc_graph* g) {
    return layout_of(g->N, g->d, g->Mmax0, g->Mmax, upper_rows(g)).total;
}

int orc_save_blob(const orc_graph* g, void* outv, uint64_t cap) {
    for (uint64_t i = 0; i < g->N; ++i)
        if (g->level[i] < 0) return -2;   /* only complete graphs are saved */
    uint64_t rows = upper_rows(g);
    orc_layout o = layout_of(g->N, g->d, g->Mmax0, g->Mmax, rows);
    if (cap < o.total) return -1;
    unsigned char* out = (unsigned char*)outv;
    memset(out, 0, o.total);
    memcpy(out, "HNSWGB01", 8);
    put32(out + 8, 1);
    put32(out + 12, (uint32_t)g->metric);
    put64(out + 16, g->N);
    put32(out + 24, g->d);
    put32(out + 28, g->M);
    put32(out + 32, g->Mmax);
    put32(out + 36, g->Mmax0);
    put32(out + 40, g->N ? (uint32_t)g->maxlevel : 0);
    put32(out + 44, g->N ? g->ep : ORC_NONE);
    put32(out + 48, (uint32_t)((g->heuristic ? 1 : 0) | (g->extend ? 2 : 0) | (g->keep ? 4 : 0)));
    put32(out + 52, g->efC);
    memcpy(out + 56, &g->mL, 8);
    put64(out + 64, rows);
    memcpy(out + o.data, g->data, g->N * g->d * 4u);
    for (uint64_t i = 0; i < g->N; ++i) out[o.level + i] = (unsigned char)g->level[i];
    for (uint64_t i = 0; i < g->N; ++i) {
        const uint32_t* nb = nbh(g, (uint32_t)i, 0);
        unsigned char* r = out + o.nbr0 + i * g->Mmax0 * 4u;
        for (uint32_t j = 0; j < g->Mmax0; ++j) put32(r + 4u * j, j < nb[0] ? nb[1 + j] : ORC_NONE);
    }
    uint64_t rr = 0;
    for (uint64_t i = 0; i < g->N; ++i) {
        for (int lc = 1; lc <= g->level[i]; ++lc, ++rr) {
            const uint32_t* nb = nbh(g, (uint32_t)i, lc);
            unsigned char* r = out + o.nbrU + rr * g->Mmax * 4u;
            for (uint32_t j = 0; j < g->Mmax; ++j) put32(r + 4u * j, j < nb[0] ? nb[1 + j] : ORC_NONE);
        }
    }
    put64(out + 72, fnv1a(out + 128, o.total - 128));
    return 0;
}

/* err: 1 short/bad header, 2 checksum, 3 bad level/enter point, 4 bad link, 5 alloc */
orc_graph* orc_load_blob(const void* blobv, uint64_t bytes, int* err) {
    const unsigned char* b = (const unsigned char*)blobv;
    int e = 0;
    orc_graph* g = NULL;
    if (bytes < 128 || memcmp(b, "HNSWGB01", 8) != 0 || get32(b + 8) != 1) { e = 1; goto fail; }
    uint64_t N = get64(b + 16), rows = get64(b + 64);
    uint32_t d = get32(b + 24), M = get32(b + 28), Mmax = get32(b + 32), Mmax0 = get32(b + 36);
    uint32_t flags = get32(b + 48), efC = get32(b + 52);
    double mL;
    memcpy(&mL, b + 56, 8);
    orc_layout o = layout_of(N, d, Mmax0, Mmax, rows);
    if (o.total != bytes) { e = 1; goto fail; }
    if (fnv1a(b + 128, bytes - 128) != get64(b + 72)) { e = 2; goto fail; }
    g = orc_new((const float*)(b + o.data), N, d, (int)get32(b + 12), M, Mmax, Mmax0, efC, mL,
                (flags & 1) != 0, (flags & 2) != 0, (flags & 4) != 0);
    if (!g) { e = 1; goto fail; }
    uint64_t rsum = 0;
    for (uint64_t i = 0; i < N; ++i) { g->level[i] = b[o.level + i]; rsum += b[o.level + i]; }
    if (rsum != rows) { e = 3; goto fail; }
    g->n_inserted = N;
    g->ep = get32(b + 44);
    g->maxlevel = (int)get32(b + 40);
    if (N > 0 && (g->ep >= N || g->level[g->ep] != g->maxlevel)) { e = 3; goto fail; }
    for (uint64_t i = 0; i < N; ++i)
        if (g->level[i] > g->maxlevel) { e = 3; goto fail; }
    uint64_t rr = 0;
    for (uint64_t i = 0; i < N; ++i) {
        if (g->level[i] > 0) {
            g->adjU[i] = (uint32_t*)calloc((size_t)g->level[i] * (Mmax + 2), sizeof(uint32_t));
            if (!g->adjU[i]) { e = 5; goto fail; }
        }
        for (int lc = 0; lc <= g->level[i]; ++lc) {
            uint32_t cap = lc == 0 ? Mmax0 : Mmax;
            const unsigned char* r = lc == 0 ? b + o.nbr0 + i * Mmax0 * 4u : b + o.nbrU + (rr++) * Mmax * 4u;
            uint32_t* nb = nbh(g, (uint32_t)i, lc);
            int ended = 0;
            for (uint32_t j = 0; j < cap; ++j) {
                uint32_t x = get32(r + 4u * j);
                if (x == ORC_NONE) { ended = 1; continue; }
                if (ended || x >= N || x == i || has_link(nb, x)) { e = 4; goto fail; }
                nb[1 + nb[0]++] = x;
            }
        }
    }
    /* every link at layer lc must point to an element present at layer lc */
    for (uint64_t i = 0; i < N; ++i)
        for (int lc = 1; lc <= g->level[i]; ++lc) {
            const uint32_t* nb = nbh(g, (uint32_t)i, lc);
            for (uint32_t j = 0; j < nb[0]; ++j)
                if (g->level[nb[1 + j]] < lc) { e = 4; goto fail; }
        }
    if (err) *err = 0;
    return g;
fail:
    orc_free(g);
    if (err) *err = e;
    return NULL;
}
