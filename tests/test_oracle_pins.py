"""Pins of the oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv:1603.09320 it checks.  None of them runs
on a GPU.
"""
import json
import math
import os
from collections import deque

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Hand-worked example (Alg. 1, 2, 4, 5)
# --------------------------------------------------------------------------
# Points p0..p5 = (0,0) (10,0) (0,10) (10,10) (5,5) (20,0); levels 1,0,0,1,0,0;
# M=2, Mmax=2, Mmax0=3, efC=6.  Squared distances:
#   d01=100 d02=100 d03=200 d04=50 d05=400 d12=200 d13=100 d14=50 d15=100
#   d23=100 d24=50 d25=500 d34=50 d35=200 d45=250
# p0: first element -> enter point, level 1, no links.
# p1: layer 1 greedy from p0 finds nothing; layer 0 W={p0}; select {p0}.
#     links p1:[0]  p0:[1]
# p2: layer 0 from p0: expand p0 -> p1 (200) inserted; W={p0:100,p1:200}.
#     heuristic: accept p0; p1: 200 < d(p1,p0)=100 fails -> rejected.
#     links p2:[0]  p0:[1,2]
# p3 (level 1): layer 1 W={p0}; links p3:[0] p0:[3] at layer 1.
#     layer 0 from {p0}: expand p0 -> p1(100), p2(100); W={p1,p2,p0}.
#     heuristic: p1 accepted; p2: 100 < d(p2,p1)=200 -> accepted; |R|=M.
#     links p3:[1,2]  p1:[0,3]  p2:[0,3]; level 1 is not > L=1: ep stays p0.
# p4 (5,5): layer 1 from p0 (50): neighbour p3 (50) has key (50,3) > (50,0)
#     so W stays {p0}.  Layer 0: expand p0 -> p1,p2 (50 each); expand p1 ->
#     p3 (50); W={p0,p1,p2,p3} all at 50.  heuristic in key order: p0
#     accepted; p1: 50 < d(p1,p0)=100 -> accepted; |R|=M.
#     links p4:[0,1]  p0:[1,2,4]  p1:[0,3,4]
# p5 (20,0): layer 1 from p0 (400): p3 (200) replaces it; ep=p3.
#     layer 0 from p3: expand p3 -> p1(100), p2(500); expand p1 -> p0(400),
#     p4(250); p4, p0, p2 expanded without news.  W sorted: p1 p3 p4 p0 p2.
#     heuristic: p1 accepted; p3: 200<d(p3,p1)=100 no; p4: 250<50 no;
#     p0: 400<100 no; p2: 500<200 no.  links p5:[1]  p1:[0,3,4,5]
#     p1 now has 4 > Mmax0=3 links -> shrink with Alg. 4 from base p1 over
#     {0,3,4,5} at distances 100,100,50,100: key order p4,p0,p3,p5; p4
#     accepted; p0: 100<d(p0,p4)=50 no; p3: 100<50 no; p5: 100<250 yes.
#     p1:[4,5]
# Query (12,1): distances p0 145, p1 5, p2 225, p3 85, p4 65, p5 65.
#   K=2, ef=2: layer 1 from p0 -> p3 (85).  Layer 0 from p3: expand p3 ->
#   p1 (5) inserted, p2 (225) rejected; expand p1 -> p4 (65) inserted and
#   p3 evicted, p5 (65,5) rejected against (65,4); expand p4 -> p0 (145)
#   rejected.  W={p1,p4}; 7 distance evaluations (ep, p3, p1, p2, p4, p5,
#   p0); 3 layer-0 expansions (p3, p1, p4); 2 upper expansions (p0, p3).
def _hand():
    with open(os.path.join(GOLD, "hand_example_2d.json")) as f:
        return json.load(f)


def test_hand_example_graph(oracle):
    h = _hand()
    X = np.array(h["points"], dtype=np.float32)
    p = h["params"]
    g = oracle.Graph.new(X, metric=0, M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"], efC=p["efC"])
    for i, l in enumerate(h["levels"]):
        g.insert(i, l)
    assert g.enter_point == h["enter_point"]
    assert g.max_level == h["max_level"]
    for k, v in h["layer1"].items():
        assert g.neighbors(int(k), 1) == v
    for k, v in h["layer0"].items():
        assert g.neighbors(int(k), 0) == v


def test_hand_example_search(oracle):
    h = _hand()
    X = np.array(h["points"], dtype=np.float32)
    p = h["params"]
    g = oracle.Graph.new(X, metric=0, M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"], efC=p["efC"])
    for i, l in enumerate(h["levels"]):
        g.insert(i, l)
    q = np.array(h["query"], dtype=np.float32)
    ids, ds, st = g.knn_search(q, 2, 2, stats=True)
    e = h["search_k2_ef2"]
    assert ids.tolist() == e["ids"] and ds.tolist() == e["dists"]
    assert (st.n_dist, st.n_hops0, st.n_hopsU) == (e["n_dist"], e["n_hops0"], e["n_hopsU"])
    ids, ds = g.knn_search(q, 1, 1)
    assert ids.tolist() == h["search_k1_ef1"]["ids"]
    assert ds.tolist() == h["search_k1_ef1"]["dists"]


def test_hand_example_trace(oracle):
    # The layer-0 beam of the search above (K=2, ef=2, from p3 at 85), state
    # after each expansion (the main loop of Alg. 2):
    #   expand p3: p1 (5) joins W, p2 (225) rejected -> W {p1, p3}; 2 evals;
    #              K-th nearest p3 (85) is the first -> stale 0
    #   expand p1: p4 (65) joins, p3 evicted; p5 (65,5) loses to (65,4)
    #              -> W {p1, p4}; 4 evals; K-th improves to p4 -> stale 0
    #   expand p4: p0 (145) rejected -> W unchanged; 5 evals; stale 1
    # With a record every T=2 expansions only the second state is kept.
    h = _hand()
    X = np.array(h["points"], dtype=np.float32)
    p = h["params"]
    g = oracle.Graph.new(X, metric=0, M=p["M"], Mmax=p["Mmax"], Mmax0=p["Mmax0"], efC=p["efC"])
    for i, l in enumerate(h["levels"]):
        g.insert(i, l)
    q = np.array(h["query"], dtype=np.float32)
    for T, key in ((1, "T1"), (2, "T2")):
        raw, topk = g.knn_search_trace(q, 2, 2, T=T)
        e = h["trace_k2_ef2"][key]
        assert raw.tolist() == e["raw"] and topk.tolist() == e["topk"]


# --------------------------------------------------------------------------
# Level distribution (the level draw of Alg. 1; Section 4.1 mL = 1/ln M; eq. (1))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("M", [8, 16])
def test_level_histogram_geometric(oracle, M):
    from paper_1603_09320_gb300 import synth
    mL = 1.0 / math.log(M)
    u = synth.uniform_open01(77, 200_000)
    lv = np.array([oracle.level_from_u(x, mL) for x in u[:200_000]])
    # P(l >= j) = exp(-j/mL) = M^-j: chi-square over levels 0..3 (+ tail)
    probs = [M ** -j - M ** -(j + 1) for j in range(4)] + [M ** -4]
    obs = [int((lv == j).sum()) for j in range(4)] + [int((lv >= 4).sum())]
    exp = [p * lv.size for p in probs]
    chi2 = sum((o - e) ** 2 / e for o, e in zip(obs, exp) if e >= 5)
    assert chi2 < 20.5  # chi2(4 dof) 0.9996 quantile
    # eq. (1): E[-ln(u) mL] + 1 = mL + 1 (the continuous draw before the floor)
    cont = -np.log(u) * mL
    assert abs(cont.mean() + 1 - (mL + 1)) < 4 * mL / math.sqrt(u.size)


def test_level_formula_closed_form(oracle):
    # floor(-ln u * mL): u = 1 -> 0; u = e^-k/mL exactly at the boundary -> k
    assert oracle.level_from_u(1.0, 0.5) == 0
    assert oracle.level_from_u(math.exp(-2.5), 1.0) == 2
    assert oracle.level_from_u(1.0 / 16 ** 3 * 0.999, 1 / math.log(16)) == 3


# --------------------------------------------------------------------------
# Graph invariants (Section 3: nested layers; Alg. 1 caps; Section 4.2.3)
# --------------------------------------------------------------------------
def _build_small(oracle, X, M=8, efC=64, **kw):
    from paper_1603_09320_gb300 import synth
    u = synth.uniform_open01(12345, X.shape[0])
    return oracle.Graph.build(X, u, M=M, efC=efC, **kw)


def test_invariants_tiny(oracle):
    from paper_1603_09320_gb300 import synth
    X = synth.base("tiny", 3000)
    M = 8
    g = _build_small(oracle, X, M=M)
    L = g.max_level
    assert g.level(g.enter_point) == L
    lv = g.levels()
    assert lv.max() == L
    links = 0
    for i in range(g.N):
        for lc in range(0, lv[i] + 1):
            nb = g.neighbors(i, lc)
            cap = 2 * M if lc == 0 else M
            assert len(nb) <= cap
            assert i not in nb
            assert len(set(nb)) == len(nb)
            for e in nb:
                # a link at layer lc points to an element present at layer lc
                # (nested subsets: present at lc means present at all lower layers)
                assert lv[e] >= lc
            links += len(nb)
        # element at level l has a (possibly empty) list on every layer <= l
        with pytest.raises(ValueError):
            g.neighbors(i, lv[i] + 1)
    # Section 4.2.3: link memory about (Mmax0 + mL*Mmax) * 4 bytes per element
    # at full lists; lists are at most that full.
    mL = 1 / math.log(M)
    assert links * 4 <= (2 * M + 1.5 * mL * M) * 4 * g.N
    assert links * 4 >= 0.3 * (2 * M) * 4 * g.N


def test_blob_roundtrip_and_rejects(oracle):
    from paper_1603_09320_gb300 import synth
    X = synth.base("tiny", 500)
    g = _build_small(oracle, X)
    b = g.to_blob()
    g2 = oracle.Graph.from_blob(b)
    assert g2.to_blob() == b
    bad = bytearray(b)
    bad[200] ^= 1  # payload byte: checksum must catch it
    with pytest.raises(ValueError):
        oracle.Graph.from_blob(bytes(bad))
    with pytest.raises(ValueError):
        oracle.Graph.from_blob(b[:-4])


# --------------------------------------------------------------------------
# Alg. 2 with ef=1 == steepest descent (the descent of Alg. 5)
# --------------------------------------------------------------------------
def test_greedy_lemma(oracle):
    from paper_1603_09320_gb300 import synth
    X = synth.base("tiny", 3000)
    g = _build_small(oracle, X)
    Q = synth.queries("tiny", 200)
    lv = g.levels()
    rng = np.random.default_rng(5)
    for qi in range(Q.shape[0]):
        lc = int(rng.integers(0, g.max_level + 1))
        cand = np.nonzero(lv >= lc)[0]
        ep = int(cand[rng.integers(0, cand.size)])
        ids, _ = g.search_layer(Q[qi], [ep], 1, lc)
        assert int(ids[0]) == g.greedy_layer(Q[qi], ep, lc)


# --------------------------------------------------------------------------
# Alg. 5 with ef >= N equals exact k-NN over the reachable set (Section 1)
# --------------------------------------------------------------------------
def _reachable0(g, start):
    seen = {start}
    dq = deque([start])
    while dq:
        c = dq.popleft()
        for e in g.neighbors(c, 0):
            if e not in seen:
                seen.add(e)
                dq.append(e)
    return seen


@pytest.mark.parametrize("name,n,metric", [("tiny", 800, 0), ("glove", 600, 1)])
def test_exhaustive_search_is_exact(oracle, name, n, metric):
    from paper_1603_09320_gb300 import synth
    X = synth.base(name, n)
    g = _build_small(oracle, X, metric=metric)
    Q = synth.queries(name, 30)
    K = 10
    bi, bd = oracle.brute_force(X, Q, K, metric=metric)
    for i in range(Q.shape[0]):
        ids, ds = g.knn_search(Q[i], K, ef=n)
        # the layer-0 enter point is what the greedy descent reaches
        ep = g.enter_point
        for lc in range(g.max_level, 0, -1):
            ep = g.greedy_layer(Q[i], ep, lc)
        R = _reachable0(g, ep)
        if len(R) == n:
            assert ids.tolist() == bi[i].tolist()
            np.testing.assert_array_equal(ds, bd[i])
        else:  # exact over the reachable component
            sub = np.array(sorted(R))
            si, sd = oracle.brute_force(X[sub], Q[i:i + 1], K, metric=metric)
            assert ids.tolist() == sub[si[0]].tolist()


def test_recall_grows_with_ef(oracle):
    from paper_1603_09320_gb300 import synth
    X = synth.base("tiny", 2000)
    g = _build_small(oracle, X)
    Q = synth.queries("tiny", 100)
    bi, _ = oracle.brute_force(X, Q, 10)
    rec = []
    for ef in (10, 40, 160, 2000):
        ids, _ = g.knn_search_batch(Q, 10, ef)
        rec.append(np.mean([len(set(ids[i]) & set(bi[i])) / 10 for i in range(len(Q))]))
    assert all(b >= a - 0.02 for a, b in zip(rec, rec[1:]))
    assert rec[-1] == 1.0


def test_brute_force_against_numpy_sort(oracle):
    # the exact k-NN itself: compare with a full numpy sort by (distance, id)
    rng = np.random.default_rng(3)
    X = rng.integers(0, 4, size=(300, 3)).astype(np.float32)  # many ties
    q = rng.integers(0, 4, size=(1, 3)).astype(np.float32)
    ids, ds = oracle.brute_force(X, q, 20)
    d = ((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1)
    order = np.lexsort((np.arange(300), d))[:20]
    assert ids[0].tolist() == order.tolist()
    assert ds[0].tolist() == d[order].tolist()


def test_brute_force_cosine_against_numpy(oracle):
    # cosine distance 1 - <q, x> on unit vectors (Section 5.2): nearest = most similar
    rng = np.random.default_rng(4)
    X = rng.standard_normal((400, 16))
    X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    q = rng.standard_normal(16)
    q = (q / np.linalg.norm(q)).astype(np.float32)[None, :]
    ids, ds = oracle.brute_force(X, q, 15, metric=1)
    sim = X.astype(np.float64) @ q[0].astype(np.float64)
    order = np.argsort(-sim, kind="stable")[:15]
    assert ids[0].tolist() == order.tolist()
    np.testing.assert_allclose(ds[0], 1.0 - sim[order], rtol=0, atol=1e-12)
    assert ds[0][0] >= 0.0 and np.all(np.diff(ds[0]) >= 0)


# --------------------------------------------------------------------------
# Alg. 3 (M nearest) and Alg. 4 (heuristic) properties
# --------------------------------------------------------------------------
def test_select_simple_is_partial_sort(oracle):
    rng = np.random.default_rng(4)
    X = rng.integers(0, 5, size=(200, 2)).astype(np.float32)
    g = oracle.Graph.new(X, M=4)
    base = np.array([2, 2], dtype=np.float32)
    cand = rng.choice(200, size=60, replace=False).astype(np.uint32)
    got = g.select_simple(base, cand, 7)
    d = ((X[cand].astype(np.float64) - 2.0) ** 2).sum(1)
    exp = cand[np.lexsort((cand, d))][:7]
    assert got == exp.tolist()


def test_heuristic_1d_gives_line_neighbours(oracle):
    # Section 3: on 1-D data the heuristic yields the exact Delaunay graph, so
    # every element keeps links to its sorted predecessor and successor.
    rng = np.random.default_rng(11)
    x = rng.permutation(np.arange(0, 400, 2)).astype(np.float32)[:150]
    X = x[:, None]
    g = oracle.Graph.build(X, np.full(150, 1.0), M=4, efC=150)  # all level 0
    order = np.argsort(x)
    for k, i in enumerate(order):
        nb = set(g.neighbors(int(i), 0))
        if k > 0:
            assert int(order[k - 1]) in nb
        if k + 1 < len(order):
            assert int(order[k + 1]) in nb
    # and ef=1 greedy search on the line finds the true nearest element
    for qv in rng.uniform(-10, 410, size=50).astype(np.float32):
        ids, ds = g.knn_search(np.array([qv], np.float32), 1, 1)
        bi, bd = oracle.brute_force(X, np.array([[qv]], np.float32), 1)
        assert ds[0] == bd[0][0]


def test_heuristic_acceptance_properties(oracle):
    # Alg. 4's acceptance loop: the first candidate is always accepted; every
    # accepted e is strictly closer to the base than to each earlier accepted
    # r; every rejected candidate examined before the last acceptance has an
    # accepted r (examined before it) with d(e,r) <= d(e,base).
    rng = np.random.default_rng(8)
    X = rng.normal(size=(400, 6)).astype(np.float32)
    g = oracle.Graph.new(X, M=8)
    for t in range(20):
        base = rng.normal(size=6).astype(np.float32)
        cand = rng.choice(400, size=80, replace=False).astype(np.uint32)
        sel = g.select_heuristic(base, cand, 10)
        db = {int(c): g.dist(base, int(c)) for c in cand}
        order = sorted(db, key=lambda c: (db[c], c))
        assert sel[0] == order[0]
        dd = lambda a, b: float(((X[a].astype(np.float64) - X[b]) ** 2).sum())
        for j, e in enumerate(sel):
            for r in sel[:j]:
                assert db[e] < dd(e, r)
        last = order.index(sel[-1])
        for e in order[:last]:
            if e in sel:
                continue
            earlier = [r for r in sel if order.index(r) < order.index(e)]
            assert any(dd(e, r) <= db[e] for r in earlier)


def test_extend_candidates_adds_the_candidates_neighbourhoods(oracle):
    # Alg. 4's extendCandidates step selects over C plus every layer-lc
    # neighbour of an element of C (the base element itself excluded); the
    # union is formed here from the graph's lists and selected without it
    p = {"M": 6, "Mmax": 6, "Mmax0": 12, "efC": 40}
    rng = np.random.default_rng(21)
    X = rng.normal(size=(500, 5)).astype(np.float32)
    g = oracle.Graph.build(X, 1.0 - rng.uniform(0.0, 1.0, 500), **p)  # u in (0, 1]
    for t in range(15):
        base_id = int(rng.integers(500))
        cand = [int(c) for c in rng.choice(500, size=12, replace=False) if c != base_id]
        union = list(cand)
        for c in cand:
            for a in g.neighbors(c, 0):
                if a != base_id and a not in union:
                    union.append(a)
        assert len(union) > len(cand)
        for keep in (False, True):
            ext = g.select_heuristic(X[base_id], cand, 6, lc=0, base_id=base_id, extend=True, keep_pruned=keep)
            ref = g.select_heuristic(X[base_id], union, 6, lc=0, base_id=base_id, keep_pruned=keep)
            assert ext == ref


def test_heuristic_bridges_clusters(oracle):
    # Fig. 2: an element on the boundary of cluster 1 gets a link into the
    # isolated cluster 2 from the heuristic, while "M nearest" picks only
    # cluster 1.
    rng = np.random.default_rng(2)
    c1 = rng.normal(0, 1.0, size=(60, 2))
    c2 = rng.normal(0, 1.0, size=(60, 2)) + np.array([9.0, 0.0])
    X = np.vstack([c1, c2]).astype(np.float32)
    base = np.array([3.0, 0.0], dtype=np.float32)
    g = oracle.Graph.new(X, M=6)
    cand = np.arange(120, dtype=np.uint32)
    simple = g.select_simple(base, cand, 6)
    heur = g.select_heuristic(base, cand, 6)
    assert all(s < 60 for s in simple)
    assert any(h >= 60 for h in heur)


def test_heuristic_beats_simple_selection_on_clustered_data(oracle):
    # Section 4 / Fig. 7: on strongly clustered low-dimensional data the
    # M-nearest selection (Alg. 3) links only inside clusters and the search
    # cannot leave the enter point's region; the heuristic (Alg. 4) keeps
    # links between clusters
    rng = np.random.default_rng(31)
    centres = rng.uniform(0, 1, (50, 4))
    X = (centres[rng.integers(0, 50, 5000)] + rng.normal(0, 0.003, (5000, 4))).astype(np.float32)
    Q = (centres[rng.integers(0, 50, 300)] + rng.normal(0, 0.003, (300, 4))).astype(np.float32)
    u = 1.0 - rng.uniform(0, 1, 5000)
    gt, _ = oracle.brute_force(X, Q, 10)

    def recall(g, ef):
        ids, _ = g.knn_search_batch(Q, 10, ef)
        return np.mean([len(set(ids[i].tolist()) & set(gt[i].tolist())) / 10 for i in range(len(Q))])

    p = dict(M=6, Mmax=6, Mmax0=12, efC=40)
    simple = oracle.Graph.build(X, u, heuristic=False, **p)
    heur = oracle.Graph.build(X, u, heuristic=True, **p)
    for ef in (10, 40):
        rs, rh = recall(simple, ef), recall(heur, ef)
        assert rh >= 0.98 and rh >= rs + 0.15, (ef, rs, rh)


def test_heuristic_tie_is_rejected(oracle):
    # Alg. 4's acceptance test read strictly: e with d(e,base) == d(e,r) is not "closer
    # to the base" than r, so it is discarded.
    X = np.array([[1.0, 0.0], [0.5, 2.0]], dtype=np.float32)  # r, e on the bisector
    g = oracle.Graph.new(X, M=2)
    base = np.array([0.0, 0.0], dtype=np.float32)
    assert g.dist(base, 1) == float(((X[1].astype(np.float64) - X[0]) ** 2).sum())
    assert g.select_heuristic(base, [0, 1], 2) == [0]
    # keepPrunedConnections refills from the discarded queue (Alg. 4's last step)
    assert g.select_heuristic(base, [0, 1], 2, keep_pruned=True) == [0, 1]
