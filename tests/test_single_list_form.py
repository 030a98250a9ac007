"""CPU check of the reformulation of Alg. 2 that the CUDA kernel implements.

The kernel keeps ONE list W sorted by key (distance, id), capped at ef, with
an "expanded" flag per entry instead of the two priority queues of Alg. 2,
merges all unvisited neighbours of the expanded element at once, and uses a
small LOSSY visited set (entries can be overwritten, so an element may be
evaluated twice).  Claims, under key order:
  * C (not yet extracted) restricted to keys <= the furthest of W is exactly
    the set of unexpanded entries of W, so "extract nearest from C" and the
    stop test become "take the first unexpanded entry of W, stop if
    there is none";
  * inserting a batch of neighbours one by one with Alg. 2's admission and eviction leaves the
    top-ef of (W u batch), independent of order;
  * an element evaluated again after the visited set forgot it is either
    already in W (its key is equal to an entry: dropped) or worse than the
    furthest of a full W (rejected), so results are unchanged.
This test runs a plain Python restatement of that form on oracle-built graphs
and compares the results with the oracle's Alg. 5.
"""
import numpy as np
import pytest


def single_list_search(X, nbr0, nbrU, ep, maxlevel, q, K, ef, metric, cache_slots):
    def dist(i):
        x = X[i].astype(np.float64)
        qq = q.astype(np.float64)
        return float(((qq - x) ** 2).sum()) if metric == 0 else 1.0 - float((qq * x).sum())

    cur = (dist(ep), ep)
    for lc in range(maxlevel, 0, -1):  # greedy descent
        while True:
            best = cur
            for e in nbrU[lc].get(cur[1], []):
                k = (dist(e), e)
                if k < best:
                    best = k
            if best == cur:
                break
            cur = best
    efp = max(ef, K)
    W = [[cur, False]]  # sorted by key, flag = expanded
    # lossy direct-mapped visited set (cache_slots=None: an exact set)
    exact = set() if cache_slots is None else None
    cache = None if cache_slots is None else [-1] * cache_slots

    def seen_before(e):
        if exact is not None:
            if e in exact:
                return True
            exact.add(e)
            return False
        s = (e * 2654435761) % cache_slots
        if cache[s] == e:
            return True
        cache[s] = e
        return False

    seen_before(cur[1])
    n_eval = 1
    while True:
        j = next((i for i, (k, f) in enumerate(W) if not f), None)
        if j is None:
            break
        W[j][1] = True
        c = W[j][0][1]
        batch = []
        for e in nbr0[c]:
            if seen_before(e):
                continue
            batch.append((dist(e), e))
            n_eval += 1
        keys = {k for k, _ in W}
        full = len(W) >= efp
        furthest = W[-1][0]
        for k in batch:
            if k in keys or (full and k > furthest):
                continue
            W.append([k, False])
        W.sort(key=lambda t: t[0])
        del W[efp:]
    out = [k for k, _ in W[:K]]
    return [e for _, e in out], [d for d, _ in out], n_eval


@pytest.mark.parametrize("name,n,cache", [("tiny", 3000, 64), ("tiny", 3000, 4096), ("glove", 1500, 128)])
def test_single_list_equals_alg2(oracle, name, n, cache):
    from paper_1603_09320_gb300 import synth
    p = synth.params(name)
    X = synth.base(name, n)
    g = oracle.Graph.build(X, synth.level_uniforms(name, n), **p)
    lv = g.levels()
    nbr0 = {i: g.neighbors(i, 0) for i in range(n)}
    nbrU = {lc: {i: g.neighbors(i, lc) for i in range(n) if lv[i] >= lc} for lc in range(1, g.max_level + 1)}
    Q = synth.queries(name, 40)
    for K, ef in ((10, 10), (10, 40), (5, 3)):
        for i in range(Q.shape[0]):
            oi, od, st = g.knn_search(Q[i], K, ef, stats=True)
            si, sd, ne = single_list_search(X, nbr0, nbrU, g.enter_point, g.max_level, Q[i], K, ef,
                                            p["metric"], cache)
            m = min(len(si), K)
            assert oi[:m].tolist() == si
            if p["metric"] == 0:  # integer data: every distance is exact
                assert od[:m].tolist() == sd
            else:
                np.testing.assert_allclose(od[:m], sd, rtol=1e-12, atol=1e-12)
            # a lossy visited set can only add evaluations, never remove them
            _, _, exact = single_list_search(X, nbr0, nbrU, g.enter_point, g.max_level, Q[i], K,
                                             ef, p["metric"], None)
            assert ne >= exact
