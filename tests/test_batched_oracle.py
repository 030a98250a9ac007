"""Pins of the oracle's batched construction (orc_build_batched: Alg. 1 with
the layer-0 insertions grouped in batches that search the graph as it stood
before the batch, the batch form of Section 4.1's parallel construction):

* with batches of one element it IS Alg. 1, applied in the order seed, then
  the rest (byte-identical to orc_insert in that order), for Alg. 3, Alg. 4
  and Alg. 4 with keepPrunedConnections, squared L2 and cosine;
* with every element in the seed it is orc_build;
* with the growing schedule, elements of one batch never link to one
  another, the graph is valid, and its recall matches the sequential one's.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1603_09320_gb300 import synth


def _levels(u, M):
    return np.array([O.level_from_u(float(x), 1.0 / np.log(M)) for x in u])


def _order(lv, n_first):
    seed = [i for i in range(len(lv)) if i < n_first or lv[i] > 0]
    rest = [i for i in range(len(lv)) if not (i < n_first or lv[i] > 0)]
    return seed, rest


def _schedule(n_seed, n_rest):
    """Batch sizes of the growing schedule."""
    bmax = min(32768, max(64, n_rest))
    out, pos, inserted = [], 0, n_seed
    while pos < n_rest:
        b = min(bmax, n_rest - pos, max(64, inserted // 16))
        out.append(b)
        pos += b
        inserted += b
    return out


@pytest.mark.parametrize("name,heuristic,keep", [("tiny", True, False), ("tiny", False, False),
                                                 ("tiny", True, True), ("glove", True, False)])
def test_batch_of_one_is_sequential_alg1(name, heuristic, keep):
    p = dict(synth.params(name))
    if name == "glove":
        p["efC"] = 40
    N = 2500
    X = synth.base(name, N)
    u = synth.level_uniforms(name, N)
    gb = O.Graph.build_batched(X, u, n_first=300, batch=1, heuristic=heuristic, keep_pruned=keep, **p)
    lv = _levels(u, p["M"])
    seed, rest = _order(lv, 300)
    gs = O.Graph.new(X, heuristic=heuristic, keep_pruned=keep, **p)
    for i in seed + rest:
        gs.insert(i, int(lv[i]))
    assert gb.to_blob() == gs.to_blob()


def test_all_seed_is_orc_build():
    p = synth.params("tiny")
    X = synth.base("tiny", 1500)
    u = synth.level_uniforms("tiny", 1500)
    assert O.Graph.build_batched(X, u, n_first=1500, **p).to_blob() == O.Graph.build(X, u, **p).to_blob()


def test_growing_batches():
    p = synth.params("tiny")
    N = 8000
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N)
    n_first = 1000
    g = O.Graph.build_batched(X, u, n_first=n_first, **p)
    g = O.Graph.from_blob(g.to_blob())  # validating loader
    lv = _levels(u, p["M"])
    seed, rest = _order(lv, n_first)
    sizes = _schedule(len(seed), len(rest))
    assert sizes[0] == max(64, len(seed) // 16) and len(sizes) > 5 and sum(sizes) == len(rest)
    batch_of = {}
    pos = 0
    for k, b in enumerate(sizes):
        for i in rest[pos:pos + b]:
            batch_of[i] = k
        pos += b
    for i in rest:  # no link inside a batch, in either direction
        assert all(batch_of.get(j) != batch_of[i] for j in g.neighbors(i, 0))
    for i in range(N):
        nb = g.neighbors(i, 0)
        assert 1 <= len(nb) <= p["Mmax0"] and i not in nb and len(set(nb)) == len(nb)
    # upper layers: Alg. 1 over the seed, as in the sequential build of the seed
    gs = O.Graph.new(X, **p)
    for i in seed:
        gs.insert(i, int(lv[i]))
    assert g.enter_point == gs.enter_point and g.max_level == gs.max_level
    for i in seed:
        for lc in range(1, int(lv[i]) + 1):
            assert g.neighbors(i, lc) == gs.neighbors(i, lc)
    # as good a graph as sequential insertion
    full = O.Graph.build(X, u, **p)
    Q = synth.queries("tiny", 300)
    gt, _ = O.brute_force(X, Q, 10)

    def recall(h, ef):
        ids, _ = h.knn_search_batch(Q, 10, ef)
        return np.mean([len(set(ids[i].tolist()) & set(gt[i].tolist())) / 10 for i in range(len(Q))])

    for ef in (16, 48):
        assert recall(g, ef) >= recall(full, ef) - 0.02


def test_extend_candidates_is_rejected():
    p = synth.params("tiny")
    X = synth.base("tiny", 200)
    with pytest.raises(RuntimeError):
        O.Graph.build_batched(X, synth.level_uniforms("tiny", 200), extend=True, **p)


def _sequential(X, u, n0, p):
    lv = _levels(u, p["M"])
    g = O.Graph.new(X, **p)
    for i in range(n0):
        g.insert(i, int(lv[i]))
    return g, lv


def test_incremental_level0_batch_of_one_is_sequential_alg1():
    # new elements all of level 0 (u = 1): batches of one are Alg. 1 in id order
    p = synth.params("tiny")
    N, n0 = 3000, 1200
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N).copy()
    u[n0:] = 1.0
    g, lv = _sequential(X, u, n0, p)
    g.insert_batched(n0, u[n0:2000], batch=1)
    g.insert_batched(2000, u[2000:], batch=1)
    ref = O.Graph.build(X, u, **p)
    assert g.to_blob() == ref.to_blob()


def test_incremental_upper_layers_are_sequential_alg1():
    # levels >= 1 among the new elements: their upper layers are Alg. 1 over
    # all elements in id order (layers >= 1 involve only elements of level >= 1)
    p = synth.params("tiny")
    N, n0 = 6000, 2500
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N)
    g, lv = _sequential(X, u, n0, p)
    for lo, hi in ((n0, 4000), (4000, N)):
        g.insert_batched(lo, u[lo:hi])
    g = O.Graph.from_blob(g.to_blob())
    full = O.Graph.build(X, u, **p)
    assert g.enter_point == full.enter_point and g.max_level == full.max_level
    assert np.array_equal(g.levels(), full.levels())
    for i in np.nonzero(lv > 0)[0]:
        for lc in range(1, int(lv[i]) + 1):
            assert g.neighbors(int(i), lc) == full.neighbors(int(i), lc)
    for i in range(N):
        nb = g.neighbors(i, 0)
        assert 1 <= len(nb) <= p["Mmax0"] and i not in nb and len(set(nb)) == len(nb)
    Q = synth.queries("tiny", 300)
    gt, _ = O.brute_force(X, Q, 10)
    for ef in (16, 48):
        r = [np.mean([len(set(ids[i].tolist()) & set(gt[i].tolist())) / 10 for i in range(len(Q))])
             for ids in (h.knn_search_batch(Q, 10, ef)[0] for h in (g, full))]
        assert r[0] >= r[1] - 0.02


def test_incremental_rejects_bad_ranges():
    p = synth.params("tiny")
    X = synth.base("tiny", 500)
    u = synth.level_uniforms("tiny", 500)
    g, _ = _sequential(X, u, 300, p)
    with pytest.raises(RuntimeError):
        g.insert_batched(200, u[200:300])  # already inserted
    with pytest.raises(RuntimeError):
        g.insert_batched(350, u[350:400])  # not contiguous with the graph
    with pytest.raises(RuntimeError):
        g.insert_batched(300, np.ones(300))  # beyond the rows
    g.insert_batched(300, u[300:500])
    assert g.N == 500


def test_explicit_schedule_is_the_default_schedule():
    """The batch sizes are a free parameter of the batch form; the default is
    the growing schedule max(64, inserted / 16) (at most 32,768, at most what
    remains).  Passing that schedule explicitly, computed here, gives the
    same graph byte for byte, and a different schedule gives another graph."""
    p = synth.params("tiny")
    N, n_first = 6000, 500
    X = synth.base("tiny", N)
    u = synth.level_uniforms("tiny", N)
    seed, rest = _order(_levels(u, p["M"]), n_first)
    sizes = _schedule(len(seed), len(rest))
    g0 = O.Graph.build_batched(X, u, n_first=n_first, **p).to_blob()
    g1 = O.Graph.build_batched(X, u, n_first=n_first, batch_sizes=sizes, **p).to_blob()
    assert g0 == g1
    g2 = O.Graph.build_batched(X, u, n_first=n_first, batch_sizes=[sizes[0] * 2], **p).to_blob()
    assert g2 != g0


def test_shrink_takes_all_of_econn_when_a_list_gets_over_256_new_links():
    """Alg. 1 shrinks an overfull list over the whole of eConn.  The hub input sends
    all 301 ray points of one batch to the hub: its list then holds, by
    Alg. 4 worked by hand, the t = 1 point of rays 0..9 (each closer to the
    hub, at 1, than to any other accepted point, at 2; every further point of
    a ray is closer to that ray's t = 1 point than to the hub; every filler f
    is closer to the t = 1 point of ray k than to the hub, since f_k - 100 >=
    80) and the t = 40 point of ray 10 (1,600 from the hub against 1,601 to
    each t = 1 point).  That point is the 301st candidate by distance: a
    shrink over the 256 closest would miss it."""
    import _hub
    X, u = _hub.hub_input()
    n = X.shape[0]
    seed, rest = _order(_levels(u, _hub.PARAMS["M"]), _hub.N_SEED)
    sizes = _schedule(len(seed), len(rest))
    assert sizes == list(_hub.FILL_BATCHES) + [_hub.RAYS]
    g = O.Graph.build_batched(X, u, n_first=_hub.N_SEED, **_hub.PARAMS)
    first, near, far = _hub.ray_ids(n)
    # every ray point of the last batch linked to the hub: 301 > 256 new links
    assert all(0 in g.neighbors(i, 0) for i in range(first, n))
    assert g.neighbors(0, 0) == near + [far]
    # the far point's rank among the hub's candidates (all 301 ray points
    # precede every filler: squared distances <= 1,600 against >= 102,400)
    d2 = ((X[first:] - X[0]) ** 2).sum(1)
    assert int(np.sum(d2 < d2[-1])) == _hub.RAYS - 1 > 256
