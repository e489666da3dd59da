"""GPU parity of adaptive PSO (params.apso; Sec. III-B) against the oracle.

* searches: the fp32-mirror oracle's trajectory, gB and split (Gini exactly;
  entropy up to a near-tie the oracle logs), in cases where the oracle scored
  elite candidates, both accepted as gB and put in the worst particle's place;
* trees and bagged forests: every node as the oracle's, with and without
  graph capture of the search;
* unsupported combinations are rejected.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, oracle_params
from tests.test_gpu_parity import _compare_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def params(S, crit, K, P, T, B, **kw):
    return S.make_params(crit, K, n_particles=P, n_iters=T, n_bins=B, apso=True, **kw)


def oparams(crit, K, P, T, B, min_leaf=1, seed=1, max_depth=8):
    op = oracle_params(O, crit, K, P, T, B, min_leaf=min_leaf, seed=seed, max_depth=max_depth)
    op.apso = 1
    return op


@pytest.mark.parametrize("crit,K,B,d,n,P,T,accepts", [
    ("gini", 4, 64, 16, 3000, 32, 40, False),   # elite candidates replace the worst
    ("entropy", 2, 64, 16, 2000, 32, 50, None),  # the single-node setting
    ("gini", 10, 128, 64, 6000, 64, 25, False),
    ("gini", 3, 32, 5, 500, 7, 30, True),       # P not a multiple of 16; accepted elites
    ("gini", 3, 32, 5, 500, 15, 30, None),      # P + 1 fills the padded slots
])
def test_apso_search_matches_oracle(ctx, crit, K, B, d, n, P, T, accepts):
    from paper_2208_07023_gb300 import binding as S
    wl = W.single_node(n, d, seed=3) if K == 2 else W.gmm(n, d, K, seed=P + d)
    gp = params(S, crit, K, P, T, B, min_leaf=2, seed=21)
    g = ctx.node_split(gp, wl.X, labels=wl.labels, node_uid=12, want_trace=True)
    r = O.node_split(oparams(crit, K, P, T, B, min_leaf=2, seed=21), wl.X, wl.labels,
                     node_uid=12)
    stop = r.split["first_near_tie"]
    upto = T + 1 if stop < 0 else stop
    assert np.array_equal(g["trace"][:upto], r.trace_loss[:upto])
    assert r.split["elite_tries"] > 0
    if accepts is not None:
        assert (r.split["elite_accepts"] > 0) == accepts
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
        assert (g["particle"], g["iter_of_best"], g["bin"]) == \
            (r.split["particle"], r.split["iter_of_best"], r.split["bin"])
        assert g["loss"] == r.split["loss"]


@pytest.mark.parametrize("bootstrap,graphs", [(False, False), (True, False), (True, True)])
def test_apso_tree_matches_oracle(ctx, bootstrap, graphs):
    from paper_2208_07023_gb300 import binding as S
    n, d, K, depth, P, T, B = 4000, 12, 5, 5, 24, 15, 64
    wl = W.gmm(n, d, K, seed=11)
    gp = params(S, "gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=5,
                n_trees=2 if bootstrap else 1, bootstrap=bootstrap)
    ctx.set_graphs(graphs)
    try:
        f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    finally:
        ctx.set_graphs(False)
    op = oparams("gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=5)
    for t in range(2 if bootstrap else 1):
        g = f.export(t)
        r = O.train_tree(op, wl.X, wl.labels, tree_id=t, bootstrap=bootstrap)
        inner, present = _compare_tree(g, r, d)
        assert np.array_equal(g["loss"][inner], r.loss[inner])
    f.free()


def test_apso_with_feature_prescreen_matches_oracle(ctx):
    # the pre-screen's subspace search runs adaptive PSO (its elite slot in the
    # subspace's swarm); gB lifted back to d features
    from paper_2208_07023_gb300 import binding as S
    n, d, K, P, T, B, top_n = 3000, 24, 4, 24, 20, 64, 6
    wl = W.gmm(n, d, K, seed=41)
    gp = params(S, "gini", K, P, T, B, min_leaf=3, seed=9, top_n=top_n)
    g = ctx.node_split(gp, wl.X, labels=wl.labels, node_uid=5, want_trace=True)
    op = oparams("gini", K, P, T, B, min_leaf=3, seed=9)
    op.top_n = top_n
    r = O.node_split(op, wl.X, wl.labels, node_uid=5)
    assert r.split["elite_tries"] > 0
    assert np.array_equal(g["trace"], r.trace_loss)
    assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
    assert np.count_nonzero(g["gbest"]) <= top_n
    assert (g["particle"], g["iter_of_best"], g["bin"]) == \
        (r.split["particle"], r.split["iter_of_best"], r.split["bin"])


def test_apso_changes_the_search_and_finds_the_planted_direction(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.single_node(2000, 16, 0.05, seed=9)
    a = ctx.node_split(params(S, "entropy", 2, 32, 50, 64, seed=4), wl.X, labels=wl.labels,
                       want_trace=True)
    b = ctx.node_split(S.make_params("entropy", 2, n_particles=32, n_iters=50, n_bins=64,
                                     seed=4), wl.X, labels=wl.labels, want_trace=True)
    assert a["trace"][0] == b["trace"][0] and not np.array_equal(a["trace"], b["trace"])
    assert abs(a["direction"] @ wl.meta["w"]) > 0.99


def test_unsupported_apso_is_rejected(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(500, 8, 3, seed=2)
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(params(S, "gini", 3, 16, 2, 32, proj=S.SLM_PROJ_BF16_TOPK, topk=4),
                       wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EUNSUPPORTED
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(params(S, "gini", 3, 256, 2, 32), wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EUNSUPPORTED
    ctx.node_split(params(S, "gini", 3, 255, 2, 32), wl.X, labels=wl.labels)
    p = params(S, "gini", 3, 16, 2, 32)
    p.apso = 2
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(p, wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EINVAL
