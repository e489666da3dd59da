"""GPU parity of the per-node feature pre-screen (params.top_n) against the
oracle (Sec. III-B, Algorithm 2: every feature scored on its own, the top n
kept, the swarm searching their subspace, gB lifted back).

* searches: the fp32-mirror oracle's trajectory, gB (lifted, zeros outside
  the kept features) and split, up to a near-tie the oracle logs;
* trees: every node as the oracle's (Gini: exact);
* top_n = d is the plain search; unsupported combinations are rejected.
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


def params(S, crit, K, P, T, B, top_n, **kw):
    return S.make_params(crit, K, n_particles=P, n_iters=T, n_bins=B, top_n=top_n, **kw)


def oparams(crit, K, P, T, B, top_n, min_leaf=1, seed=1, max_depth=8):
    op = oracle_params(O, crit, K, P, T, B, min_leaf=min_leaf, seed=seed, max_depth=max_depth)
    op.top_n = top_n
    return op


@pytest.mark.parametrize("crit,K,B,d,n,P,T,top_n", [
    ("gini", 4, 64, 16, 3000, 32, 20, 5),
    ("entropy", 2, 64, 32, 2000, 32, 30, 4),
    ("gini", 6, 128, 64, 5000, 48, 10, 12),
    ("gini", 3, 32, 9, 700, 20, 25, 1),
])
def test_prescreened_search_matches_oracle(ctx, crit, K, B, d, n, P, T, top_n):
    from paper_2208_07023_gb300 import binding as S
    wl = W.single_node(n, d, seed=4) if K == 2 else W.gmm(n, d, K, seed=d + n)
    rng = np.random.default_rng(d)
    idx = np.sort(rng.choice(n, int(0.8 * n), replace=False)).astype(np.int32)
    gp = params(S, crit, K, P, T, B, top_n, min_leaf=3, seed=17)
    g = ctx.node_split(gp, wl.X, labels=wl.labels, sample_idx=idx, node_uid=33,
                       want_trace=True)
    op = oparams(crit, K, P, T, B, top_n, min_leaf=3, seed=17)
    feat, _, _ = O.select_features(op, wl.X, wl.labels, None, top_n, idx=idx)
    r = O.node_split(op, wl.X, wl.labels, idx=idx, node_uid=33)
    stop = r.split["first_near_tie"]
    upto = T + 1 if stop < 0 else stop
    assert np.array_equal(g["trace"][:upto], r.trace_loss[:upto])
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
        assert set(np.flatnonzero(g["gbest"])) <= set(feat.tolist())
        assert (g["particle"], g["iter_of_best"], g["bin"]) == \
            (r.split["particle"], r.split["iter_of_best"], r.split["bin"])
        assert g["loss"] == r.split["loss"]


def test_prescreened_regression_search(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(4000, 24, seed=5)
    gp = params(S, "mse", 0, 32, 15, 64, 6, min_leaf=10, seed=2)
    g = ctx.node_split(gp, wl.X, y=wl.y, node_uid=4, want_trace=True)
    op = oparams("mse", 0, 32, 15, 64, 6, min_leaf=10, seed=2)
    r = O.node_split(op, wl.X, None, wl.y, node_uid=4)
    stop = r.split["first_near_tie"]
    upto = 16 if stop < 0 else stop
    assert np.allclose(g["trace"][:upto], r.trace_loss[:upto], rtol=1e-9, atol=0)
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)


@pytest.mark.parametrize("bootstrap", [False, True])
def test_prescreened_tree_matches_oracle(ctx, bootstrap):
    from paper_2208_07023_gb300 import binding as S
    n, d, K, depth, P, T, B, top_n = 4000, 20, 5, 5, 24, 12, 64, 6
    wl = W.gmm(n, d, K, seed=7)
    gp = params(S, "gini", K, P, T, B, top_n, min_leaf=10, max_depth=depth, seed=3,
                n_trees=2 if bootstrap else 1, bootstrap=bootstrap)
    f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    op = oparams("gini", K, P, T, B, top_n, min_leaf=10, max_depth=depth, seed=3)
    for t in range(2 if bootstrap else 1):
        g = f.export(t)
        r = O.train_tree(op, wl.X, wl.labels, tree_id=t, bootstrap=bootstrap)
        inner, present = _compare_tree(g, r, d)
        assert np.array_equal(g["loss"][inner], r.loss[inner])
        # every direction lives on at most top_n features
        dirs = np.asarray(g["dir"]).reshape(-1, d)[np.asarray(g["kind"]).reshape(-1) == 1]
        assert len(dirs) > 0 and (np.count_nonzero(dirs, axis=1) <= top_n).all()
    f.free()


def test_top_n_equal_to_d_is_the_plain_search(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(2000, 12, 3, seed=8)
    a = ctx.node_split(params(S, "gini", 3, 16, 10, 32, 0, seed=5), wl.X, labels=wl.labels,
                       want_trace=True)
    b = ctx.node_split(params(S, "gini", 3, 16, 10, 32, 12, seed=5), wl.X, labels=wl.labels,
                       want_trace=True)
    assert np.array_equal(a["trace"], b["trace"]) and np.array_equal(a["gbest"], b["gbest"])


def test_unsupported_prescreens_are_rejected(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(500, 8, 3, seed=9)
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(params(S, "gini", 3, 16, 2, 32, -1), wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(params(S, "gini", 3, 16, 2, 32, 3, proj=S.SLM_PROJ_BF16_TOPK, topk=4),
                       wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EUNSUPPORTED
    Xw = np.random.default_rng(1).standard_normal((300, 300)).astype(np.float32)
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(params(S, "gini", 3, 16, 2, 32, 10), Xw, labels=wl.labels[:300])
    assert e.value.status == S.SLM_EUNSUPPORTED
