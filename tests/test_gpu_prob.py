"""GPU parity of the probabilistic search (Sec. II-B: the projection search
of the original SLM, kept as a baseline for the swarm search) against the
oracle's fp32-mirror restatement, on the same seeded inputs:

* the feature ranking, every batch's best loss, the best candidate's index,
  vector, bin and split, and the cosine pruning's kept candidates: exact;
* ragged last batches, R above d (taken as d), gamma = 1 (uniform ranks),
  ranges that give only zero vectors, q = 0, sample subsets with
  multiplicities, regression, and d above 256 (the ranking in chunks);
* arguments outside the documented ranges are rejected.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def _pair(S, I, R, gamma, alpha0, alpha, batch, q, cn=9, cd=10):
    return (S.make_prob(I, R, gamma, alpha0, alpha, batch, q, cn, cd),
            O.make_prob(I, R, gamma, alpha0, alpha, batch, q, cn, cd))


def _compare(g, r, d):
    assert np.array_equal(g["rank_feat"], r.rank_feat)
    assert np.array_equal(g["trace"], r.trace_loss)
    assert g["particle"] == r.split["particle"]
    assert g["iter_of_best"] == r.split["iter_of_best"]
    assert np.array_equal(g["best"].astype(np.float64), r.best)
    assert g["valid"] == r.split["valid"]
    if g["valid"]:
        for k in ("bin", "loss", "n_left", "n_right"):
            assert g[k] == r.split[k], k
        assert g["threshold"] == np.float32(r.split["threshold"])
        nrm = np.linalg.norm(r.best)
        assert np.allclose(g["direction"], r.best / nrm, atol=1e-6)
    assert np.array_equal(g["kept"], r.kept)


@pytest.mark.parametrize("crit,K,B,d,n,I,R,gamma,alpha0,alpha,batch,q,n_kept", [
    ("gini", 4, 64, 16, 3000, 1000, 4, 0.8, 8.0, 0.05, 64, 4, 4),     # ragged last batch
    ("entropy", 3, 128, 32, 4000, 500, 6, 0.9, 12.0, 0.1, 100, 8, 8),
    ("gini", 6, 32, 8, 2000, 300, 12, 1.0, 3.0, 0.0, 256, 5, 5),      # R > d, uniform ranks
    ("gini", 10, 128, 64, 6000, 700, 3, 0.7, 20.0, 0.02, 37, 16, 16),
    # one coefficient, and only rank 1 has a nonzero range (floor(1.5 e^-0.3)
    # = 1, floor(1.5 e^-0.6) = 0): every candidate is 0 or +-e of the best
    # feature, one direction to keep
    ("entropy", 2, 64, 5, 800, 129, 1, 0.5, 1.5, 0.3, 16, 3, 1),
])
def test_prob_search_matches_oracle(ctx, crit, K, B, d, n, I, R, gamma, alpha0, alpha, batch,
                                    q, n_kept):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(n, d, K, seed=d + I)
    rng = np.random.default_rng(I)
    idx = np.sort(rng.choice(n, int(0.85 * n), replace=False)).astype(np.int32)
    sp, op = _pair(S, I, R, gamma, alpha0, alpha, batch, q)
    g = ctx.prob_search(gpu_params(S, crit, K, 1, 0, B, min_leaf=3, seed=21), sp, wl.X,
                        labels=wl.labels, sample_idx=idx, node_uid=9)
    r = O.prob_search(oracle_params(O, crit, K, 1, 0, B, min_leaf=3, seed=21), op, wl.X,
                      wl.labels, idx=idx, node_uid=9)
    _compare(g, r, d)
    assert g["valid"] and len(g["kept"]) == n_kept


def test_prob_search_weighted_and_regression(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(2500, 12, 5, seed=3)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 2500, 2000).astype(np.int32)
    idx, wts = np.unique(idx, return_counts=True)
    idx, wts = idx.astype(np.int32), wts.astype(np.uint32)
    sp, op = _pair(S, 400, 5, 0.85, 6.0, 0.05, 64, 6)
    g = ctx.prob_search(gpu_params(S, "gini", 5, 1, 0, 64, min_leaf=2, seed=8), sp, wl.X,
                        labels=wl.labels, sample_idx=idx, weights=wts, node_uid=31)
    r = O.prob_search(oracle_params(O, "gini", 5, 1, 0, 64, min_leaf=2, seed=8), op, wl.X,
                      wl.labels, idx=idx, wts=wts, node_uid=31)
    _compare(g, r, 12)
    rg = W.tanh_regression(3000, 10, seed=7)
    sp, op = _pair(S, 300, 4, 0.8, 8.0, 0.05, 64, 4)
    g = ctx.prob_search(gpu_params(S, "mse", 0, 1, 0, 64, min_leaf=5, seed=2), sp, rg.X,
                        y=rg.y, node_uid=3)
    r = O.prob_search(oracle_params(O, "mse", 0, 1, 0, 64, min_leaf=5, seed=2), op, rg.X,
                      None, rg.y, node_uid=3)
    assert np.array_equal(g["rank_feat"], r.rank_feat)
    assert np.array_equal(g["best"].astype(np.float64), r.best)
    assert g["particle"] == r.split["particle"] and g["bin"] == r.split["bin"]
    assert np.allclose(g["trace"], r.trace_loss, rtol=1e-9)
    assert np.array_equal(g["kept"], r.kept)


def test_prob_search_wide_node(ctx):
    """d = 300: the features are ranked in two scoring chunks."""
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(3000, 300, 4, seed=13)
    sp, op = _pair(S, 200, 8, 0.95, 10.0, 0.01, 128, 3)
    g = ctx.prob_search(gpu_params(S, "gini", 4, 1, 0, 64, min_leaf=2, seed=6), sp, wl.X,
                        labels=wl.labels, node_uid=2)
    r = O.prob_search(oracle_params(O, "gini", 4, 1, 0, 64, min_leaf=2, seed=6), op, wl.X,
                      wl.labels, node_uid=2)
    _compare(g, r, 300)


def test_prob_search_degenerate(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(1000, 6, 3, seed=1)
    gp = gpu_params(S, "gini", 3, 1, 0, 32, min_leaf=2, seed=4)
    opp = oracle_params(O, "gini", 3, 1, 0, 32, min_leaf=2, seed=4)
    # alpha0 < 1: every coefficient range is {0}, so every candidate is the
    # zero vector: no valid split, nothing kept
    sp, op = _pair(S, 70, 3, 0.8, 0.9, 0.0, 32, 4)
    g = ctx.prob_search(gp, sp, wl.X, labels=wl.labels, node_uid=1)
    r = O.prob_search(opp, op, wl.X, wl.labels, node_uid=1)
    _compare(g, r, 6)
    assert not g["valid"] and len(g["kept"]) == 0 and np.all(np.isinf(g["trace"]))
    # q = 0 and a single candidate
    sp, op = _pair(S, 1, 2, 0.8, 5.0, 0.1, 64, 0)
    g = ctx.prob_search(gp, sp, wl.X, labels=wl.labels, node_uid=4)
    r = O.prob_search(opp, op, wl.X, wl.labels, node_uid=4)
    _compare(g, r, 6)
    # cos threshold 1 prunes only exact multiples (and the kept one itself)
    sp, op = _pair(S, 300, 2, 0.6, 4.0, 0.0, 64, 50, cn=1, cd=1)
    g = ctx.prob_search(gp, sp, wl.X, labels=wl.labels, node_uid=5)
    r = O.prob_search(opp, op, wl.X, wl.labels, node_uid=5)
    _compare(g, r, 6)


def test_prob_search_rejects_bad_arguments(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(500, 6, 3, seed=2)
    gp = gpu_params(S, "gini", 3, 1, 0, 32)
    for kw in ({"n_candidates": 0}, {"R": 0}, {"R": 65}, {"gamma": 0.0}, {"gamma": 1.5},
               {"alpha0": -1.0}, {"alpha0": 101.0}, {"alpha": -0.1}, {"batch": 0},
               {"batch": 257}, {"q": -1}, {"cos_den": 0}, {"cos_num": 11}):
        sp = S.make_prob(**{**dict(n_candidates=10), **kw})
        with pytest.raises(S.SlmError) as e:
            ctx.prob_search(gp, sp, wl.X, labels=wl.labels)
        assert e.value.status == S.SLM_EINVAL, kw
