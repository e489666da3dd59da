"""Pins for the oracle's per-node feature pre-screen (Sec. III-B, Algorithm
2: each feature's own split loss, the top n features kept, the swarm searches
their subspace).

Checked against things other than the oracle's own scoring: a per-edge brute
force over the binned feature with the textbook impurities, an exact ranking
(rational Gini scores, ties to the lower feature), the special cases n = d (no
pre-screen) and n = 1 (the best single feature's split, whichever sign the
one-dimensional swarm ends with), a planted problem whose informative
features are known, and the definition of the lifted search.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def brute_feature_loss(x, labels, K, B, min_leaf, crit):
    """Best split loss of one feature: B uniform bins on [min, max] computed
    in float as the mirror does, every interior edge scored directly."""
    x = x.astype(np.float32)
    lo, hi = x.min(), x.max()
    if not hi > lo:
        return None
    inv_w = np.float32(B) / np.float32(hi - lo)
    bins = np.floor((x - lo) * inv_w).astype(np.int64)
    bins = np.clip(bins, 0, B - 1)
    n = x.size
    best = None
    prev_nl = -1
    for b in range(1, B):
        left = bins < b
        nl = int(left.sum())
        nr = n - nl
        if nl == prev_nl:
            continue
        prev_nl = nl
        if nl < min_leaf or nr < min_leaf:
            continue
        loss = 0.0
        for side in (left, ~left):
            c = np.bincount(labels[side], minlength=K).astype(np.float64)
            p = c / c.sum()
            if crit == "gini":
                loss += c.sum() * (1.0 - (p ** 2).sum())
            else:
                nz = p[p > 0]
                loss += -c.sum() * (nz * np.log(nz)).sum()
        loss /= n
        if best is None or loss < best[0]:
            best = (loss, b)
    return best


@pytest.mark.parametrize("crit", ["gini", "entropy"])
def test_feature_scores_by_brute_force(crit):
    rng = np.random.default_rng(4)
    n, d, K, B = 400, 7, 3, 16
    X = rng.standard_normal((n, d)).astype(np.float32)
    X[:, 3] = np.round(X[:, 3])  # many equal values
    labels = ((X[:, 1] > 0.3).astype(np.int32) + (X[:, 5] > -0.5)).astype(np.int32)
    p = O.make_params(crit, K, n_bins=B, min_leaf=5)
    feat, ev, _ = O.select_features(p, X, labels, None, 3)
    for k in range(d):
        want = brute_feature_loss(X[:, k], labels, K, B, 5, crit)
        if want is None:
            assert not ev[k]["valid"]
            continue
        assert ev[k]["valid"] and ev[k]["bin"] == want[1]
        assert ev[k]["loss"] == pytest.approx(want[0], rel=1e-12, abs=1e-15)


def exact_order(ev, crit):
    """Features from best to worst score: Gini by the exact rational Q
    (larger is better), entropy by the loss; invalid last; ties to the lower
    feature."""
    def key(k):
        e = ev[k]
        if not e["valid"]:
            return (1, 0, k)
        if crit == "gini":
            return (0, -Fraction(int(e["q_num"]), int(e["q_den"])), k)
        return (0, e["loss"], k)
    return sorted(range(len(ev)), key=key)


@pytest.mark.parametrize("crit,n", [("gini", 1), ("gini", 4), ("entropy", 3), ("gini", 9)])
def test_selection_is_the_exact_ranking(crit, n):
    rng = np.random.default_rng(5)
    N, d, K = 600, 10, 4
    X = rng.standard_normal((N, d)).astype(np.float32)
    X[:, 6] = X[:, 2]  # an exact tie: the lower feature wins
    labels = (np.argmax(X[:, :K] + 0.5 * rng.standard_normal((N, K)), axis=1)).astype(np.int32)
    p = O.make_params(crit, K, n_bins=32, min_leaf=3)
    feat, ev, _ = O.select_features(p, X, labels, None, n)
    want = sorted(exact_order(ev, crit)[:n])
    assert list(feat) == want
    if n >= 3 and 6 in feat:
        assert 2 in feat


def test_top_n_equal_to_d_is_the_plain_search():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((500, 6)).astype(np.float32)
    labels = (X[:, 0] + X[:, 4] > 0).astype(np.int32)
    a = O.node_split(O.make_params("gini", 2, 16, 10, 32, min_leaf=2), X, labels, None)
    b = O.node_split(O.make_params("gini", 2, 16, 10, 32, min_leaf=2, top_n=6), X, labels, None)
    assert np.array_equal(a.gbest, b.gbest) and a.split == b.split


def test_top_1_reaches_the_best_single_feature():
    rng = np.random.default_rng(7)
    n, d, K, B = 800, 8, 2, 32
    X = rng.standard_normal((n, d)).astype(np.float32)
    labels = (X[:, 5] > 0.2).astype(np.int32)
    labels[rng.random(n) < 0.1] ^= 1
    p = O.make_params("gini", K, 8, 5, B, min_leaf=2, top_n=1)
    feat, ev, _ = O.select_features(p, X, labels, None, 1)
    assert list(feat) == [5]
    r = O.node_split(p, X, labels, None)
    assert np.count_nonzero(r.gbest) == 1 and r.gbest[5] != 0
    want = brute_feature_loss(X[:, 5], labels, K, B, 2, "gini")[0]
    # z = a x_5 for either sign of a: the same interior edges, mirrored
    assert r.split["loss"] == pytest.approx(want, rel=1e-6)


def test_planted_features_are_selected_and_searched():
    rng = np.random.default_rng(8)
    n, d = 2000, 12
    X = rng.standard_normal((n, d)).astype(np.float32)
    w = np.zeros(d)
    w[[3, 9]] = [0.8, -0.6]
    labels = (X.astype(np.float64) @ w > 0).astype(np.int32)
    p = O.make_params("entropy", 2, 24, 30, 64, min_leaf=2, top_n=2)
    feat, _, _ = O.select_features(p, X, labels, None, 2)
    assert list(feat) == [3, 9]
    r = O.node_split(p, X, labels, None)
    assert set(np.flatnonzero(r.gbest)) <= {3, 9}
    assert abs(r.direction @ (w / np.linalg.norm(w))) > 0.99


def test_lifted_search_is_the_subspace_search():
    rng = np.random.default_rng(9)
    n, d, K = 700, 9, 3
    X = rng.standard_normal((n, d)).astype(np.float32)
    labels = rng.integers(0, K, n).astype(np.int32)
    labels[X[:, 1] > 0.5] = 2
    idx = np.sort(rng.choice(n, 500, replace=False)).astype(np.int32)
    p = O.make_params("gini", K, 16, 12, 32, min_leaf=4, top_n=4, seed=3)
    feat, _, _ = O.select_features(p, X, labels, None, 4, idx=idx)
    r = O.node_split(p, X, labels, None, idx=idx, node_uid=21)
    q = O.make_params("gini", K, 16, 12, 32, min_leaf=4, seed=3)
    s = O.node_split(q, np.ascontiguousarray(X[:, feat]), labels, None, idx=idx, node_uid=21)
    lifted = np.zeros(d)
    lifted[feat] = s.gbest
    assert np.array_equal(r.gbest, lifted)
    assert r.split["loss"] == s.split["loss"] and r.split["bin"] == s.split["bin"]
    assert np.array_equal(r.trace_loss, s.trace_loss)
