"""Pins for the oracle's probabilistic search (Sec. II-B, the projection
search of the original SLM): candidate vectors follow Eqs. dynamic / exp_a
and the rank-ordered selection; the search returns the exact argmin over
its candidates as scored by a separate entry point (ora_eval_swarm), the
features are ranked by their own split losses, and the cosine pruning keeps
a greedy set whose pairwise cosines stay below the threshold."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W


def _key(e):
    """Sort key of a score: valid first, then better (Gini: larger Q)."""
    if not e["valid"]:
        return (1, 0)
    if e["q_den"]:
        return (0, -Fraction(int(e["q_num"]), int(e["q_den"])))
    return (0, e["loss"])


def test_candidates_follow_the_dynamic_range_and_selection():
    d = 12
    rank = np.random.default_rng(0).permutation(d).astype(np.int32)
    pp = O.make_prob(R=4, gamma=0.7, alpha0=9.0, alpha=0.2)
    cnt = np.zeros(d)
    for c in range(3000):
        a = O.prob_candidate(5, 17, c, rank, pp)
        assert np.all(a == np.round(a))               # integer coefficients (Eq. dynamic)
        nz = np.nonzero(a)[0]
        assert nz.size <= 4                          # R selected, zero draws allowed
        for f in nz:
            r = int(np.nonzero(rank == f)[0][0]) + 1  # 1-based rank of feature f
            assert abs(a[f]) <= math.floor(9.0 * math.exp(-0.2 * r))  # Eq. exp_a
            cnt[r - 1] += 1
        assert np.array_equal(a, O.prob_candidate(5, 17, c, rank, pp))  # counter-based
    # selection frequency falls with the rank (P_d decays)
    assert np.all(np.diff(cnt[:6]) < 0)
    # R = d selects every rank; gamma = 1 selects ranks uniformly
    full = O.make_prob(R=d, gamma=0.5, alpha0=100.0, alpha=0.0)
    sel = np.zeros(d)
    for c in range(200):
        sel += O.prob_candidate(1, 2, c, rank, full) != 0
    assert np.all(sel >= 190)  # only zero draws (1 in 201) leave a rank out
    flat = O.make_prob(R=1, gamma=1.0, alpha0=100.0, alpha=0.0)
    hit = np.zeros(d)
    for c in range(6000):
        hit[np.nonzero(O.prob_candidate(3, 4, c, rank, flat))[0]] += 1
    assert hit.min() > 0.8 * 500 and hit.max() < 1.2 * 500


@pytest.mark.parametrize("crit,precision", [("gini", O.F32_MIRROR), ("entropy", O.F32_MIRROR),
                                            ("mse", O.F32_MIRROR), ("gini", O.F64)])
def test_search_is_the_argmin_over_its_candidates(crit, precision):
    if crit == "mse":
        wl = W.tanh_regression(700, 6, seed=3)
        kw = dict(y=wl.y)
        K = 0
    else:
        wl = W.gmm(700, 6, 3, seed=3)
        kw = dict(labels=wl.labels)
        K = 3
    p = O.make_params(crit, K, n_bins=32, min_leaf=5, seed=9, precision=precision)
    pp = O.make_prob(n_candidates=150, R=3, gamma=0.8, alpha0=6.0, alpha=0.1, batch=40, q=3)
    r = O.prob_search(p, pp, wl.X, node_uid=4, **kw)
    # the features' own scores, through ora_eval_swarm
    eye = np.eye(6)
    fe, _, _ = O.eval_swarm(p, wl.X, kw.get("labels"), kw.get("y"), eye)
    assert list(r.rank_feat) == sorted(range(6), key=lambda k: (_key(fe[k]), k))
    cands = np.array([O.prob_candidate(9, 4, c, r.rank_feat, pp) for c in range(150)])
    ev, _, _ = O.eval_swarm(p, wl.X, kw.get("labels"), kw.get("y"), cands)
    best = min(range(150), key=lambda c: (_key(ev[c]), c))
    assert r.split["particle"] == best and np.array_equal(r.best, cands[best])
    assert r.split["bin"] == ev[best]["bin"] and r.split["loss"] == ev[best]["loss"]
    # the trace is the best so far after each batch of 40
    for b, tl in enumerate(r.trace_loss):
        upto = min(150, (b + 1) * 40)
        bb = min(range(upto), key=lambda c: (_key(ev[c]), c))
        assert tl == (ev[bb]["loss"] if ev[bb]["valid"] else np.inf)
    # cosine pruning: greedy, best first, pairwise cos^2 <= 0.81 among the kept
    kept = list(r.kept)
    assert kept and kept[0] == best
    alive = [c for c in range(150) if np.any(cands[c])]
    order = []
    while alive and len(order) < 3:
        b = min(alive, key=lambda c: (_key(ev[c]), c))
        order.append(b)
        a = cands[b]
        alive = [c for c in alive if c != b and
                 100 * int(a @ cands[c]) ** 2 <= 81 * int(a @ a) * int(cands[c] @ cands[c])]
    assert kept == order


def test_planted_single_feature_is_found():
    """Labels set by feature 4 alone: it ranks first, and with one
    coefficient per candidate the best split is that feature's own split."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((1000, 8)).astype(np.float32)
    lab = (X[:, 4] > 0.3).astype(np.int32)
    p = O.make_params("gini", 2, n_bins=64, min_leaf=5, seed=2)
    pp = O.make_prob(n_candidates=64, R=1, gamma=0.2, alpha0=3.0, alpha=0.0)
    r = O.prob_search(p, pp, X, lab, node_uid=1)
    assert r.rank_feat[0] == 4
    own = O.eval_swarm(p, X, lab, None, np.eye(8)[[4]])[0][0]
    assert r.split["loss"] == own["loss"]
    assert np.count_nonzero(r.best) == 1 and r.best[4] != 0
