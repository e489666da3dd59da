"""Pins for the oracle's reduced-precision search mode (ORA_BF16_TOPK).

The mode scores every particle on a bfloat16 projection (row and position
rounded to bfloat16, exact dot product rounded once to float), re-scores the
top-k on the float mirror projection, feeds pbest the re-scored value where
there is one and picks gbest among the re-scored particles only.

Pins: bfloat16 rounding against torch's conversion (a library routine); the
projection against exact rational arithmetic; scores against a brute force
over the bins; the top-k merge against a brute-force ranking; the special
case k = P, where the mode must reduce to the float mirror search exactly.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W

torch = pytest.importorskip("torch")


def torch_bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy()


def f32_nearest(fr: Fraction) -> np.float32:
    """Nearest float32 (ties to even) of an exact rational, normal range."""
    if fr == 0:
        return np.float32(0.0)
    sign = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scaled = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q, r = divmod(scaled.numerator, scaled.denominator)
    if 2 * r > scaled.denominator or (2 * r == scaled.denominator and q & 1):
        q += 1
    return np.float32(sign * q * 2.0 ** (e - 23))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(3)
    vals = np.concatenate([
        rng.standard_normal(4000).astype(np.float32) * np.float32(10.0) ** rng.integers(-30, 30, 4000),
        np.float32([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -126, 3e-41,
                    -1e-45, 3.389e38, 3.4e38, -3.4e38, 0.0, -0.0, np.inf, -np.inf]),
    ]).astype(np.float32)
    ours = O.bf16_round(vals)
    ref = torch_bf16(vals)
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    nan = O.bf16_round(np.float32([np.nan]))
    assert np.isnan(nan[0])


def bf16_params(**kw):
    base = dict(criterion="gini", n_classes=3, n_particles=6, n_iters=0, n_bins=16,
                min_leaf=2, precision=O.BF16_TOPK, topk=0)
    base.update(kw)
    return O.make_params(**base)


def test_bf16_projection_is_rounded_exact_dot():
    rng = np.random.default_rng(5)
    n, d, P = 60, 37, 5
    X = rng.standard_normal((n, d)).astype(np.float32)
    lab = rng.integers(0, 3, n).astype(np.int32)
    pos = rng.uniform(-1, 1, (P, d)).astype(np.float32).astype(np.float64)
    _, _, z = O.eval_swarm(bf16_params(n_particles=P), X, lab, None, pos, want_z=True)
    Xb = torch_bf16(X)
    Ab = torch_bf16(pos.astype(np.float32))
    for i in range(P):
        for s in range(0, n, 7):
            exact = sum(Fraction(float(Xb[s, j])) * Fraction(float(Ab[i, j])) for j in range(d))
            assert z[i, s] == float(f32_nearest(exact)), (i, s)


def edge_losses_from_bins(bins, lab, yv, w, B, K, crit, min_leaf):
    best, best_b = np.inf, -1
    for b in range(1, B):
        left = bins < b
        nl, nr = w[left].sum(), w[~left].sum()
        if nl < min_leaf or nr < min_leaf:
            continue
        tot = 0.0
        for side in (left, ~left):
            ws = w[side]
            ns = ws.sum()
            if crit == "mse":
                ybar = (ws * yv[side]).sum() / ns
                tot += (ws * (yv[side] - ybar) ** 2).sum()
            else:
                p = np.bincount(lab[side], weights=ws, minlength=K) / ns
                if crit == "gini":
                    tot += ns * (1.0 - (p ** 2).sum())
                else:
                    nz = p[p > 0]
                    tot += -ns * (nz * np.log(nz)).sum()
        loss = tot / w.sum()
        if loss < best - 1e-12:
            best, best_b = loss, b
    return best, best_b


@pytest.mark.parametrize("crit,K", [("gini", 3), ("entropy", 4), ("mse", 0)])
def test_bf16_scores_follow_their_bins(crit, K):
    rng = np.random.default_rng(11)
    n, d, P, B = 150, 9, 4, 12
    X = rng.standard_normal((n, d)).astype(np.float32)
    lab = rng.integers(0, max(K, 2), n).astype(np.int32) if crit != "mse" else None
    yv = rng.standard_normal(n).astype(np.float32) if crit == "mse" else None
    w = rng.integers(1, 4, n).astype(np.uint32)
    p = bf16_params(criterion=crit, n_classes=K, n_particles=P, n_bins=B)
    pos = rng.uniform(-1, 1, (P, d))
    ev, bins, _ = O.eval_swarm(p, X, lab, yv, pos, wts=w, want_bins=True)
    for i in range(P):
        sb = O.score_bins(p, lab, yv, bins[i], wts=w)
        assert sb["bin"] == ev[i]["bin"] and sb["loss"] == ev[i]["loss"]
        bf, bb = edge_losses_from_bins(bins[i], lab if lab is not None else np.zeros(n, np.int64),
                                       yv.astype(np.float64) if yv is not None else None,
                                       w.astype(np.float64), B, max(K, 1), crit, 2)
        assert bb == ev[i]["bin"]
        assert abs(bf - ev[i]["loss"]) <= 1e-12 * max(1.0, abs(bf))


def rank_key(e, crit):
    """Sort key: invalid last, then lower loss (Gini: larger exact Q)."""
    if not e["valid"]:
        return (1, 0)
    if crit == "gini":
        return (0, -Fraction(int(e["q_num"]), int(e["q_den"])))
    return (0, e["loss"])


@pytest.mark.parametrize("crit,K", [("gini", 4), ("entropy", 3), ("mse", 0)])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_topk_merge_brute_force(crit, K, k):
    rng = np.random.default_rng(17 + k)
    n, d, P = 220, 13, 10
    X = rng.standard_normal((n, d)).astype(np.float32)
    lab = rng.integers(0, max(K, 2), n).astype(np.int32) if crit != "mse" else None
    yv = (X[:, 0] + 0.3 * rng.standard_normal(n)).astype(np.float32) if crit == "mse" else None
    pos = rng.uniform(-1, 1, (P, d))
    pos[4] = pos[2]  # an exact tie: the lower index must be taken first
    kw = dict(criterion=crit, n_classes=K, n_particles=P, n_bins=24)
    eb, _, _ = O.eval_swarm(bf16_params(topk=0, **kw), X, lab, yv, pos)
    em, _, _ = O.eval_swarm(O.make_params(precision=O.F32_MIRROR, min_leaf=2, **kw),
                            X, lab, yv, pos)
    merged, _, _ = O.eval_swarm(bf16_params(topk=k, **kw), X, lab, yv, pos)
    order = sorted(range(P), key=lambda i: (rank_key(eb[i], crit), i))
    chosen = set(order[:k])
    for i in range(P):
        want = em[i] if i in chosen else eb[i]
        assert merged[i]["loss"] == want["loss"] and merged[i]["bin"] == want["bin"], i


def test_topk_equal_P_reduces_to_mirror_search():
    """With every particle re-scored, the reduced-precision pass only orders
    particles, which nothing then uses: the search is the mirror search."""
    wl = W.gmm(900, 6, 3, seed=4)
    X, lab = wl.X, wl.labels
    for crit in ("gini", "entropy"):
        kw = dict(criterion=crit, n_classes=3, n_particles=12, n_iters=15, n_bins=32,
                  min_leaf=5, seed=21)
        m = O.node_split(O.make_params(precision=O.F32_MIRROR, **kw), X, lab, node_uid=9)
        b = O.node_split(O.make_params(precision=O.BF16_TOPK, topk=12, **kw), X, lab, node_uid=9)
        assert np.array_equal(m.trace_loss, b.trace_loss)
        assert np.array_equal(m.trace_particle, b.trace_particle)
        assert np.array_equal(m.gbest, b.gbest)
        assert m.split["bin"] == b.split["bin"]


@pytest.mark.parametrize("crit,K", [("gini", 3), ("mse", 0)])
@pytest.mark.parametrize("topk", [1, 4])
def test_bf16_gbest_score_is_the_float_score(crit, K, topk):
    """gbest is chosen among re-scored particles: its score must equal the
    float mirror score of the returned position, and the trace never rises."""
    wl = W.tanh_regression(1500, 12, seed=2) if crit == "mse" else W.gmm(1500, 12, 3, seed=2)
    X, lab, yv = wl.X, wl.labels, wl.y
    kw = dict(criterion=crit, n_classes=K, n_particles=16, n_iters=20, n_bins=32,
              min_leaf=5, seed=8)
    r = O.node_split(O.make_params(precision=O.BF16_TOPK, topk=topk, **kw), X, lab, yv,
                     node_uid=3)
    ev, _, _ = O.eval_swarm(O.make_params(precision=O.F32_MIRROR, **kw), X, lab, yv,
                            r.gbest[None, :])
    assert ev[0]["loss"] == r.split["loss"] and ev[0]["bin"] == r.split["bin"]
    assert np.all(np.diff(r.trace_loss) <= 0)


def test_bf16_search_quality_planted():
    """On a planted hyperplane the reduced-precision search must reach the
    same neighbourhood of loss as the float search."""
    wl = W.single_node(2000, 16, seed=7)
    X, lab = wl.X, wl.labels
    kw = dict(criterion="entropy", n_classes=2, n_particles=32, n_iters=50, n_bins=64,
              min_leaf=1, seed=1)
    m = O.node_split(O.make_params(precision=O.F32_MIRROR, **kw), X, lab)
    b = O.node_split(O.make_params(precision=O.BF16_TOPK, topk=8, **kw), X, lab)
    assert b.split["loss"] <= m.split["loss"] * 1.05 + 1e-3


def test_gbest_only_from_rescored_particles():
    """Features at 256 +- 0.4 all round to 256 in bfloat16, so the reduced
    projection sees only the two informative features and every bfloat16 score
    is optimistic. Were gbest allowed to take a bfloat16 score, it would take
    one of those; the returned score must be the float score of gB."""
    rng = np.random.default_rng(2)
    n, d = 600, 8
    lab = rng.integers(0, 2, n).astype(np.int32)
    X = np.empty((n, d), np.float32)
    X[:, :2] = 0.7 * lab[:, None] + rng.normal(0.0, 0.5, (n, 2))
    X[:, 2:] = 256.0 + rng.uniform(-0.4, 0.4, (n, d - 2))
    kw = dict(criterion="gini", n_classes=2, n_particles=16, n_iters=6, n_bins=32,
              min_leaf=5, seed=3)
    pos = np.random.default_rng(9).uniform(-1, 1, (16, d))
    eb, _, _ = O.eval_swarm(O.make_params(precision=O.BF16_TOPK, topk=0, **kw), X, lab, None, pos)
    em, _, _ = O.eval_swarm(O.make_params(precision=O.F32_MIRROR, **kw), X, lab, None, pos)
    assert sum(b["loss"] < m["loss"] for b, m in zip(eb, em)) >= 12
    r = O.node_split(O.make_params(precision=O.BF16_TOPK, topk=1, **kw), X, lab, node_uid=1)
    ev, _, _ = O.eval_swarm(O.make_params(precision=O.F32_MIRROR, **kw), X, lab, None,
                            r.gbest[None, :])
    assert ev[0]["q_num"] == r.split["q_num"] and ev[0]["q_den"] == r.split["q_den"]
