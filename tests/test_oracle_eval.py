"""Pins for the oracle's scoring of one projection (Eqs. 1, 3-4; Sec. IV).

The oracle bins z uniformly, histograms, prefix-scans the B-1 edges and takes
the criterion from the prefix counts. These tests check it against a brute
force that never histograms or scans: each edge's two child sets are formed
directly from the samples and scored with the textbook impurity formulas
(Gini 1 - sum p^2, entropy -sum p ln p, two-pass variance), plus closed forms
and invariants.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W


def edge_count_bins(z, zmin, zmax, B):
    """Bin index as the number of interior edges zmin + k (zmax-zmin)/B,
    k = 1..B-1, lying at or below z."""
    edges = zmin + (zmax - zmin) * np.arange(1, B) / B
    return np.searchsorted(edges, z, side="right"), edges


def textbook_loss(lab, yv, w, left, K, crit):
    n = w.sum()
    total = 0.0
    for side in (left, ~left):
        ws = w[side]
        ns = ws.sum()
        if crit == "mse":
            ybar = (ws * yv[side]).sum() / ns
            total += (ws * (yv[side] - ybar) ** 2).sum()
            continue
        p = np.bincount(lab[side], weights=ws, minlength=K) / ns
        if crit == "gini":
            imp = 1.0 - (p ** 2).sum()
        else:
            nz = p[p > 0]
            imp = -(nz * np.log(nz)).sum()
        total += ns * imp
    return total / n


def brute_force_best(bins, lab, yv, w, B, K, crit, min_leaf):
    best, best_b, losses = np.inf, -1, {}
    for b in range(1, B):
        left = bins < b
        nl, nr = w[left].sum(), w[~left].sum()
        if nl < min_leaf or nr < min_leaf:
            continue
        loss = textbook_loss(lab, yv, w, left, K, crit)
        losses[b] = loss
        if loss < best:
            best, best_b = loss, b
    return best, best_b, losses


CASES = [
    ("gini", 3, 16, 1), ("gini", 5, 7, 3), ("entropy", 2, 16, 1),
    ("entropy", 4, 32, 2), ("mse", 0, 16, 1), ("mse", 0, 9, 4),
]


@pytest.mark.parametrize("crit,K,B,min_leaf", CASES)
@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
@pytest.mark.parametrize("weighted", [False, True])
def test_binned_scan_matches_brute_force(crit, K, B, min_leaf, precision, weighted):
    rng = np.random.default_rng(hash((crit, K, B, precision, weighted)) & 0xFFFF)
    n, d, P = 150, 5, 6
    X = rng.standard_normal((n + 20, d)).astype(np.float32)
    idx = rng.choice(n + 20, n, replace=False).astype(np.int32)
    labels = rng.integers(0, max(K, 2), n + 20).astype(np.int32) if crit != "mse" else None
    y = rng.standard_normal(n + 20).astype(np.float32) if crit == "mse" else None
    wts = rng.integers(1, 4, n).astype(np.uint32) if weighted else None
    pos = rng.uniform(-1, 1, (P, d)).astype(np.float32).astype(np.float64)
    p = O.make_params(crit, K, P, 0, B, min_leaf=min_leaf, precision=precision)
    res, bins, z = O.eval_swarm(p, X, labels, y, pos, idx=idx, wts=wts,
                                want_bins=True, want_z=True)
    w = np.ones(n) if wts is None else wts.astype(np.float64)
    lab = labels[idx] if labels is not None else None
    yv = y[idx].astype(np.float64) if y is not None else None
    for i in range(P):
        # the projection is a^T x (Eq. 1)
        zt = X[idx].astype(np.float64) @ pos[i]
        # dot-product rounding bound: d * u * sum_j |x_j a_j|
        u = 2.0**-53 if precision == O.F64 else 2.0**-24
        scale = np.abs(X[idx]).astype(np.float64) @ np.abs(pos[i])
        assert np.all(np.abs(z[i] - zt) <= 2 * d * u * scale)
        r = res[i]
        assert r["zmin"] == z[i].min() and r["zmax"] == z[i].max()
        # each bin is the number of interior edges at or below z
        eb, edges = edge_count_bins(z[i], r["zmin"], r["zmax"], B)
        close = np.min(np.abs(z[i][:, None] - edges[None, :]), axis=1) <= 1e-5 * (r["zmax"] - r["zmin"])
        assert np.all((bins[i] == eb) | close)
        best, best_b, losses = brute_force_best(bins[i], lab, yv, w, B, K, crit, min_leaf)
        if not np.isfinite(best):
            assert r["valid"] == 0 and np.isinf(r["loss"])
            continue
        assert r["valid"] == 1
        assert r["loss"] == pytest.approx(best, rel=1e-10, abs=1e-12)
        # the chosen edge is a minimiser; among exact ties the smallest edge
        assert losses[r["bin"]] == pytest.approx(best, rel=1e-10, abs=1e-12)
        assert r["bin"] <= min(b for b, l in losses.items() if abs(l - best) <= 1e-10 * abs(best) + 1e-12)
        left = bins[i] < r["bin"]
        assert r["n_left"] == w[left].sum() and r["n_right"] == w[~left].sum()
        if crit == "gini":
            # loss = 1 - Q/n with Q the exact rational the oracle compares
            assert r["loss"] == pytest.approx(1.0 - r["q_num"] / r["q_den"] / w.sum(), rel=1e-12)


def test_closed_form_values():
    # Two classes, feature 0 separates them perfectly: loss 0 for every criterion.
    X = np.array([[0.0], [1.0], [2.0], [3.0], [10.0], [11.0], [12.0], [13.0]], np.float32)
    lab = np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32)
    for crit in ("gini", "entropy"):
        p = O.make_params(crit, 2, 1, 0, 4, min_leaf=1, precision=O.F64)
        r = O.eval_swarm(p, X, lab, None, np.ones((1, 1)))[0][0]
        assert r["loss"] == 0.0 and r["n_left"] == 4 and r["n_right"] == 4
    # Alternating labels on equally spaced points, 2 bins: each child holds a
    # 50/50 mix -> Gini 0.5, entropy ln 2.
    X = np.arange(8, dtype=np.float32)[:, None]
    lab = np.array([0, 1, 0, 1, 0, 1, 0, 1], np.int32)
    r = O.eval_swarm(O.make_params("gini", 2, 1, 0, 2, precision=O.F64), X, lab, None, np.ones((1, 1)))[0][0]
    assert r["loss"] == pytest.approx(0.5, abs=1e-15)
    r = O.eval_swarm(O.make_params("entropy", 2, 1, 0, 2, precision=O.F64), X, lab, None, np.ones((1, 1)))[0][0]
    assert r["loss"] == pytest.approx(np.log(2.0), abs=1e-15)
    # Regression: y = 0 on the left half, 1 on the right: MSE 0.
    y = np.array([0, 0, 0, 0, 1, 1, 1, 1], np.float32)
    r = O.eval_swarm(O.make_params("mse", 0, 1, 0, 2, precision=O.F64), X, None, y, np.ones((1, 1)))[0][0]
    assert r["loss"] == 0.0
    # Identical projections: no threshold exists.
    X = np.ones((10, 2), np.float32)
    r = O.eval_swarm(O.make_params("gini", 2, 1, 0, 8), X, np.arange(10, dtype=np.int32) % 2, None,
                     np.array([[0.3, -0.2]]))[0][0]
    assert r["valid"] == 0 and np.isinf(r["loss"])
    # min_leaf larger than half the node: no admissible edge.
    X = np.arange(10, dtype=np.float32)[:, None]
    r = O.eval_swarm(O.make_params("gini", 2, 1, 0, 8, min_leaf=6), X, np.arange(10, dtype=np.int32) % 2,
                     None, np.ones((1, 1)))[0][0]
    assert r["valid"] == 0


@pytest.mark.parametrize("crit", ["gini", "entropy"])
def test_axis_aligned_equals_cart(crit):
    """A particle fixed to e_j scores feature j alone; with integer feature
    values 0..B-1 every bin holds one value, so the binned scan sees every
    threshold and must equal CART's best split on that feature."""
    tree = pytest.importorskip("sklearn.tree")
    rng = np.random.default_rng(5)
    n, d, B, K = 400, 3, 32, 3
    X = rng.integers(0, B, (n, d)).astype(np.float32)
    X[0, :] = 0
    X[1, :] = B - 1
    lab = ((X[:, 1] > 11) + (X[:, 1] > 20) + (rng.random(n) < 0.2)).astype(np.int32) % K
    p = O.make_params(crit, K, 1, 0, B, min_leaf=1, precision=O.F64)
    for j in range(d):
        e = np.zeros((1, d)); e[0, j] = 1.0
        r = O.eval_swarm(p, X, lab, None, e)[0][0]
        clf = tree.DecisionTreeClassifier(max_depth=1, criterion=crit if crit == "gini" else "entropy",
                                          random_state=0).fit(X[:, j:j + 1], lab)
        t = clf.tree_
        if t.node_count == 1:
            continue
        nl, nr = t.weighted_n_node_samples[1], t.weighted_n_node_samples[2]
        cart = (nl * t.impurity[1] + nr * t.impurity[2]) / n
        if crit == "entropy":
            cart *= np.log(2.0)  # sklearn's entropy is in bits, the oracle's in nats
        assert r["loss"] == pytest.approx(cart, rel=1e-9, abs=1e-12)
        # CART puts x <= thr on the left; the oracle puts bin < b on the left
        assert (r["n_left"], r["n_right"]) == (nl, nr) or r["loss"] == pytest.approx(cart, abs=1e-12)


@pytest.mark.parametrize("crit", ["gini", "entropy", "mse"])
def test_children_never_worse_than_parent(crit):
    """Concavity of Gini / entropy and the variance decomposition: the best
    weighted child impurity never exceeds the parent's."""
    wl = W.gmm(600, 6, 4, seed=3) if crit != "mse" else W.tanh_regression(600, 6, seed=3)
    rng = np.random.default_rng(0)
    pos = rng.uniform(-1, 1, (20, 6))
    p = O.make_params(crit, 4, 20, 0, 32, precision=O.F64)
    res, bins, _ = O.eval_swarm(p, wl.X, wl.labels, wl.y, pos, want_bins=True)
    if crit == "mse":
        yv = wl.y.astype(np.float64)
        parent = yv.var()
    else:
        q = np.bincount(wl.labels, minlength=4) / wl.n
        parent = 1 - (q ** 2).sum() if crit == "gini" else -(q[q > 0] * np.log(q[q > 0])).sum()
    for i, r in enumerate(res):
        assert r["loss"] <= parent + 1e-12
        if crit == "mse":
            # SSE_parent = SSE_L + SSE_R + nL nR / n (ybar_L - ybar_R)^2
            left = bins[i] < r["bin"]
            nl, nr = left.sum(), (~left).sum()
            gap = yv[left].mean() - yv[~left].mean()
            assert wl.n * parent == pytest.approx(wl.n * r["loss"] + nl * nr / wl.n * gap ** 2, rel=1e-12)


@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
def test_scale_and_permutation_invariance(precision):
    wl = W.gmm(500, 8, 3, seed=11)
    rng = np.random.default_rng(1)
    pos = rng.uniform(-1, 1, (8, 8)).astype(np.float32).astype(np.float64)
    p = O.make_params("gini", 3, 8, 0, 16, precision=precision)
    base, bins, _ = O.eval_swarm(p, wl.X, wl.labels, None, pos, want_bins=True)
    # scaling by 2 is exact in binary: identical bins and losses
    r2, bins2, _ = O.eval_swarm(p, wl.X, wl.labels, None, 2.0 * pos, want_bins=True)
    assert np.array_equal(bins, bins2)
    assert [r["loss"] for r in base] == [r["loss"] for r in r2]
    # shuffling the node's sample order changes nothing
    perm = rng.permutation(wl.n).astype(np.int32)
    r3, bins3, _ = O.eval_swarm(p, wl.X, wl.labels, None, pos, idx=perm, want_bins=True)
    assert np.array_equal(bins3[:, np.argsort(perm)], bins)
    assert [(r["loss"], r["bin"]) for r in base] == [(r["loss"], r["bin"]) for r in r3]


def test_mirror_agrees_with_f64():
    wl = W.gmm(3000, 16, 5, seed=2)
    rng = np.random.default_rng(2)
    pos = rng.uniform(-1, 1, (16, 16)).astype(np.float32).astype(np.float64)
    a = O.eval_swarm(O.make_params("gini", 5, 16, 0, 64, precision=O.F64), wl.X, wl.labels, None, pos,
                     want_bins=True, want_z=True)
    b = O.eval_swarm(O.make_params("gini", 5, 16, 0, 64, precision=O.F32_MIRROR), wl.X, wl.labels, None,
                     pos, want_bins=True, want_z=True)
    for i in range(16):
        za, zb = a[2][i], b[2][i]
        scale = np.abs(wl.X).astype(np.float64) @ np.abs(pos[i])
        assert np.all(np.abs(za - zb) <= 16 * 2.0**-24 * scale)
        mism = a[1][i] != b[1][i]
        assert mism.mean() < 1e-3
        assert a[0][i]["loss"] == pytest.approx(b[0][i]["loss"], rel=1e-2)
