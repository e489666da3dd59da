"""GPU parity of the reduced-precision search (SLM_PROJ_BF16_TOPK).

The bfloat16 pass runs on the tensor cores, whose FP32 accumulation order is
not the oracle's; the oracle forms the bfloat16 dot product exactly and
rounds once. So:
* per evaluation, the GPU's range and bins may differ from the oracle's only
  for samples within the accumulation error bound of a bin edge (bound:
  (ceil(d/16) + 1) 2^-22 sum_j |x~_j a~_j|), and the scores must follow
  exactly from the GPU's own bins (oracle histogram + scan of those bins);
* the top-k merge is exact: the k best by that score (ties to the lower
  index) carry the oracle's FP32 mirror score bit for bit, the others the
  bfloat16 score of their bins;
* whole searches agree with the oracle's BF16_TOPK search up to the first
  iteration the oracle flags (a sample whose bfloat16 product is not exact in
  float lying near an edge, or a near-tie); small-integer features make the
  products exact, so the comparison runs for several iterations;
* every split of a tree is an FP32 score: the oracle's mirror re-score of
  the returned direction on the node's samples matches it exactly.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def bf16_gpu_params(S, crit, K, P, T, B, topk, min_leaf=2, seed=1, max_depth=8):
    return S.make_params(crit, K, n_particles=P, n_iters=T, n_bins=B, min_leaf=min_leaf,
                         seed=seed, max_depth=max_depth, proj=S.SLM_PROJ_BF16_TOPK, topk=topk)


def node_inputs(crit, n, d, K, seed, n_idx=None, weighted=False):
    rng = np.random.default_rng(seed)
    wl = W.tanh_regression(n, d, seed=seed) if crit == "mse" else W.gmm(n, d, K, seed=seed)
    idx = rng.choice(n, n_idx, replace=False).astype(np.int32) if n_idx else None
    m = n if idx is None else n_idx
    wts = rng.integers(1, 4, m).astype(np.uint32) if weighted else None
    return wl, idx, wts


def accumulation_bound(X, idx, pos):
    """Per (particle, entry) bound on |GPU z - correctly rounded z|."""
    rows = X if idx is None else X[idx]
    xb = O.bf16_round(rows).astype(np.float64)
    ab = O.bf16_round(pos.astype(np.float32)).astype(np.float64)
    sabs = np.abs(ab) @ np.abs(xb).T
    d = X.shape[1]
    return ((d + 15) // 16 + 1) * 2.0 ** -22 * sabs


def check_bins(g, gbins, z, bound, B):
    """GPU bins against the oracle's z binned with the GPU's range."""
    zmin, inv_w = np.float32(g["zmin"]), np.float32(g["inv_w"])
    pos = ((z.astype(np.float32) - zmin).astype(np.float32) * inv_w).astype(np.float32)
    rb = np.clip(np.floor(pos), 0, B - 1).astype(np.int64)
    mism = rb != gbins
    if mism.any():
        k = np.round(pos[mism].astype(np.float64))
        margin = bound[mism] * float(inv_w) + 2.0 ** -20 * B
        assert np.all(np.abs(pos[mism] - k) <= margin), "a bin differs away from an edge"
    return int(mism.sum())


def check_score(g, r, crit):
    assert g["valid"] == r["valid"]
    if not r["valid"]:
        return
    assert (g["bin"], g["n_left"], g["n_right"]) == (r["bin"], r["n_left"], r["n_right"])
    if crit == "gini":
        assert (g["q_num"], g["q_den"], g["loss"]) == (r["q_num"], r["q_den"], r["loss"])
    elif crit == "entropy":
        assert g["loss"] == pytest.approx(r["loss"], rel=1e-12)
    else:
        assert g["loss"] == pytest.approx(r["loss"], rel=1e-9)


BF16_CASES = [
    # crit, K, B, d, n, n_idx, P, weighted
    ("gini", 10, 128, 64, 3000, 700, 64, False),
    ("gini", 5, 64, 16, 5000, None, 16, True),        # dp = d = 16
    ("entropy", 4, 32, 37, 6000, 4099, 20, True),     # dp = 48, ragged tail, P' = 32
    ("mse", 0, 256, 128, 4000, 2500, 64, False),      # the regression-tree shape
    ("mse", 0, 100, 200, 3000, None, 33, True),       # two K chunks (128 + 80)
    ("gini", 3, 16, 3, 1000, None, 100, False),       # N = 112 columns
]


@pytest.mark.parametrize("crit,K,B,d,n,n_idx,P,weighted", BF16_CASES)
def test_bf16_scores_follow_bins(ctx, crit, K, B, d, n, n_idx, P, weighted):
    from paper_2208_07023_gb300 import binding as S
    wl, idx, wts = node_inputs(crit, n, d, K, seed=B + d, n_idx=n_idx, weighted=weighted)
    pos = np.random.default_rng(8).uniform(-1, 1, (P, d)).astype(np.float32)
    gp = bf16_gpu_params(S, crit, K, P, 0, B, topk=0, min_leaf=3)
    res, bins = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y, sample_idx=idx,
                                   weights=wts, want_bins=True)
    op = O.make_params(crit, K, P, 0, B, min_leaf=3, precision=O.BF16_TOPK, topk=0)
    ref, _, z = O.eval_swarm(op, wl.X, wl.labels, wl.y, pos.astype(np.float64), idx=idx,
                             wts=wts, want_z=True)
    bound = accumulation_bound(wl.X, idx, pos)
    total = 0
    for i, (g, r) in enumerate(zip(res, ref)):
        assert g["valid"] == r["valid"] or not np.isfinite(g["loss"])
        assert abs(g["zmin"] - r["zmin"]) <= bound[i].max() + 1e-30
        total += check_bins(g, bins[i], z[i], bound[i], B)
        sb = O.score_bins(op, wl.labels, wl.y, bins[i], idx=idx, wts=wts)
        check_score(g, sb, crit)
    assert total <= max(3, bins.size // 2000)


def rank_key(e, crit):
    if not e["valid"]:
        return (1, 0)
    if crit == "gini":
        return (0, -Fraction(int(e["q_num"]), int(e["q_den"])))
    return (0, e["loss"])


@pytest.mark.parametrize("crit,K,B,d,n,n_idx,P,weighted", BF16_CASES)
@pytest.mark.parametrize("k", [1, 8])
def test_bf16_topk_merge_exact(ctx, crit, K, B, d, n, n_idx, P, weighted, k):
    from paper_2208_07023_gb300 import binding as S
    wl, idx, wts = node_inputs(crit, n, d, K, seed=B + d, n_idx=n_idx, weighted=weighted)
    rng = np.random.default_rng(9)
    pos = rng.uniform(-1, 1, (P, d)).astype(np.float32)
    pos[P - 1] = pos[0]  # an exact tie: the lower index ranks first
    gp = bf16_gpu_params(S, crit, K, P, 0, B, topk=k, min_leaf=3)
    res, bins = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y, sample_idx=idx,
                                   weights=wts, want_bins=True)
    op = O.make_params(crit, K, P, 0, B, min_leaf=3, precision=O.BF16_TOPK, topk=0)
    reduced = [O.score_bins(op, wl.labels, wl.y, bins[i], idx=idx, wts=wts) for i in range(P)]
    order = sorted(range(P), key=lambda i: (rank_key(reduced[i], crit), i))
    chosen = sorted(order[:k])
    mirror, _, _ = O.eval_swarm(oracle_params(O, crit, K, len(chosen), 0, B, min_leaf=3),
                                wl.X, wl.labels, wl.y, pos[chosen].astype(np.float64),
                                idx=idx, wts=wts)
    for q, i in enumerate(chosen):
        g, r = res[i], mirror[q]
        assert g["zmin"] == np.float32(r["zmin"]) and g["inv_w"] == np.float32(r["inv_w"])
        check_score(g, r, crit)
    for i in set(range(P)) - set(chosen):
        check_score(res[i], reduced[i], crit)


def integer_node(n, d, K, seed):
    """Gaussian-mixture classes on small-integer features: every bfloat16
    product is exact and, for most positions, so is every partial sum."""
    wl = W.gmm(n, d, K, seed=seed)
    return np.clip(np.round(wl.X), -8, 8).astype(np.float32), wl.labels


@pytest.mark.parametrize("crit,K,B,d,n,P,T,k", [
    ("gini", 3, 64, 16, 3000, 32, 30, 8),
    ("gini", 6, 128, 40, 5000, 48, 20, 4),
    ("entropy", 3, 64, 16, 2500, 32, 30, 8),
])
def test_bf16_node_split_trajectory(ctx, crit, K, B, d, n, P, T, k):
    from paper_2208_07023_gb300 import binding as S
    X, lab = integer_node(n, d, K, seed=d + P)
    gp = bf16_gpu_params(S, crit, K, P, T, B, topk=k, seed=7)
    g = ctx.node_split(gp, X, labels=lab, node_uid=11, want_trace=True)
    op = O.make_params(crit, K, P, T, B, min_leaf=2, seed=7, precision=O.BF16_TOPK, topk=k)
    r = O.node_split(op, X, lab, node_uid=11)
    stop = r.split["first_near_tie"]
    upto = T + 1 if stop < 0 else stop
    assert np.array_equal(g["trace"][:upto], r.trace_loss[:upto])
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
        assert (g["particle"], g["iter_of_best"], g["bin"]) == \
            (r.split["particle"], r.split["iter_of_best"], r.split["bin"])
    # gB's score is its FP32 score, whatever the path
    m = O.eval_swarm(oracle_params(O, crit, K, 1, 0, B, min_leaf=2), X, lab, None,
                     g["gbest"].astype(np.float64)[None, :])[0][0]
    assert m["bin"] == g["bin"] and m["loss"] == pytest.approx(g["loss"], rel=1e-12)
    assert np.all(np.diff(g["trace"]) <= 0)


def node_members(leaf, h):
    out = np.zeros(leaf.shape[0], bool)
    node = leaf.copy()
    while True:
        out |= node == h
        if (node <= h).all():
            break
        node = np.where(node > h, (node - 1) // 2, node)
    return np.nonzero(out)[0].astype(np.int32)


@pytest.mark.parametrize("crit,K", [("mse", 0), ("gini", 4)])
def test_bf16_tree_splits_are_fp32_scores(ctx, crit, K):
    from paper_2208_07023_gb300 import binding as S
    n, d, B, P, T, depth = 6000, 24, 64, 16, 10, 4
    wl = W.tanh_regression(n, d, seed=3) if crit == "mse" else W.gmm(n, d, K, seed=3)
    gp = bf16_gpu_params(S, crit, K, P, T, B, topk=4, min_leaf=20, max_depth=depth, seed=5)
    f = ctx.train_tree(gp, wl.X, labels=wl.labels, y=wl.y)
    try:
        g = f.export(0)
        _, _, leaf = ctx.predict(f, wl.X, want_leaf=True)
    finally:
        f.free()
    leaf = leaf[:, 0]
    inner = np.nonzero(g["kind"] == 1)[0]
    assert len(inner) >= 3
    op = oracle_params(O, crit, K, 1, 0, B, min_leaf=20)
    for h in inner:
        idx = node_members(leaf, h)
        e = O.eval_swarm(op, wl.X, wl.labels, wl.y, g["dir"][h].astype(np.float64)[None, :],
                         idx=idx)[0][0]
        assert (e["bin"], e["n_left"], e["n_right"]) == (g["bin"][h], g["n_left"][h],
                                                         g["n_right"][h])
        assert np.float32(e["zmin"]) == g["zmin"][h] and np.float32(e["inv_w"]) == g["inv_w"][h]
        assert e["loss"] == pytest.approx(g["loss"][h], rel=1e-9)
    for h in np.nonzero(g["kind"] == 0)[0]:
        assert (leaf == h).sum() == g["weight"][h]


def test_bf16_rejects_bad_topk_and_sizes(ctx):
    from paper_2208_07023_gb300 import binding as S
    X = np.random.default_rng(1).standard_normal((100, 8)).astype(np.float32)
    lab = (np.arange(100) % 2).astype(np.int32)
    for topk in (0, 17):
        with pytest.raises(S.SlmError) as e:
            ctx.node_split(bf16_gpu_params(S, "gini", 2, 16, 3, 16, topk=topk), X, labels=lab)
        assert e.value.status == S.SLM_EINVAL
    Xw = np.random.default_rng(1).standard_normal((100, 600)).astype(np.float32)
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(bf16_gpu_params(S, "gini", 2, 256, 3, 16, topk=8), Xw, labels=lab)
    assert e.value.status == S.SLM_EUNSUPPORTED
