"""Oracle parity at the shapes of the bagged-forest and learned-proposal
workloads (the full-size runs themselves are too large for the oracle).

* Bagged forest of the forest workload's shape: 48 particles (the swarm
  width whose tiles both projection paths use), bootstrap multiplicities,
  d = 32, K = 5 Gaussian-mixture classes, n = 20,000, depth 8, 128 bins,
  Gini; 30 iterations instead of 60 to bound the oracle's time. Every tree
  equals the oracle's tree of the same id node by node (kind, direction,
  range, bin, child counts, weight, loss, leaf class), with the folded
  projection (the default) and with the separate projection kernels at
  forced 48-particle tiles.
* Seeded BF16 search at the proposal workload's widths: d = 256, K = 20,
  P = 64, top-8 FP32 re-scoring, from the learned start the search's own
  kernels give (slm_seeded_start). At d = 256 no start keeps the bfloat16
  sums exact (the oracle flags its first evaluation), so the exact facts are
  checked instead: the bins of the start follow the oracle's z up to the
  accumulation bound and the scores follow from the bins; the 8 best
  particles carry the oracle's FP32 mirror scores bit for bit; the search
  with T = 0 returns the best of them (its start is that start); and every
  gB of the full search is an exact FP32 score, never increasing.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def _same_tree(g, r):
    assert np.array_equal(g["kind"], r.kind)
    inner = r.kind == 1
    present = r.kind >= 0
    assert np.array_equal(g["dir"][inner].astype(np.float64), r.dir[inner])
    assert np.array_equal(g["zmin"][inner], r.zmin[inner].astype(np.float32))
    assert np.array_equal(g["inv_w"][inner], r.inv_w[inner].astype(np.float32))
    assert np.array_equal(g["bin"][inner], r.bin[inner])
    assert np.array_equal(g["n_left"][inner], r.n_left[inner].astype(np.int64))
    assert np.array_equal(g["n_right"][inner], r.n_right[inner].astype(np.int64))
    assert np.array_equal(g["loss"][inner], r.loss[inner])
    assert np.array_equal(g["weight"][present], r.weight[present].astype(np.int64))
    assert np.array_equal(g["leaf_class"][present], r.leaf_class[present])
    return int(inner.sum())


def test_forest_of_the_forest_workload_shape_matches_oracle_trees():
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(20_000, 32, 5, seed=41)
    # 10 % of the labels flipped: deep trees instead of four clean splits
    rng = np.random.default_rng(41)
    flip = rng.random(wl.n) < 0.1
    labels = np.where(flip, rng.integers(0, 5, wl.n), wl.labels).astype(np.int32)
    n_trees, T = 3, 30
    gp = gpu_params(S, "gini", 5, 48, T, 128, min_leaf=20, max_depth=8, seed=6,
                    n_trees=n_trees, bootstrap=True)
    op = oracle_params(O, "gini", 5, 48, T, 128, min_leaf=20, max_depth=8, seed=6)
    ref = [O.train_tree(op, wl.X, labels, tree_id=t, bootstrap=True) for t in range(n_trees)]
    ctx = context()
    try:
        for fused in (True, False):
            ctx.set_fused_step(fused, always=True)
            if not fused:
                ctx.force_tiles(48, 2, False)
            f = ctx.train_tree(gp, wl.X, labels=labels)
            splits = [_same_tree(f.export(t), ref[t]) for t in range(n_trees)]
            assert min(splits) >= 16  # deep trees, not stumps
            f.free()
            ctx.force_tiles(0)
    finally:
        ctx.set_fused_step(True)
        ctx.close()


def test_seeded_bf16_search_at_the_proposal_workload_widths():
    from paper_2208_07023_gb300 import binding as S
    from tests.test_gpu_bf16 import accumulation_bound, check_bins, check_score, rank_key
    d, K, P, T, B, k = 256, 20, 64, 15, 128, 8
    wl = W.gmm(4000, d, K, seed=43)
    X, lab = wl.X, wl.labels
    ctx = context()
    prop = ctx.proposal(seed=11)
    ctx.use_proposal(prop)
    try:
        gp = S.make_params("gini", K, n_particles=P, n_iters=T, n_bins=B, min_leaf=2, seed=7,
                           proj=S.SLM_PROJ_BF16_TOPK, topk=k, seeded=True)
        x0 = ctx.seeded_start(gp, X, labels=lab, node_uid=11)
        assert x0.shape == (P, d) and np.isfinite(x0).all()
        assert np.array_equal(x0, ctx.seeded_start(gp, X, labels=lab, node_uid=11))
        u = O.swarm_uniforms(7, 11, 0, P, d, 1)
        assert not np.array_equal(x0, (2.0 * u - 1.0).astype(np.float32))
        # the bfloat16 pass over the start: bins and scores
        ge = S.make_params("gini", K, n_particles=P, n_iters=0, n_bins=B, min_leaf=2,
                           proj=S.SLM_PROJ_BF16_TOPK, topk=0)
        red, bins = ctx.evaluate_swarm(ge, X, x0, labels=lab, want_bins=True)
        op = O.make_params("gini", K, P, 0, B, min_leaf=2, precision=O.BF16_TOPK, topk=0)
        _, _, z = O.eval_swarm(op, X, lab, None, x0.astype(np.float64), want_z=True)
        bound = accumulation_bound(X, None, x0)
        moved = sum(check_bins(red[i], bins[i], z[i], bound[i], B) for i in range(P))
        assert moved <= max(3, bins.size // 2000)
        sb = [O.score_bins(op, lab, None, bins[i]) for i in range(P)]
        for i in range(P):
            check_score(red[i], sb[i], "gini")
        # the k best carry their FP32 mirror scores bit for bit
        ge.topk = k
        merged, _ = ctx.evaluate_swarm(ge, X, x0, labels=lab)
        chosen = sorted(sorted(range(P), key=lambda i: (rank_key(sb[i], "gini"), i))[:k])
        mirror, _, _ = O.eval_swarm(oracle_params(O, "gini", K, k, 0, B, min_leaf=2), X, lab,
                                    None, x0[chosen].astype(np.float64))
        for q, i in enumerate(chosen):
            check_score(merged[i], mirror[q], "gini")
        # a search with no iterations keeps the best re-scored particle
        best = min(chosen, key=lambda i: (rank_key(merged[i], "gini"), i))
        g0 = ctx.node_split(S.make_params("gini", K, n_particles=P, n_iters=0, n_bins=B,
                                          min_leaf=2, seed=7, proj=S.SLM_PROJ_BF16_TOPK,
                                          topk=k, seeded=True),
                            X, labels=lab, node_uid=11)
        assert g0["particle"] == best
        assert np.array_equal(g0["gbest"], x0[best])
        assert (g0["q_num"], g0["q_den"], g0["bin"]) == \
            (merged[best]["q_num"], merged[best]["q_den"], merged[best]["bin"])
        # the full search: every gB an exact FP32 score, never worse
        g = ctx.node_split(gp, X, labels=lab, node_uid=11, want_trace=True)
        assert g["trace"][0] == g0["loss"]
        assert np.all(np.diff(g["trace"]) <= 0)
        m = O.eval_swarm(oracle_params(O, "gini", K, 1, 0, B, min_leaf=2), X, lab, None,
                         g["gbest"].astype(np.float64)[None, :])[0][0]
        assert (m["bin"], m["q_num"], m["q_den"]) == (g["bin"], g["q_num"], g["q_den"])
    finally:
        ctx.use_proposal(None)
        prop.free()
        ctx.close()
