"""Graph-captured searches and projection tile shapes change nothing the
method computes.

* graphs on / off: identical node searches (trajectory trace, gB, split) and
  identical trees of a bagged forest (every exported array);
* every projection tile shape (8 / 16 / 24 / 32 / 48 particles per group that
  divides the padded swarm, 1 or 2 CTAs per SM, rows from the level copy or
  gathered from the forest's base rows), forced, and the autotuned one:
  identical trees;
* the tuner records shapes and a valid choice; graphs are launched, and
  reused (updated) across the levels and trees of a run;
* invalid shapes are rejected.
"""
import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    c.set_node_search(False)  # the per-iteration kernels these tests vary (the default)
    yield c
    c.close()


def forest_arrays(ctx, p, wl):
    f = ctx.train_tree(p, wl.X, labels=wl.labels)
    out = [f.export(t) for t in range(f.info()["n_trees"])]
    f.free()
    return out


def same_forest(a, b):
    assert len(a) == len(b)
    for ga, gb in zip(a, b):
        assert ga.keys() == gb.keys()
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), k


def test_graphs_do_not_change_a_search(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(3000, 24, 4, seed=5)
    p = gpu_params(S, "gini", 4, 40, 30, 64, min_leaf=5, seed=3)
    res = []
    for on in (False, True):
        ctx.set_graphs(on)
        res.append(ctx.node_split(p, wl.X, labels=wl.labels, node_uid=7, want_trace=True))
    ctx.set_graphs(True)
    a, b = res
    assert np.array_equal(a["trace"], b["trace"])
    assert np.array_equal(a["gbest"].view(np.uint32), b["gbest"].view(np.uint32))
    assert (a["bin"], a["n_left"], a["loss"]) == (b["bin"], b["n_left"], b["loss"])


def test_graphs_do_not_change_a_forest(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(4000, 16, 5, seed=6)
    p = gpu_params(S, "gini", 5, 48, 12, 64, min_leaf=10, seed=2, max_depth=5, n_trees=6,
                   bootstrap=True)
    ctx.set_graphs(False)
    a = forest_arrays(ctx, p, wl)
    ctx.set_graphs(True)
    g0 = ctx.graph_stats()
    b = forest_arrays(ctx, p, wl)
    g1 = ctx.graph_stats()
    c = forest_arrays(ctx, p, wl)
    g2 = ctx.graph_stats()
    same_forest(a, b)
    same_forest(a, c)
    # one graph launch per searched level; the second forest repeats the
    # first one's launch shapes, so its graphs are kept ones, launched again
    # (same buffers) or updated in place
    assert g1["launches"] - g0["launches"] >= 2
    assert g2["launches"] - g1["launches"] == g1["launches"] - g0["launches"]
    kept = (g2["reuses"] - g1["reuses"]) + (g2["updates"] - g1["updates"])
    assert kept == g2["launches"] - g1["launches"]
    assert g2["instantiations"] == g1["instantiations"]


def test_repeated_search_relaunches_its_graph(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(2000, 16, 3, seed=9)
    p = gpu_params(S, "entropy", 3, 32, 20, 64, min_leaf=5, seed=8)
    ctx.set_graphs(True)
    a = ctx.node_split(p, wl.X, labels=wl.labels, node_uid=3, want_trace=True)
    g0 = ctx.graph_stats()
    b = ctx.node_split(p, wl.X, labels=wl.labels, node_uid=3, want_trace=True)
    g1 = ctx.graph_stats()
    assert np.array_equal(a["trace"], b["trace"])
    assert g1["launches"] == g0["launches"] + 1
    assert g1["reuses"] + g1["updates"] == g0["reuses"] + g0["updates"] + 1
    # another seed: same launches, other arguments
    p2 = gpu_params(S, "entropy", 3, 32, 20, 64, min_leaf=5, seed=9)
    ctx.node_split(p2, wl.X, labels=wl.labels, node_uid=3)
    g2 = ctx.graph_stats()
    assert g2["instantiations"] == g1["instantiations"]


@pytest.mark.parametrize("crit,K", [("mse", 0), ("gini", 4)])
def test_graphs_do_not_change_a_bf16_tree(ctx, crit, K):
    """Levels of one tree share the launch sequence but not grid or cluster
    shapes: each shape gets its own executable graph."""
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(6000, 24, seed=3) if crit == "mse" else W.gmm(6000, 24, K, seed=3)
    p = S.make_params(crit, K, n_particles=16, n_iters=10, n_bins=64, min_leaf=20,
                      max_depth=4, seed=5, proj=S.SLM_PROJ_BF16_TOPK, topk=4)
    out = []
    for on in (False, True, True):
        ctx.set_graphs(on)
        f = ctx.train_tree(p, wl.X, labels=wl.labels, y=wl.y)
        out.append([f.export(0)])
        f.free()
    same_forest(out[0], out[1])
    same_forest(out[0], out[2])


@pytest.mark.parametrize("P", [48, 64, 20])
def test_every_tile_shape_gives_the_same_forest(ctx, P):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(5000, 32, 5, seed=P)
    p = gpu_params(S, "gini", 5, P, 8, 128, min_leaf=10, seed=4, max_depth=4, n_trees=3,
                   bootstrap=True)
    ctx.set_tuning(False)
    ctx.set_fused_step(False)  # the tile shapes of the separate projection kernel
    ref = forest_arrays(ctx, p, wl)
    Pp = (P + 15) // 16 * 16
    for pg in (8, 16, 24, 32, 48):
        if Pp % pg:
            continue
        for cps in (1, 2):
            for gather in (False, True):
                ctx.force_tiles(pg, cps, gather)
                same_forest(ref, forest_arrays(ctx, p, wl))
                assert ctx.tuning_stats()["last_pg"] == pg
    ctx.force_tiles(0)
    ctx.set_tuning(True)
    n0 = ctx.tuning_stats()["shapes"]
    same_forest(ref, forest_arrays(ctx, p, wl))
    st = ctx.tuning_stats()
    assert st["shapes"] > n0
    assert st["last_pg"] in (8, 16, 24, 32, 48) and Pp % st["last_pg"] == 0
    assert st["last_ctas_per_sm"] in (1, 2)
    ctx.set_fused_step(True)


@pytest.mark.parametrize("crit,bootstrap", [("gini", True), ("entropy", False),
                                             ("gini", False), ("entropy", True)])
def test_small_node_kernel_gives_the_same_forest(ctx, crit, bootstrap):
    """Warp-per-particle histograms for small nodes against the cluster
    kernel for every node, and every node small."""
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(6000, 12, 6, seed=21)
    p = gpu_params(S, crit, 6, 24, 10, 64, min_leaf=8, seed=6, max_depth=6, n_trees=4,
                   bootstrap=bootstrap)
    out = []
    for bound in (0, 4096, 1 << 30):
        ctx.set_small_nodes(bound, 0)
        out.append(forest_arrays(ctx, p, wl))
    ctx.set_small_nodes()
    same_forest(out[0], out[1])
    same_forest(out[0], out[2])


def test_small_node_kernel_gives_the_same_search(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(3000, 20, 10, seed=22)
    for crit in ("gini", "entropy"):
        p = gpu_params(S, crit, 10, 64, 25, 128, min_leaf=3, seed=7)
        res = []
        for bound in (0, 1 << 30):
            ctx.set_small_nodes(bound, 0)
            res.append(ctx.node_split(p, wl.X, labels=wl.labels, node_uid=5, want_trace=True))
        ctx.set_small_nodes()
        assert np.array_equal(res[0]["trace"], res[1]["trace"])
        assert np.array_equal(res[0]["gbest"].view(np.uint32), res[1]["gbest"].view(np.uint32))
        assert (res[0]["bin"], res[0]["n_left"]) == (res[1]["bin"], res[1]["n_left"])


def test_invalid_tiles_are_rejected(ctx):
    from paper_2208_07023_gb300 import binding as S
    for pg, cps in ((12, 1), (16, 3), (64, 2)):
        with pytest.raises(S.SlmError) as e:
            ctx.force_tiles(pg, cps)
        assert e.value.status == 1
    assert S.lib().slm_force_tiles(ctx.handle, 16, 2, 2) == 1
    # 32 does not divide 48 (P = 48 pads to 48)
    ctx.force_tiles(32, 2)
    wl = W.gmm(1000, 8, 3, seed=1)
    p = gpu_params(S, "gini", 3, 48, 2, 32, min_leaf=5)
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(p, wl.X, labels=wl.labels)
    assert e.value.status == 1
    ctx.force_tiles(0)
    ctx.node_split(p, wl.X, labels=wl.labels)
    assert S.lib().slm_set_graphs(ctx.handle, 2) == 1
    assert S.lib().slm_set_small_nodes(ctx.handle, -1, 0) == 1
    assert S.lib().slm_set_small_nodes(ctx.handle, 16, -2) == 1
    assert S.lib().slm_set_tuning(ctx.handle, -1) == 1


@pytest.mark.parametrize("crit,bootstrap", [("gini", True), ("entropy", False),
                                             ("gini", False), ("entropy", True)])
def test_persistent_node_search_gives_the_same_forest(ctx, crit, bootstrap):
    """Whole searches in one launch (nodes resident in shared memory) against
    the per-iteration kernels: identical trees, also when only the deeper
    levels fit."""
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(4000, 12, 6, seed=31)
    p = gpu_params(S, crit, 6, 40, 12, 64, min_leaf=8, seed=3, max_depth=6, n_trees=3,
                   bootstrap=bootstrap)
    out = []
    for on in (False, True):
        ctx.set_node_search(on)
        out.append(forest_arrays(ctx, p, wl))
        if on:
            assert ctx.last_node_search() >= 1
    ctx.set_node_search(False)
    same_forest(out[0], out[1])
    # rows too large for shared memory at the top levels, resident below
    wl2 = W.gmm(20000, 48, 4, seed=32)
    p2 = gpu_params(S, crit, 4, 32, 8, 128, min_leaf=20, seed=4, max_depth=7)
    out2 = []
    for on in (False, True):
        ctx.set_node_search(on)
        out2.append(forest_arrays(ctx, p2, wl2))
    ctx.set_node_search(False)
    same_forest(out2[0], out2[1])


@pytest.mark.parametrize("P,n,d", [(32, 2000, 16), (64, 700, 64), (20, 150, 5), (48, 3000, 8)])
def test_persistent_node_search_gives_the_same_trajectory(ctx, P, n, d):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(n, d, 4, seed=P + d)
    for crit in ("gini", "entropy"):
        p = gpu_params(S, crit, 4, P, 30, 64, min_leaf=2, seed=9)
        res = []
        for on in (False, True):
            ctx.set_node_search(on)
            res.append(ctx.node_split(p, wl.X, labels=wl.labels, node_uid=11, want_trace=True))
            # rows go to shared memory in 16-byte chunks: d a multiple of 4
            assert (ctx.last_node_search() >= 1) == (on and d % 4 == 0)
        ctx.set_node_search(False)
        a, b = res
        assert np.array_equal(a["trace"], b["trace"])
        assert np.array_equal(a["gbest"].view(np.uint32), b["gbest"].view(np.uint32))
        assert (a["bin"], a["n_left"], a["iter_of_best"], a["particle"]) == \
            (b["bin"], b["n_left"], b["iter_of_best"], b["particle"])
