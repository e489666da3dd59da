"""The swarm move folded into the projection (k_step, the default for plain
FP32 searches of 16, 32, 48 or 64 padded particles) gives the results of the
projection / histogram / move kernels bit for bit: traces, gbest, splits,
trees (classification and regression) and bagged forests, over feature
counts that fill whole 32-feature chunks, end in a partial chunk or are not
a multiple of 4, every supported padded swarm width, ragged tiles, levels
whose small nodes take the warp-per-particle histogram, graph-captured
loops, and zero iterations. The oracle comparisons of the other GPU tests run
the folded path too, since it is the default."""
import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    a, b = context(), context()
    a.set_fused_step(True, always=True)  # fold every eligible batch, however long
    b.set_fused_step(False)
    yield a, b
    a.close()
    b.close()


def same_tree(fa, fb, n_trees=1):
    for t in range(n_trees):
        ga, gb = fa.export(t), fb.export(t)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), (t, k)


@pytest.mark.parametrize("n,d,P,T", [
    (5000, 64, 64, 12),   # whole chunks, the widest swarm
    (3001, 36, 45, 9),    # a partial chunk, ragged tail, 48 padded particles
    (2000, 20, 32, 7),    # below one chunk
    (1500, 30, 7, 6),     # d % 4 != 0, 16 padded particles
    (7777, 128, 50, 5),
    (900, 1, 16, 4),      # one feature
    (2500, 16, 64, 0),    # zero iterations: the initial swarm only
])
def test_search_identical_folded_and_separate(ctxs, n, d, P, T):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    before = a.set_fused_step(True, always=True)
    wl = W.gmm(n, d, 5, seed=d + P)
    p = gpu_params(S, "gini", 5, P, T, 64, min_leaf=5, seed=3)
    ra = a.node_split(p, wl.X, labels=wl.labels, node_uid=9, want_trace=True)
    rb = b.node_split(p, wl.X, labels=wl.labels, node_uid=9, want_trace=True)
    assert a.set_fused_step(True, always=True) == before + 1  # the search ran folded
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"])
    for k in ("bin", "q_num", "q_den", "n_left", "n_right", "particle", "iter_of_best"):
        assert ra[k] == rb[k], k


@pytest.mark.parametrize("crit", ["entropy", "mse"])
def test_search_identical_other_criteria(ctxs, crit):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    if crit == "mse":
        wl = W.tanh_regression(6000, 24, seed=8)
        kw = dict(y=wl.y)
    else:
        wl = W.gmm(6000, 24, 3, seed=8)
        kw = dict(labels=wl.labels)
    p = gpu_params(S, crit, 3, 40, 15, 128, min_leaf=5, seed=4)
    ra = a.node_split(p, wl.X, node_uid=2, want_trace=True, **kw)
    rb = b.node_split(p, wl.X, node_uid=2, want_trace=True, **kw)
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"]) and ra["bin"] == rb["bin"]


@pytest.mark.parametrize("crit,K,P", [("gini", 6, 64), ("mse", 0, 32), ("entropy", 4, 48)])
def test_tree_identical_folded_and_separate(ctxs, crit, K, P):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    if crit == "mse":
        wl = W.tanh_regression(20000, 32, seed=4)
        kw = dict(y=wl.y)
    else:
        wl = W.gmm(20000, 32, K, seed=4)
        kw = dict(labels=wl.labels)
    # depth 7: the deep levels' small nodes take the warp-per-particle kernel
    p = gpu_params(S, crit, K, P, 10, 64, min_leaf=10, max_depth=7, seed=5)
    fa, fb = a.train_tree(p, wl.X, **kw), b.train_tree(p, wl.X, **kw)
    same_tree(fa, fb)
    fa.free()
    fb.free()


def test_forest_and_graphs_identical_folded_and_separate(ctxs):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(30000, 16, 4, seed=6)
    p = gpu_params(S, "gini", 4, 24, 8, 64, min_leaf=10, max_depth=5, seed=7, n_trees=8,
                   bootstrap=True)
    fb = b.train_tree(p, wl.X, labels=wl.labels)
    fa = a.train_tree(p, wl.X, labels=wl.labels)
    same_tree(fa, fb, 8)
    fa.free()
    a.set_graphs(True)
    try:
        fg = a.train_tree(p, wl.X, labels=wl.labels)
        same_tree(fg, fb, 8)
        fg.free()
    finally:
        a.set_graphs(False)
    fb.free()


def test_default_folds_short_levels_only():
    """The default folds a batch whose projection is a few waves of row
    tiles and leaves a long one to the separate kernels; results match."""
    from paper_2208_07023_gb300 import binding as S
    c = context()
    try:
        ref = context()
        ref.set_fused_step(False)
        p = gpu_params(S, "gini", 4, 64, 3, 64, min_leaf=5, seed=2)
        for n, folded in ((20000, True), (400000, False)):  # 157 / 3125 tiles of 128 rows
            wl = W.gmm(n, 16, 4, seed=5)
            before = c.set_fused_step(True)
            r = c.node_split(p, wl.X, labels=wl.labels, node_uid=3, want_trace=True)
            assert c.set_fused_step(True) == before + int(folded)
            q = ref.node_split(p, wl.X, labels=wl.labels, node_uid=3, want_trace=True)
            assert np.array_equal(r["trace"], q["trace"]) and r["bin"] == q["bin"]
            assert np.array_equal(r["gbest"], q["gbest"])
        with pytest.raises(S.SlmError):
            c._check(S.lib().slm_set_fused_step(c.handle, 3, None))
        ref.close()
    finally:
        c.close()


@pytest.mark.parametrize("P,d", [(64, 64), (32, 20), (16, 30), (48, 12)])
def test_every_tile_shape_gives_the_same_search(ctxs, P, d):
    """The folded projection's tile shapes (rows per unit 32-256, every
    particle or half of them per unit) project the same z and move the same
    swarm: searches identical to the unfolded kernels for each shape, and a
    swarm width without a shape falls back to shape 0."""
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(3001, d, 4, seed=P)
    p = gpu_params(S, "gini", 4, P, 6, 64, min_leaf=5, seed=7)
    rb = b.node_split(p, wl.X, labels=wl.labels, node_uid=5, want_trace=True)
    try:
        # shapes each swarm width has (3-5: half the particles per unit)
        have = {64: {0, 1, 2, 3, 4, 5}, 32: {0, 1, 2, 3, 4}, 16: {0, 1}, 48: {0}}[P]
        for sh in range(6):
            a.set_step_shape(sh)
            ra = a.node_split(p, wl.X, labels=wl.labels, node_uid=5, want_trace=True)
            used = a.set_step_shape(sh)
            assert used == (sh if sh in have else 0)
            assert np.array_equal(ra["trace"], rb["trace"])
            assert np.array_equal(ra["gbest"], rb["gbest"]) and ra["bin"] == rb["bin"]
        fa = None
        a.set_step_shape(5 if P == 64 else 2)
        pt = gpu_params(S, "gini", 4, P, 4, 64, min_leaf=5, max_depth=5, seed=2)
        fa = a.train_tree(pt, wl.X, labels=wl.labels)
        fb = b.train_tree(pt, wl.X, labels=wl.labels)
        same_tree(fa, fb)
        fa.free()
        fb.free()
    finally:
        a.set_step_shape(-1)
    with pytest.raises(S.SlmError):
        a.set_step_shape(6)
