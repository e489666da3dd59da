"""The FP32 projection staged by tensor-map tile copies (the default) and by
per-thread asynchronous copies give identical results: the same z, ranges,
searches and trees, bit for bit, over feature counts that fill whole
32-feature chunks, end in a partial chunk, stay below one chunk, or are not
a multiple of 4 (no tensor map: both take the per-thread copies); particle
groups of every width; ragged tiles; bagged forests (gathered rows)."""
import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    a, b = context(), context()
    b.set_projection_tma(False)
    yield a, b
    a.close()
    b.close()


def same_tree(fa, fb, n_trees=1):
    for t in range(n_trees):
        ga, gb = fa.export(t), fb.export(t)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), (t, k)


@pytest.mark.parametrize("n,d,P", [
    (5000, 64, 64),   # whole chunks, 16-particle groups
    (3001, 36, 24),   # a partial chunk, ragged tail
    (2000, 20, 48),   # below one chunk, the widest group
    (1500, 30, 7),    # d % 4 != 0: no tensor map
    (7777, 128, 32),
])
def test_search_identical_with_and_without_tensor_maps(ctxs, n, d, P):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(n, d, 5, seed=d + P)
    p = gpu_params(S, "gini", 5, P, 12, 64, min_leaf=5, seed=3)
    ra = a.node_split(p, wl.X, labels=wl.labels, node_uid=9, want_trace=True)
    rb = b.node_split(p, wl.X, labels=wl.labels, node_uid=9, want_trace=True)
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"]) and ra["bin"] == rb["bin"]


@pytest.mark.parametrize("crit,K", [("gini", 6), ("mse", 0)])
def test_tree_identical_with_and_without_tensor_maps(ctxs, crit, K):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    if crit == "mse":
        wl = W.tanh_regression(20000, 32, seed=4)
        kw = dict(y=wl.y)
    else:
        wl = W.gmm(20000, 32, K, seed=4)
        kw = dict(labels=wl.labels)
    p = gpu_params(S, crit, K, 32, 10, 64, min_leaf=10, max_depth=6, seed=5)
    fa, fb = a.train_tree(p, wl.X, **kw), b.train_tree(p, wl.X, **kw)
    same_tree(fa, fb)
    fa.free()
    fb.free()


def test_forest_identical_with_and_without_tensor_maps(ctxs):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(30000, 16, 4, seed=6)
    p = gpu_params(S, "gini", 4, 24, 8, 64, min_leaf=10, max_depth=5, seed=7, n_trees=8,
                   bootstrap=True)
    fa, fb = a.train_tree(p, wl.X, labels=wl.labels), b.train_tree(p, wl.X, labels=wl.labels)
    same_tree(fa, fb, 8)
    fa.free()
    fb.free()
