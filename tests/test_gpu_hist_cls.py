"""The latency-oriented histogram kernels (k_hist_cls for classification,
k_hist_mse for regression; the defaults of FP32 searches) score exactly like
the staged-copy kernel they replace there: identical traces, gbest, splits,
trees and bagged forests for Gini, entropy and the squared error, class
counts spanning every register-array width (2 .. 32), bin counts that are
not multiples of 32 (down to 2, up to 256), multiplicities, nodes too small
for 16-byte loads of a whole slice, and levels whose small nodes go to the
warp-per-particle kernel. The oracle comparisons of the other GPU tests run
them too, since they are the default."""
import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    a, b = context(), context()
    b.set_class_hist(False)
    yield a, b
    a.close()
    b.close()


@pytest.fixture(scope="module")
def ctx_step():
    """The other placement of the gbest step and move (the default is the
    projection blocks; this one takes the last histogram block per node)."""
    c = context()
    c.set_fused_step(True, always=True)
    c.set_class_hist(True, node_step=True)
    yield c
    c.close()


def same_tree(fa, fb, n_trees=1):
    for t in range(n_trees):
        ga, gb = fa.export(t), fb.export(t)
        for k in ga:
            assert np.array_equal(ga[k], gb[k]), (t, k)


@pytest.mark.parametrize("crit", ["gini", "entropy"])
@pytest.mark.parametrize("n,d,K,P,B", [
    (6000, 24, 2, 32, 64),
    (5003, 16, 5, 48, 50),    # bins not a multiple of 32, ragged slices
    (9000, 32, 10, 64, 128),
    (4000, 12, 20, 16, 128),
    (3000, 8, 32, 24, 2),     # the most classes, two bins
    (37, 4, 3, 16, 16),       # a node smaller than one 16-byte group per thread
])
def test_search_identical_with_both_histogram_kernels(ctxs, ctx_step, crit, n, d, K, P, B):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(n, d, K, seed=n % 97 + K)
    p = gpu_params(S, crit, K, P, 10, B, min_leaf=3, seed=5)
    rb = b.node_split(p, wl.X, labels=wl.labels, node_uid=4, want_trace=True)
    for c in (a, ctx_step):  # the move in k_step, or in the last histogram block
        ra = c.node_split(p, wl.X, labels=wl.labels, node_uid=4, want_trace=True)
        assert np.array_equal(ra["trace"], rb["trace"])
        assert np.array_equal(ra["gbest"], rb["gbest"])
        for k in ("bin", "q_num", "q_den", "loss", "n_left", "n_right", "particle",
                  "iter_of_best"):
            assert ra[k] == rb[k], k


@pytest.mark.parametrize("crit,bootstrap", [("gini", False), ("entropy", True), ("gini", True)])
def test_forest_identical_with_both_histogram_kernels(ctxs, ctx_step, crit, bootstrap):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(24000, 20, 6, seed=11)
    p = gpu_params(S, crit, 6, 32, 8, 128, min_leaf=10, max_depth=7, seed=3,
                   n_trees=3 if bootstrap else 1, bootstrap=bootstrap)
    fb = b.train_tree(p, wl.X, labels=wl.labels)
    for c in (a, ctx_step):
        fa = c.train_tree(p, wl.X, labels=wl.labels)
        same_tree(fa, fb, p.n_trees)
        fa.free()
    # every level through the classification kernel (no warp-per-particle
    # nodes), so each level's move runs in the last histogram blocks
    ctx_step.set_small_nodes(0, 0)
    try:
        fa = ctx_step.train_tree(p, wl.X, labels=wl.labels)
        same_tree(fa, fb, p.n_trees)
        fa.free()
    finally:
        ctx_step.set_small_nodes()
    fb.free()


def test_unfused_search_identical_with_both_histogram_kernels(ctxs):
    """The new kernel under the three-kernel iteration (no folded move)."""
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.gmm(8000, 20, 4, seed=12)
    p = gpu_params(S, "gini", 4, 100, 8, 64, min_leaf=5, seed=9)  # 112 padded: not folded
    ra = a.node_split(p, wl.X, labels=wl.labels, node_uid=1, want_trace=True)
    rb = b.node_split(p, wl.X, labels=wl.labels, node_uid=1, want_trace=True)
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"]) and ra["bin"] == rb["bin"]


@pytest.mark.parametrize("n,d,P,B,weighted", [
    (6000, 24, 32, 64, False),
    (5003, 16, 48, 256, False),   # the most bins, ragged slices
    (20000, 12, 64, 128, False),  # a cluster of slices per particle
    (37, 4, 16, 16, False),       # a node smaller than one 16-byte group per thread
    (9000, 20, 40, 100, True),    # multiplicities (bagging)
])
def test_regression_identical_with_both_histogram_kernels(ctxs, n, d, P, B, weighted):
    """The squared-error kernel (lane-private copies of the fixed-point bin
    moments) scores exactly like the staged-copy counting-sort kernel."""
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.tanh_regression(n, d, seed=n % 89)
    p = gpu_params(S, "mse", 0, P, 8, B, min_leaf=3, seed=7)
    kw = {}
    if weighted:
        rng = np.random.default_rng(3)
        idx, w = np.unique(rng.integers(0, n, n), return_counts=True)
        kw = dict(sample_idx=idx.astype(np.int32), weights=w.astype(np.uint32))
    ra = a.node_split(p, wl.X, y=wl.y, node_uid=6, want_trace=True, **kw)
    rb = b.node_split(p, wl.X, y=wl.y, node_uid=6, want_trace=True, **kw)
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"])
    for k in ("bin", "loss", "n_left", "n_right", "particle", "iter_of_best"):
        assert ra[k] == rb[k], k


@pytest.mark.parametrize("bootstrap", [False, True])
def test_regression_trees_identical_with_both_histogram_kernels(ctxs, bootstrap):
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.tanh_regression(30000, 16, seed=4)
    p = gpu_params(S, "mse", 0, 32, 6, 128, min_leaf=10, max_depth=7, seed=2,
                   n_trees=3 if bootstrap else 1, bootstrap=bootstrap)
    fa = a.train_tree(p, wl.X, y=wl.y)
    fb = b.train_tree(p, wl.X, y=wl.y)
    same_tree(fa, fb, p.n_trees)
    fa.free()
    fb.free()


def test_bf16_regression_identical_with_both_histogram_kernels(ctxs):
    """The BF16 form's reduced pass (its last CTA per node selecting the top
    k) and FP32 re-scoring pass on the squared-error kernel: the same search
    and tree as with the staged-copy kernel."""
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.tanh_regression(20000, 32, seed=6)
    p = S.make_params("mse", 0, n_particles=64, n_iters=6, n_bins=128, min_leaf=5, seed=3,
                      max_depth=6, proj=S.SLM_PROJ_BF16_TOPK, topk=8)
    ra = a.node_split(p, wl.X, y=wl.y, node_uid=2, want_trace=True)
    rb = b.node_split(p, wl.X, y=wl.y, node_uid=2, want_trace=True)
    assert np.array_equal(ra["trace"], rb["trace"])
    assert np.array_equal(ra["gbest"], rb["gbest"])
    for k in ("bin", "loss", "n_left", "n_right", "particle", "iter_of_best"):
        assert ra[k] == rb[k], k
    fa = a.train_tree(p, wl.X, y=wl.y)
    fb = b.train_tree(p, wl.X, y=wl.y)
    same_tree(fa, fb)
    fa.free()
    fb.free()


def test_regression_pairs_of_particles_per_block(ctxs):
    """Wide regression levels (at least 4,096 node-particle pairs) score two
    particles per block, here with an odd swarm (the last block one
    particle): the same trees as the staged-copy kernel."""
    from paper_2208_07023_gb300 import binding as S
    a, b = ctxs
    wl = W.tanh_regression(40000, 12, seed=9)
    p = gpu_params(S, "mse", 0, 127, 3, 64, min_leaf=8, max_depth=8, seed=5)
    fa = a.train_tree(p, wl.X, y=wl.y)
    fb = b.train_tree(p, wl.X, y=wl.y)
    same_tree(fa, fb)
    g = fa.export(0)
    assert (g["kind"] == 1).sum() >= 64  # levels of 32+ nodes x 127 particles were scored
    fa.free()
    fb.free()
