"""GPU parity at the limits of the parameters: the largest swarm (P = 256,
and P = 255 with adaptive PSO, whose elite candidate takes the 256th slot),
a single feature (d = 1, directions +-a), the fewest bins (B = 2: one edge),
and nodes just above and below the admissible size."""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def compare(ctx, gp, op, X, labels, uid=5):
    g = ctx.node_split(gp, X, labels=labels, node_uid=uid, want_trace=True)
    r = O.node_split(op, X, labels, node_uid=uid)
    assert np.array_equal(g["trace"], r.trace_loss)
    assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
    assert (g["particle"], g["iter_of_best"], g["bin"], g["n_left"]) == \
        (r.split["particle"], r.split["iter_of_best"], r.split["bin"], r.split["n_left"])
    return g, r


@pytest.mark.parametrize("P,apso", [(256, False), (255, True)])
def test_largest_swarm(ctx, P, apso):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(1500, 8, 3, seed=P)
    gp = S.make_params("gini", 3, n_particles=P, n_iters=6, n_bins=32, min_leaf=5, seed=2,
                       apso=apso)
    op = oracle_params(O, "gini", 3, P, 6, 32, min_leaf=5, seed=2)
    op.apso = 1 if apso else 0
    compare(ctx, gp, op, wl.X, wl.labels)


def test_single_feature_and_two_bins(ctx):
    from paper_2208_07023_gb300 import binding as S
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3000, 1)).astype(np.float32)
    lab = (X[:, 0] > 0.3).astype(np.int32)
    for B in (2, 64):
        gp = gpu_params(S, "gini", 2, 16, 10, B, min_leaf=5, seed=3)
        op = oracle_params(O, "gini", 2, 16, 10, B, min_leaf=5, seed=3)
        g, r = compare(ctx, gp, op, X, lab)
        if B == 2:
            assert g["bin"] == 1  # the one interior edge
    # a one-feature tree: every direction is +-1 times a scale
    f = ctx.train_tree(gpu_params(S, "gini", 2, 16, 10, 64, min_leaf=5, seed=3, max_depth=3),
                       X, labels=lab)
    e = f.export(0)
    inner = e["kind"] == 1
    assert inner.any() and np.all(e["dir"][inner, 0] != 0)
    f.free()


def test_node_size_at_the_split_limit(ctx):
    # a node splits only with at least 2 min_leaf samples (weight)
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(200, 4, 2, seed=9)
    for n, want_valid in ((20, True), (19, False)):
        gp = gpu_params(S, "gini", 2, 8, 4, 16, min_leaf=10, seed=1, max_depth=1)
        f = ctx.train_tree(gp, wl.X[:n], labels=wl.labels[:n])
        e = f.export(0)
        r = O.train_tree(oracle_params(O, "gini", 2, 8, 4, 16, min_leaf=10, seed=1,
                                       max_depth=1), wl.X[:n], wl.labels[:n])
        assert np.array_equal(e["kind"], r.kind)
        assert (e["kind"][0] == 1) == (want_valid and r.kind[0] == 1)
        f.free()
