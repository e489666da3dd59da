"""Parity at the full size of the regression-tree workload with the bfloat16
tensor-core projection and top-8 FP32 re-scoring (n=200,000, d=128,
y = sum of 8 tanh ridges + noise, depth <= 10, min leaf 20, P=64, T=80,
B=256, MSE), in the configuration the benchmark times.

Every split of the grown tree is an FP32 score of its direction: the oracle
re-scores each internal node's gB on the node's samples with the FP32 mirror
projection and must reproduce its bins, counts and range exactly and its
loss to 1e-9 (double sums in another order). Structure is checked at every
node.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, oracle_params

pytestmark = pytest.mark.gpu

CFG = W.SETTINGS["regtree_n200k_d128"]


@pytest.fixture(scope="module")
def grown():
    ctx = context()
    wl = CFG["builder"](1)
    from paper_2208_07023_gb300 import binding as S
    gp = S.make_params("mse", 0, n_particles=CFG["n_particles"], n_iters=CFG["n_iters"],
                       n_bins=CFG["n_bins"], min_leaf=CFG["min_leaf"],
                       max_depth=CFG["max_depth"], seed=1, proj=S.SLM_PROJ_BF16_TOPK,
                       topk=CFG["topk"])
    f = ctx.train_tree(gp, wl.X, y=wl.y)
    g = f.export(0)
    _, val, leaf = ctx.predict(f, wl.X, want_leaf=True)
    yield wl, g, leaf[:, 0], val
    f.free()
    ctx.close()


def members_by_node(leaf):
    """Sorted training-sample ids of every heap node on the samples' paths."""
    anc, ids = [], []
    node = leaf.astype(np.int64).copy()
    s = np.arange(leaf.shape[0])
    while True:
        anc.append(node.copy())
        ids.append(s)
        if (node == 0).all():
            break
        keep = node > 0
        node, s = (node[keep] - 1) // 2, s[keep]
    a, i = np.concatenate(anc), np.concatenate(ids)
    order = np.lexsort((i, a))
    a, i = a[order], i[order]
    cuts = np.flatnonzero(np.diff(a)) + 1
    return {int(a[c0]): i[c0:c1].astype(np.int32)
            for c0, c1 in zip(np.r_[0, cuts], np.r_[cuts, a.size])}


def test_structure(grown):
    wl, g, leaf, val = grown
    assert g["weight"][0] == wl.n
    inner = np.nonzero(g["kind"] == 1)[0]
    assert len(inner) >= 100
    for h in inner:
        l, r = 2 * h + 1, 2 * h + 2
        assert g["n_left"][h] == g["weight"][l] and g["n_right"][h] == g["weight"][r]
        assert min(g["weight"][l], g["weight"][r]) >= CFG["min_leaf"]
    for h in np.nonzero(g["kind"] == 0)[0]:
        on = leaf == h
        assert on.sum() == g["weight"][h]
        assert g["leaf_value"][h] == pytest.approx(wl.y[on].astype(np.float64).mean(), rel=1e-9,
                                                   abs=1e-12)
    # the tree explains most of the variance of the training targets
    assert np.mean((val - wl.y) ** 2) < 0.5 * np.var(wl.y)


def test_every_split_rescored_by_oracle(grown):
    wl, g, leaf, _ = grown
    op = oracle_params(O, "mse", 0, 1, 0, CFG["n_bins"], min_leaf=CFG["min_leaf"])
    mem = members_by_node(leaf)
    for h in np.nonzero(g["kind"] == 1)[0]:
        idx = mem[int(h)]
        e = O.eval_swarm(op, wl.X, None, wl.y, g["dir"][h].astype(np.float64)[None, :],
                         idx=idx)[0][0]
        assert (e["bin"], e["n_left"], e["n_right"]) == (g["bin"][h], g["n_left"][h],
                                                         g["n_right"][h])
        assert np.float32(e["zmin"]) == g["zmin"][h] and np.float32(e["inv_w"]) == g["inv_w"][h]
        assert e["loss"] == pytest.approx(g["loss"][h], rel=1e-9)
