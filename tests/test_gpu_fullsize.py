"""Parity at the full size of the classification-tree workload, in the launch
configuration the benchmark times (n=50,000, d=64, K=10 Gaussian mixture,
depth <= 8, min leaf 20, P=64, T=100, B=128, Gini).

The oracle cannot grow this tree in seconds, so it checks sampled outputs one
by one: every internal node's gB is re-scored by the oracle on the node's
samples (bins, counts and the exact Gini rational must agree), and the full
swarm search of the root and of a few deep nodes is repeated by the oracle
(identical gB and trajectory). Structural invariants are checked everywhere.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params, oracle_params

pytestmark = pytest.mark.gpu

CFG = W.SETTINGS["tree_n50k_d64_k10"]


@pytest.fixture(scope="module")
def grown():
    ctx = context()
    wl = CFG["builder"](1)
    from paper_2208_07023_gb300 import binding as S
    gp = gpu_params(S, "gini", 10, CFG["n_particles"], CFG["n_iters"], CFG["n_bins"],
                    min_leaf=CFG["min_leaf"], max_depth=CFG["max_depth"], seed=1)
    f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    g = f.export(0)
    _, _, leaf = ctx.predict(f, wl.X, want_leaf=True)
    yield wl, g, leaf[:, 0], f.info()
    f.free()
    ctx.close()


def node_members(leaf, h):
    """Training samples whose path passes through heap node h."""
    out = np.zeros(leaf.shape[0], bool)
    node = leaf.copy()
    while True:
        out |= node == h
        if (node <= h).all():
            break
        node = np.where(node > h, (node - 1) // 2, node)
    return np.nonzero(out)[0].astype(np.int32)


def test_structure(grown):
    wl, g, leaf, info = grown
    H = len(g["kind"])
    assert g["weight"][0] == wl.n
    for h in np.nonzero(g["kind"] == 1)[0]:
        l, r = 2 * h + 1, 2 * h + 2
        assert g["n_left"][h] == g["weight"][l] and g["n_right"][h] == g["weight"][r]
        assert g["weight"][l] + g["weight"][r] == g["weight"][h]
        assert min(g["weight"][l], g["weight"][r]) >= CFG["min_leaf"]
    for h in np.nonzero(g["kind"] == 0)[0]:
        assert (leaf == h).sum() == g["weight"][h]
        cnt = np.bincount(wl.labels[leaf == h], minlength=10)
        assert g["leaf_class"][h] == int(np.argmax(cnt))
    # training loss falls with depth: misclassified training samples
    err = np.mean(g["leaf_class"][leaf] != wl.labels)
    assert err < 0.5
    searched = sum(len(node_members(leaf, h)) for h in np.nonzero(g["kind"] >= 0)[0]
                   if g["kind"][h] == 1)
    assert info["evaluations"] >= searched * CFG["n_particles"] * (CFG["n_iters"] + 1)


def test_every_split_rescored_by_oracle(grown):
    wl, g, leaf, _ = grown
    op = oracle_params(O, "gini", 10, 1, 0, CFG["n_bins"], min_leaf=CFG["min_leaf"])
    inner = np.nonzero(g["kind"] == 1)[0]
    for h in inner:
        idx = node_members(leaf, h)
        e = O.eval_swarm(op, wl.X, wl.labels, None, g["dir"][h].astype(np.float64)[None, :],
                         idx=idx)[0][0]
        assert (e["bin"], e["n_left"], e["n_right"]) == (g["bin"][h], g["n_left"][h],
                                                         g["n_right"][h])
        assert np.float32(e["zmin"]) == g["zmin"][h] and np.float32(e["inv_w"]) == g["inv_w"][h]
        assert e["loss"] == g["loss"][h]


@pytest.mark.parametrize("pick", ["root", "deep0", "deep1"])
def test_sampled_node_searches(grown, pick):
    wl, g, leaf, _ = grown
    inner = np.nonzero(g["kind"] == 1)[0]
    h = {"root": 0, "deep0": inner[-1], "deep1": inner[len(inner) // 2]}[pick]
    idx = node_members(leaf, h)
    op = oracle_params(O, "gini", 10, CFG["n_particles"], CFG["n_iters"], CFG["n_bins"],
                       min_leaf=CFG["min_leaf"], seed=1)
    r = O.node_split(op, wl.X, wl.labels, idx=idx, node_uid=int(h))
    assert np.array_equal(r.gbest, g["dir"][h].astype(np.float64))
    assert r.split["bin"] == g["bin"][h] and r.split["loss"] == g["loss"][h]
