"""GPU parity: libslm (through its C ABI) against the CPU oracle.

Bars:
* integer work (bins, counts, partitions, node ids) bit-exact against the
  oracle's fp32 mirror, which runs the same fused multiply-add sequence;
  against the fp64 oracle, bin mismatches only for samples within 1e-6
  (relative to the projected range) of a bin edge;
* Gini decisions exact (both sides compare exact rationals), so whole swarm
  trajectories and trees are identical; entropy losses within 1e-12 relative
  (both in double; only log() may differ in the last place) and trajectories
  identical up to the oracle's first logged near-tie; MSE losses within 1e-9
  relative (per-bin sums of doubles are accumulated in another order);
* projections / impurities against the fp64 oracle within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, edge_distance, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


# ---------------------------------------------------------------- RNG -------

@pytest.mark.parametrize("seed,uid,t,P,d,purpose", [
    (1, 0, 0, 32, 16, 1), (0xDEADBEEF12345, 65536 + 7, 99, 64, 64, 3),
    (7, 3, 5, 5, 13, 4), (2**64 - 1, 2**32 - 1, 2**31, 3, 1, 2)])
def test_swarm_draws_bitwise(ctx, seed, uid, t, P, d, purpose):
    g = ctx.swarm_uniforms(seed, uid, t, P, d, purpose)
    o = O.swarm_uniforms(seed, uid, t, P, d, purpose)
    assert np.array_equal(g.view(np.uint32), o.view(np.uint32))


@pytest.mark.parametrize("n", [1, 5, 1000, 100_003])
def test_bootstrap_bitwise(ctx, n):
    for tree in (0, 1, 63):
        assert np.array_equal(ctx.bootstrap(42, tree, n), O.bootstrap(42, tree, n))


# ------------------------------------------------------------ scoring -------

def _node_inputs(crit, n, d, K, seed, n_idx=None, weighted=False):
    rng = np.random.default_rng(seed)
    if crit == "mse":
        wl = W.tanh_regression(n, d, seed=seed)
    else:
        wl = W.gmm(n, d, K, seed=seed)
    idx = None
    if n_idx is not None:
        idx = rng.choice(n, n_idx, replace=False).astype(np.int32)
    wts = None
    if weighted:
        m = n if idx is None else n_idx
        wts = rng.integers(1, 4, m).astype(np.uint32)
    return wl, idx, wts


SCORE_CASES = [
    # crit, K, B, d, n, n_idx, P, weighted
    ("gini", 10, 128, 64, 3000, 700, 64, False),      # one CTA per group
    ("gini", 10, 128, 64, 9000, 5003, 48, True),      # chunked, ragged tail
    ("entropy", 2, 64, 16, 2000, None, 32, False),
    ("entropy", 5, 32, 37, 6000, 4099, 20, True),     # d not a multiple of 4
    ("mse", 0, 256, 32, 4000, 1500, 16, False),
    ("mse", 0, 100, 9, 7000, None, 33, True),
    ("gini", 32, 80, 3, 2500, None, 17, False),       # largest B*K
]


@pytest.mark.parametrize("crit,K,B,d,n,n_idx,P,weighted", SCORE_CASES)
def test_scores_match_mirror_bitwise(ctx, crit, K, B, d, n, n_idx, P, weighted):
    from paper_2208_07023_gb300 import binding as S
    wl, idx, wts = _node_inputs(crit, n, d, K, seed=B + d, n_idx=n_idx, weighted=weighted)
    rng = np.random.default_rng(5)
    pos = rng.uniform(-1, 1, (P, d)).astype(np.float32)
    gp = gpu_params(S, crit, K, P, 0, B, min_leaf=3)
    res, bins = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y,
                                   sample_idx=idx, weights=wts, want_bins=True)
    op = oracle_params(O, crit, K, P, 0, B, min_leaf=3)
    ref, rbins, _ = O.eval_swarm(op, wl.X, wl.labels, wl.y, pos.astype(np.float64),
                                 idx=idx, wts=wts, want_bins=True)
    assert np.array_equal(bins, rbins)
    for g, r in zip(res, ref):
        assert g["valid"] == r["valid"]
        assert g["zmin"] == np.float32(r["zmin"]) and g["inv_w"] == np.float32(r["inv_w"])
        if not r["valid"]:
            continue
        assert (g["bin"], g["n_left"], g["n_right"]) == (r["bin"], r["n_left"], r["n_right"])
        if crit == "gini":
            assert (g["q_num"], g["q_den"], g["loss"]) == (r["q_num"], r["q_den"], r["loss"])
        elif crit == "entropy":
            assert g["loss"] == pytest.approx(r["loss"], rel=1e-12)
        else:
            assert g["loss"] == pytest.approx(r["loss"], rel=1e-9)


@pytest.mark.parametrize("crit,K,B,d,n,n_idx,P,weighted", SCORE_CASES[:5])
def test_scores_match_f64_oracle(ctx, crit, K, B, d, n, n_idx, P, weighted):
    from paper_2208_07023_gb300 import binding as S
    wl, idx, wts = _node_inputs(crit, n, d, K, seed=B + d, n_idx=n_idx, weighted=weighted)
    rng = np.random.default_rng(6)
    pos = rng.uniform(-1, 1, (P, d)).astype(np.float32)
    gp = gpu_params(S, crit, K, P, 0, B, min_leaf=3)
    res, bins = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y,
                                   sample_idx=idx, weights=wts, want_bins=True)
    op = oracle_params(O, crit, K, P, 0, B, min_leaf=3, precision=O.F64)
    ref, rbins, z = O.eval_swarm(op, wl.X, wl.labels, wl.y, pos.astype(np.float64),
                                 idx=idx, wts=wts, want_bins=True, want_z=True)
    for i, (g, r) in enumerate(zip(res, ref)):
        span = max(abs(r["zmin"]), abs(r["zmax"]))
        assert abs(g["zmin"] - r["zmin"]) <= 1e-5 * span
        mism = bins[i] != rbins[i]
        if mism.any():
            dist = edge_distance(z[i][mism], r["zmin"], r["zmax"], B)
            assert np.all(dist <= 1e-6 * (r["zmax"] - r["zmin"] + span))
        elif r["valid"]:
            assert g["bin"] == r["bin"]
            assert g["loss"] == pytest.approx(r["loss"], rel=1e-5)


def test_degenerate_nodes(ctx):
    from paper_2208_07023_gb300 import binding as S
    X = np.ones((300, 4), np.float32)
    lab = (np.arange(300) % 3).astype(np.int32)
    gp = gpu_params(S, "gini", 3, 5, 0, 16)
    pos = np.random.default_rng(0).uniform(-1, 1, (5, 4)).astype(np.float32)
    res, _ = ctx.evaluate_swarm(gp, X, pos, labels=lab)
    assert all(r["valid"] == 0 and np.isinf(r["loss"]) for r in res)
    # empty node
    res, _ = ctx.evaluate_swarm(gp, X, pos, labels=lab, sample_idx=np.zeros(0, np.int32))
    assert all(r["valid"] == 0 for r in res)
    # min_leaf larger than half the node
    X = np.random.default_rng(1).standard_normal((40, 2)).astype(np.float32)
    gp = gpu_params(S, "gini", 3, 2, 0, 8, min_leaf=21)
    res, _ = ctx.evaluate_swarm(gp, X, pos[:2, :2].copy(), labels=lab[:40].copy())
    assert all(r["valid"] == 0 for r in res)
    # B = 2: one edge
    gp = gpu_params(S, "entropy", 3, 2, 0, 2)
    res, _ = ctx.evaluate_swarm(gp, X, pos[:2, :2].copy(), labels=lab[:40].copy())
    ref, _, _ = O.eval_swarm(oracle_params(O, "entropy", 3, 2, 0, 2), X, lab[:40], None,
                             pos[:2, :2].astype(np.float64))
    assert [r["bin"] for r in res] == [r["bin"] for r in ref]


def test_bad_arguments_are_rejected(ctx):
    from paper_2208_07023_gb300 import binding as S
    X = np.random.default_rng(1).standard_normal((50, 3)).astype(np.float32)
    pos = np.ones((2, 3), np.float32)
    with pytest.raises(S.SlmError) as e:
        ctx.evaluate_swarm(gpu_params(S, "gini", 3, 2, 0, 16), X, pos,
                           labels=np.full(50, 3, np.int32))
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.evaluate_swarm(gpu_params(S, "gini", 3, 2, 0, 16), X, pos,
                           labels=np.zeros(50, np.int32),
                           sample_idx=np.array([0, 50], np.int32))
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.evaluate_swarm(gpu_params(S, "gini", 40, 2, 0, 16), X, pos,
                           labels=np.zeros(50, np.int32))
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.node_split(gpu_params(S, "gini", 2, 0, 5, 16), X, labels=np.zeros(50, np.int32))
    assert e.value.status == S.SLM_EINVAL


# -------------------------------------------------------- swarm search -------

@pytest.mark.parametrize("crit,K,B,d,n,n_idx,P,T", [
    ("gini", 4, 64, 16, 3000, None, 32, 20),
    ("gini", 10, 128, 64, 8000, 6001, 64, 12),    # chunked node
    ("gini", 3, 32, 5, 500, None, 7, 30),         # P not a multiple of 16
    ("entropy", 2, 64, 16, 2000, None, 32, 50),   # the single-node setting
])
def test_node_split_trajectory(ctx, crit, K, B, d, n, n_idx, P, T):
    from paper_2208_07023_gb300 import binding as S
    wl, idx, _ = _node_inputs(crit, n, d, K, seed=P + T, n_idx=n_idx)
    if crit == "entropy" and K == 2:
        wl = W.single_node(n, d, seed=3)
    gp = gpu_params(S, crit, K, P, T, B, min_leaf=2, seed=99)
    g = ctx.node_split(gp, wl.X, labels=wl.labels, sample_idx=idx, node_uid=77,
                       want_trace=True)
    r = O.node_split(oracle_params(O, crit, K, P, T, B, min_leaf=2, seed=99), wl.X,
                     wl.labels, idx=idx, node_uid=77)
    stop = r.split["first_near_tie"]
    upto = T + 1 if stop < 0 else stop
    assert np.array_equal(g["trace"][:upto], r.trace_loss[:upto])
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
        assert (g["particle"], g["iter_of_best"], g["bin"]) == \
            (r.split["particle"], r.split["iter_of_best"], r.split["bin"])
        assert g["loss"] == r.split["loss"]
        assert np.allclose(g["direction"], r.direction, atol=1e-6)
        assert g["threshold"] == np.float32(r.split["threshold"])


def test_node_split_regression(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(3000, 12, seed=2)
    gp = gpu_params(S, "mse", 0, 16, 15, 64, min_leaf=5, seed=4)
    g = ctx.node_split(gp, wl.X, y=wl.y, node_uid=5, want_trace=True)
    r = O.node_split(oracle_params(O, "mse", 0, 16, 15, 64, min_leaf=5, seed=4), wl.X,
                     None, wl.y, node_uid=5)
    stop = r.split["first_near_tie"]
    upto = 16 if stop < 0 else stop
    assert np.allclose(g["trace"][:upto], r.trace_loss[:upto], rtol=1e-9)
    # the returned gbest re-scored by the oracle gives the reported loss
    e = O.eval_swarm(oracle_params(O, "mse", 0, 1, 0, 64, min_leaf=5), wl.X, None, wl.y,
                     g["gbest"].astype(np.float64)[None, :])[0][0]
    assert e["loss"] == pytest.approx(g["loss"], rel=1e-9) and e["bin"] == g["bin"]


def test_host_and_device_inputs_agree(ctx):
    """Device pointers are used in place; host arrays are staged by the call."""
    import ctypes
    torch = pytest.importorskip("torch")
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(2500, 8, 3, seed=4)
    gp = gpu_params(S, "gini", 3, 16, 10, 32, min_leaf=4)
    h = ctx.node_split(gp, wl.X, labels=wl.labels, node_uid=1)
    Xd = torch.from_numpy(wl.X).cuda()
    Ld = torch.from_numpy(wl.labels).cuda()
    dd = torch.empty(8, dtype=torch.float32, device="cuda")
    sp = S.slm_split()
    torch.cuda.synchronize()
    st = S.lib().slm_node_split(ctx.handle, ctypes.byref(gp), Xd.data_ptr(), 2500, 8,
                                Ld.data_ptr(), None, None, None, 2500, 1, dd.data_ptr(),
                                None, ctypes.byref(sp), None)
    assert st == S.SLM_OK
    assert (sp.eval.q_num, sp.eval.q_den, sp.eval.bin) == (h["q_num"], h["q_den"], h["bin"])
    assert np.array_equal(dd.cpu().numpy(), h["direction"])


# -------------------------------------------------------------- trees -------

def _compare_tree(g, r, d):
    H = len(r.kind)
    assert np.array_equal(g["kind"], r.kind)
    inner = r.kind == 1
    assert np.array_equal(g["dir"][inner].astype(np.float64), r.dir[inner])
    assert np.array_equal(g["zmin"][inner], r.zmin[inner].astype(np.float32))
    assert np.array_equal(g["inv_w"][inner], r.inv_w[inner].astype(np.float32))
    assert np.array_equal(g["bin"][inner], r.bin[inner])
    assert np.array_equal(g["n_left"][inner], r.n_left[inner].astype(np.int64))
    assert np.array_equal(g["n_right"][inner], r.n_right[inner].astype(np.int64))
    present = r.kind >= 0
    assert np.array_equal(g["weight"][present], r.weight[present].astype(np.int64))
    return inner, present


@pytest.mark.parametrize("n,d,K,depth,P,T,B", [
    (3000, 8, 4, 5, 16, 15, 32),
    (12000, 20, 6, 6, 32, 10, 64),   # root and level-1 nodes take the chunked path
])
def test_tree_matches_oracle(ctx, n, d, K, depth, P, T, B):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(n, d, K, seed=d)
    gp = gpu_params(S, "gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=3)
    f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    g = f.export(0)
    op = oracle_params(O, "gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=3)
    r = O.train_tree(op, wl.X, wl.labels)
    inner, present = _compare_tree(g, r, d)
    assert np.array_equal(g["loss"][inner], r.loss[inner])
    assert np.array_equal(g["leaf_class"][present], r.leaf_class[present])
    cls, _, leaf = ctx.predict(f, wl.X, want_leaf=True)
    rc, _, rl = O.predict(op, r, wl.X)
    assert np.array_equal(cls, rc) and np.array_equal(leaf[:, 0], rl)
    Xt = W.gmm(2000, d, K, seed=d + 100).X
    assert np.array_equal(ctx.predict(f, Xt)[0], O.predict(op, r, Xt)[0])
    info = f.info()
    f.free()
    assert info["evaluations"] > 0


def _members(leaf, h):
    out = np.zeros(leaf.shape[0], bool)
    node = leaf.copy()
    while True:
        out |= node == h
        if (node <= h).all():
            break
        node = np.where(node > h, (node - 1) // 2, node)
    return np.nonzero(out)[0].astype(np.int32)


def _same_node(g, r, h):
    if g["kind"][h] != r.kind[h]:
        return False
    if r.kind[h] != 1:
        return True
    return (np.array_equal(g["dir"][h].astype(np.float64), r.dir[h]) and g["bin"][h] == r.bin[h]
            and g["zmin"][h] == np.float32(r.zmin[h]))


def _check_tree_up_to_near_ties(g, r, op, X, labels, y, tree_id=0):
    """Identical nodes, except below a node where the two searches part after
    a near-tie that the oracle logged (double sums in another order); tree_id:
    the tree's global id (node uids (tree_id << 16) | h)."""
    _, _, leaf = O.predict(op, r, X)
    H = len(r.kind)
    diverged = 0
    for h in range(H):
        anc, ok = h, True
        while anc > 0:
            anc = (anc - 1) // 2
            ok &= _same_node(g, r, anc)
        if not ok or r.kind[h] == -1 or _same_node(g, r, h):
            continue
        idx = _members(leaf, h)
        rs = O.node_split(op, X, labels, y, idx=idx, node_uid=(tree_id << 16) | h)
        assert rs.split["first_near_tie"] >= 0, f"node {h} differs without a near-tie"
        diverged += 1
    return diverged


def test_entropy_and_regression_trees(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(4000, 6, 3, seed=12)
    gp = gpu_params(S, "entropy", 3, 16, 10, 32, min_leaf=10, max_depth=4, seed=2)
    g = ctx.train_tree(gp, wl.X, labels=wl.labels).export(0)
    op = oracle_params(O, "entropy", 3, 16, 10, 32, min_leaf=10, max_depth=4, seed=2)
    r = O.train_tree(op, wl.X, wl.labels)
    _check_tree_up_to_near_ties(g, r, op, wl.X, wl.labels, None)
    for seed in (12, 13):
        wl = W.tanh_regression(4000, 6, seed=seed)
        gp = gpu_params(S, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=4, seed=2)
        f = ctx.train_tree(gp, wl.X, y=wl.y)
        g = f.export(0)
        op = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=4, seed=2)
        r = O.train_tree(op, wl.X, None, wl.y)
        diverged = _check_tree_up_to_near_ties(g, r, op, wl.X, None, wl.y)
        if diverged == 0:
            present = r.kind >= 0
            assert np.allclose(g["leaf_value"][present], r.leaf_value[present], rtol=1e-12,
                               atol=1e-12)
            _, val, _ = ctx.predict(f, wl.X)
            _, rv, _ = O.predict(op, r, wl.X)
            assert np.allclose(val, rv, rtol=1e-12, atol=1e-12)
        # every leaf predicts the mean target of its own samples
        _, val, leaf = ctx.predict(f, wl.X, want_leaf=True)
        for h in np.unique(leaf[:, 0]):
            m = leaf[:, 0] == h
            assert g["leaf_value"][h] == pytest.approx(wl.y[m].astype(np.float64).mean(),
                                                        rel=1e-9, abs=1e-12)


def test_bagged_forest_matches_oracle_trees(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(5000, 8, 5, seed=21)
    gp = gpu_params(S, "gini", 5, 16, 8, 32, min_leaf=10, max_depth=5, seed=8,
                    n_trees=4, bootstrap=True)
    f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    op = oracle_params(O, "gini", 5, 16, 8, 32, min_leaf=10, max_depth=5, seed=8)
    votes = np.zeros((wl.n, 5), np.int64)
    for t in range(4):
        r = O.train_tree(op, wl.X, wl.labels, tree_id=t, bootstrap=True)
        inner, present = _compare_tree(f.export(t), r, 8)
        votes[np.arange(wl.n), O.predict(op, r, wl.X)[0]] += 1
    cls, _, _ = ctx.predict(f, wl.X)
    assert np.array_equal(cls, np.argmax(votes, axis=1))


def test_grow_level_steps_match_train_tree(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(3000, 8, 4, seed=5)
    gp = gpu_params(S, "gini", 4, 16, 10, 32, min_leaf=10, max_depth=4, seed=6)
    f = ctx.forest_begin(gp, wl.X, labels=wl.labels)
    splits = []
    while True:
        k = f.grow_level()
        splits.append(k)
        if k == 0:
            break
    a = f.export(0)
    b = ctx.train_tree(gp, wl.X, labels=wl.labels).export(0)
    for key in a:
        assert np.array_equal(a[key], b[key]), key
    assert splits[0] == 1 and sum(splits) == int((a["kind"] == 1).sum())


# ------------------------------------------------ persistent node search -----

@pytest.mark.parametrize("crit,K,B,d,n,P,T", [
    ("entropy", 2, 64, 16, 2000, 32, 50),   # the single-node setting
    ("gini", 6, 128, 32, 700, 48, 15),
    ("gini", 3, 32, 8, 300, 20, 25),        # P not a multiple of 8
])
def test_persistent_node_search_matches_oracle(ctx, crit, K, B, d, n, P, T):
    """The whole search in one launch, the node resident in shared memory:
    trajectory and split of the fp32-mirror oracle."""
    from paper_2208_07023_gb300 import binding as S
    wl = W.single_node(n, d, seed=5) if K == 2 else W.gmm(n, d, K, seed=d)
    gp = gpu_params(S, crit, K, P, T, B, min_leaf=2, seed=41)
    ctx.set_node_search(True)
    try:
        g = ctx.node_split(gp, wl.X, labels=wl.labels, node_uid=9, want_trace=True)
        assert ctx.last_node_search() >= 1
    finally:
        ctx.set_node_search(False)
    r = O.node_split(oracle_params(O, crit, K, P, T, B, min_leaf=2, seed=41), wl.X,
                     wl.labels, node_uid=9)
    stop = r.split["first_near_tie"]
    upto = T + 1 if stop < 0 else stop
    assert np.array_equal(g["trace"][:upto], r.trace_loss[:upto])
    if stop < 0:
        assert np.array_equal(g["gbest"].astype(np.float64), r.gbest)
        assert (g["particle"], g["iter_of_best"], g["bin"]) == \
            (r.split["particle"], r.split["iter_of_best"], r.split["bin"])
        assert g["loss"] == r.split["loss"]


def test_persistent_node_search_tree_matches_oracle(ctx):
    from paper_2208_07023_gb300 import binding as S
    n, d, K, depth, P, T, B = 3000, 8, 4, 5, 16, 15, 32
    wl = W.gmm(n, d, K, seed=d)
    gp = gpu_params(S, "gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=3)
    ctx.set_node_search(True)
    try:
        f = ctx.train_tree(gp, wl.X, labels=wl.labels)
    finally:
        ctx.set_node_search(False)
    g = f.export(0)
    f.free()
    op = oracle_params(O, "gini", K, P, T, B, min_leaf=10, max_depth=depth, seed=3)
    r = O.train_tree(op, wl.X, wl.labels)
    inner, present = _compare_tree(g, r, d)
    assert np.array_equal(g["loss"][inner], r.loss[inner])
    assert np.array_equal(g["leaf_class"][present], r.leaf_class[present])
