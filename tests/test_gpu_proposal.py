"""GPU parity of the learned swarm proposal against the oracle, and what the
trained network gains.

* node statistics: FP32 partial sums (shifted by the node's first row) vs the
  oracle's double two-pass sums: within 1e-4 relative of the block's scale;
* network forward, loss and gradient (bfloat16 weights, FP32 accumulation vs
  the oracle in double with the same rounded weights): outputs within 1e-3,
  loss within 1e-4 relative, gradients within 1e-3 of each tensor's largest
  entry on all but a few entries (a ReLU whose input is within rounding of 0
  may switch) and cosine > 0.9999;
* first Adam step: w - lr sign(g) up to eps;
* seeded positions: bit-exact against the oracle (same stream, same
  correctly rounded operations);
* gain: after training on (statistics, PSO-best direction) pairs of
  single-node problems (planted hyperplane, d = 8..64), seeded searches of
  held-out nodes start from a lower loss and reach the plain search's final
  loss in fewer iterations (median).
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


def rand_net(seed):
    rng = np.random.default_rng(seed)
    m = {}
    for k, shp in O.MLP_SHAPES.items():
        if k.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1]))
            m[k] = rng.uniform(-lim, lim, shp).astype(np.float32)
        else:
            m[k] = (0.05 * rng.standard_normal(shp)).astype(np.float32)
    return m


def rand_batch(seed, n, dmax=60):
    rng = np.random.default_rng(seed)
    dims = rng.integers(3, dmax, n).astype(np.int32)
    s = np.zeros((n, O.MLP_IN), np.float32)
    a = np.zeros((n, O.MLP_D), np.float32)
    for r in range(n):
        d = dims[r]
        for k in list(range(rng.integers(2, 6))) + [O.MLP_K]:
            s[r, k * 256:k * 256 + d] = rng.standard_normal(d)
        v = rng.standard_normal(d)
        a[r, :d] = v / np.linalg.norm(v)
    return s, dims, a


@pytest.mark.parametrize("case", ["cls", "cls_weighted", "mse"])
def test_node_stats(ctx, case):
    if case == "mse":
        wl = W.tanh_regression(5000, 40, seed=3)
        idx, w = None, None
        g = ctx.node_stats(wl.X, y=wl.y)
        r = O.node_stats(wl.X, y=wl.y)
    else:
        wl = W.gmm(6000, 37, 7, seed=4)
        rng = np.random.default_rng(5)
        idx = rng.choice(6000, 3001, replace=False).astype(np.int32)
        w = rng.integers(1, 4, 3001).astype(np.uint32) if case == "cls_weighted" else None
        g = ctx.node_stats(wl.X, labels=wl.labels, n_classes=7, sample_idx=idx, weights=w)
        r = O.node_stats(wl.X, wl.labels, 7, idx=idx, wts=w)
    for k in range(21):
        gb, rb = g[k * 256:(k + 1) * 256], r[k * 256:(k + 1) * 256]
        scale = max(1e-6, np.abs(rb).max())
        assert np.max(np.abs(gb - rb)) <= 1e-4 * scale, k


def test_forward_matches_oracle(ctx):
    m = rand_net(1)
    prop = ctx.proposal(seed=3)
    try:
        prop.set(m)
        s, _, _ = rand_batch(2, 9)
        g = prop.forward(s)
        r, _, _ = O.mlp_forward({k: v.astype(np.float64) for k, v in m.items()}, s, bf16=True)
        assert np.max(np.abs(g - r)) <= 1e-3 * max(1.0, np.abs(r).max())
    finally:
        prop.free()


def test_loss_and_gradient_match_oracle(ctx):
    m = rand_net(4)
    prop = ctx.proposal(seed=3)
    try:
        prop.set(m)
        s, dims, a = rand_batch(5, 12)
        lg, gg = prop.loss_grad(s, dims, a)
        lr, gr = O.mlp_loss_grad({k: v.astype(np.float64) for k, v in m.items()}, s, dims, a,
                                 bf16=True)
        assert lg == pytest.approx(lr, rel=1e-4)
        for k in O.MLP_SHAPES:
            x, y = gg[k].astype(np.float64).ravel(), gr[k].ravel()
            scale = max(1e-12, np.abs(y).max())
            close = np.abs(x - y) <= 1e-3 * scale
            assert close.mean() >= 0.999, (k, close.mean())
            cos = x @ y / (np.linalg.norm(x) * np.linalg.norm(y) + 1e-30)
            assert cos > 0.9999, (k, cos)
    finally:
        prop.free()


def test_first_adam_step(ctx):
    m = rand_net(6)
    prop = ctx.proposal(seed=3)
    try:
        prop.set(m)
        s, dims, a = rand_batch(7, 8)
        _, g = prop.loss_grad(s, dims, a)
        prop.train(s, dims, a, epochs=1, batch=8, lr=1e-3, seed=1)
        after = prop.get()
        for k in O.MLP_SHAPES:
            big = np.abs(g[k]) > 1e-4
            step = (m[k] - after[k])[big]
            assert np.allclose(step, 1e-3 * np.sign(g[k][big]), rtol=1e-3, atol=1e-7), k
    finally:
        prop.free()


@pytest.mark.parametrize("P,d", [(64, 16), (33, 200), (5, 3)])
def test_seed_positions_bitwise(ctx, P, d):
    rng = np.random.default_rng(P + d)
    mu = rng.standard_normal(d).astype(np.float32)
    mu /= np.linalg.norm(mu)
    rho = rng.uniform(0, 2, P).astype(np.float32)
    g = ctx.swarm_seed(123456789, 70001, P, d, mu, rho)
    r = O.swarm_seed(123456789, 70001, P, d, mu, rho)
    assert np.array_equal(g.view(np.uint32), r.view(np.uint32))


def planted_node(seed, d):
    """The single-node pattern: isotropic features, labels by a planted
    hyperplane with 5 % flipped (the best direction is the class-mean
    difference, which the statistics carry)."""
    wl = W.single_node(1000, d, 0.05, seed=seed)
    return wl.X, wl.labels


def test_trained_proposal_gains(ctx):
    from paper_2208_07023_gb300 import binding as S
    P, T, B = 32, 40, 64
    base = dict(n_particles=P, n_iters=T, n_bins=B, min_leaf=5)
    # training pairs: statistics of a node and the direction plain PSO finds
    stats, dims, targets = [], [], []
    for i in range(1500):
        d = (8, 16, 32, 64)[i % 4]
        X, lab = planted_node(1000 + i, d)
        r = ctx.node_split(S.make_params("entropy", 2, seed=i + 1, **base), X, labels=lab,
                           node_uid=i)
        stats.append(ctx.node_stats(X, labels=lab, n_classes=2))
        t = np.zeros(256, np.float32)
        t[:d] = r["direction"]
        targets.append(t)
        dims.append(d)
    stats, dims, targets = np.array(stats), np.array(dims, np.int32), np.array(targets)
    prop = ctx.proposal(seed=11)
    try:
        losses = prop.train(stats, dims, targets, epochs=20, batch=64, lr=1e-3, seed=3)
        assert losses[-1] < 0.5 * losses[0]
        ctx.use_proposal(prop)
        first_plain, first_seed, it_plain, it_seed = [], [], [], []
        for i in range(32):
            d = (8, 16, 32, 64)[i % 4]
            X, lab = planted_node(90000 + i, d)
            plain = ctx.node_split(S.make_params("entropy", 2, seed=77 + i, **base), X,
                                   labels=lab, node_uid=i, want_trace=True)
            seeded = ctx.node_split(S.make_params("entropy", 2, seed=77 + i, seeded=True, **base),
                                    X, labels=lab, node_uid=i, want_trace=True)
            target = plain["trace"][-1]
            first_plain.append(plain["trace"][0])
            first_seed.append(seeded["trace"][0])
            it_plain.append(int(np.argmax(plain["trace"] <= target)))
            hit = np.nonzero(seeded["trace"] <= target)[0]
            it_seed.append(int(hit[0]) if hit.size else T + 1)
        assert np.median(first_seed) < np.median(first_plain)
        assert np.median(it_seed) < np.median(it_plain)
    finally:
        ctx.use_proposal(None)
        prop.free()
