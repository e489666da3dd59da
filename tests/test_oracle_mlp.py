"""Pins for the oracle's learned swarm proposal: node statistics, the 3-layer
network, its loss gradient, Adam and the seeded initial swarm.

Each is checked against something other than itself: numpy's weighted means
and variances, numpy matrix products (with torch's bfloat16 rounding of the
weights), central finite differences in double, the straight-through reading
of the bfloat16 gradient (equal to the exact gradient at rounded weights),
Adam written out from its definition, and the seeded positions rebuilt from the
documented Philox stream.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")


def rand_net(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    m = {}
    for k, shp in O.MLP_SHAPES.items():
        if k.startswith("W"):
            lim = np.sqrt(6.0 / (shp[0] + shp[1])) * scale
            m[k] = rng.uniform(-lim, lim, shp).astype(np.float32).astype(np.float64)
        else:
            m[k] = (0.05 * rng.standard_normal(shp)).astype(np.float32).astype(np.float64)
    return m


def rand_inputs(seed, n, dmax=40):
    rng = np.random.default_rng(seed)
    dims = rng.integers(3, dmax, n).astype(np.int32)
    s = np.zeros((n, O.MLP_IN))
    a = np.zeros((n, O.MLP_D))
    for r in range(n):
        d = dims[r]
        for k in list(range(rng.integers(2, 6))) + [O.MLP_K]:
            s[r, k * O.MLP_D:k * O.MLP_D + d] = rng.standard_normal(d)
        v = rng.standard_normal(d)
        a[r, :d] = v / np.linalg.norm(v)
    return s, dims, a


def test_node_stats_against_numpy():
    rng = np.random.default_rng(1)
    n, d, K = 500, 11, 4
    X = rng.standard_normal((n, d)).astype(np.float32) * 3 + 1
    lab = rng.integers(0, K - 1, n).astype(np.int32)  # class K-1 absent
    idx = rng.choice(n, 300, replace=False).astype(np.int32)
    w = rng.integers(1, 5, 300).astype(np.uint32)
    s = O.node_stats(X, lab, K, idx=idx, wts=w)
    Xs = X[idx].astype(np.float64)
    mu = np.average(Xs, axis=0, weights=w)
    for k in range(K):
        sel = lab[idx] == k
        blk = s[k * 256:(k + 1) * 256]
        if sel.any():
            want = np.average(Xs[sel], axis=0, weights=w[sel]) - mu
            assert np.allclose(blk[:d], want, rtol=1e-12, atol=1e-12)
        else:
            assert not blk.any()
        assert not blk[d:].any()
    var = np.cov(Xs.T, aweights=w, bias=True).diagonal()
    assert np.allclose(s[20 * 256:20 * 256 + d], var, rtol=1e-10)
    assert not s[4 * 256:20 * 256].any() and not s[20 * 256 + d:].any()


def test_node_stats_regression_quarters():
    rng = np.random.default_rng(2)
    n, d = 400, 6
    X = rng.standard_normal((n, d)).astype(np.float32)
    y = rng.uniform(-2, 3, n).astype(np.float32)
    s = O.node_stats(X, y=y)
    lo, hi = y.min(), y.max()
    g = np.minimum(3, np.floor(np.float32(4) * ((y - lo) / np.float32(hi - lo))).astype(int))
    mu = X.astype(np.float64).mean(axis=0)
    for k in range(4):
        want = X[g == k].astype(np.float64).mean(axis=0) - mu
        assert np.allclose(s[k * 256:k * 256 + d], want, rtol=1e-12, atol=1e-12)
    assert not s[4 * 256:20 * 256].any()


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_is_three_dense_layers(bf16):
    m = rand_net(3)
    s, _, _ = rand_inputs(4, 5)
    out, h1, h2 = O.mlp_forward(m, s, bf16=bf16)
    W = {k: m[k] for k in m}
    if bf16:
        for k in ("W1", "W2", "W3"):
            W[k] = torch.from_numpy(m[k].astype(np.float32)).to(torch.bfloat16).double().numpy()
    r1 = np.maximum(s @ W["W1"] + W["b1"], 0)
    r2 = np.maximum(r1 @ W["W2"] + W["b2"], 0)
    r3 = r2 @ W["W3"] + W["b3"]
    assert np.allclose(h1, r1, rtol=1e-12, atol=1e-12)
    assert np.allclose(h2, r2, rtol=1e-12, atol=1e-12)
    assert np.allclose(out, r3, rtol=1e-12, atol=1e-12)


def loss_by_definition(o, dims, a):
    """The loss written out from its definition, per sample, in numpy."""
    P, D = O.MLP_P, O.MLP_D
    tot = 0.0
    for r in range(o.shape[0]):
        d = dims[r]
        mu, ar = o[r, :d], a[r, :d]
        c, mm = mu @ ar, mu @ mu
        ldir = 1 - c * c / (mm + 1e-12)
        delta = np.linalg.norm(mu / np.sqrt(mm) - np.sign(c if c != 0 else 1) * ar)
        rho = np.logaddexp(0, o[r, D:D + P])
        tau = (np.arange(P) + 0.5) / P
        u = delta - rho
        tot += ldir + np.mean(np.maximum(tau * u, (tau - 1) * u))
    return tot / o.shape[0]


def test_loss_value_by_definition():
    m = rand_net(5)
    s, dims, a = rand_inputs(6, 7)
    loss, _ = O.mlp_loss_grad(m, s, dims, a, bf16=False)
    out, _, _ = O.mlp_forward(m, s, bf16=False)
    assert loss == pytest.approx(loss_by_definition(out, dims, a), rel=1e-12)


def test_gradient_matches_finite_differences():
    m = rand_net(7)
    s, dims, a = rand_inputs(8, 3)
    _, g = O.mlp_loss_grad(m, s, dims, a, bf16=False)
    rng = np.random.default_rng(9)
    h = 1e-6
    for k in O.MLP_SHAPES:
        flat = m[k].reshape(-1)
        gk = g[k].reshape(-1)
        # entries with a non-zero gradient, plus random ones
        cand = np.flatnonzero(np.abs(gk) > 1e-6)
        picks = np.concatenate([rng.choice(cand, min(6, cand.size), replace=False),
                                rng.integers(0, flat.size, 3)])
        for i in picks:
            old = flat[i]
            flat[i] = old + h
            lp, _ = O.mlp_loss_grad(m, s, dims, a, bf16=False)
            flat[i] = old - h
            lm, _ = O.mlp_loss_grad(m, s, dims, a, bf16=False)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gk[i]) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, gk[i])


def test_bf16_gradient_is_the_gradient_at_rounded_weights():
    m = rand_net(10)
    s, dims, a = rand_inputs(11, 3)
    lq, gq = O.mlp_loss_grad(m, s, dims, a, bf16=True)
    mr = dict(m)
    for k in ("W1", "W2", "W3"):
        mr[k] = O.bf16_round(m[k].astype(np.float32)).astype(np.float64)
    lr_, gr = O.mlp_loss_grad(mr, s, dims, a, bf16=False)
    assert lq == lr_
    for k in O.MLP_SHAPES:
        assert np.array_equal(gq[k], gr[k])


def test_adam_by_definition_and_convergence():
    rng = np.random.default_rng(12)
    w = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    g = rng.standard_normal(50)
    w2, m2, v2 = O.adam_step(w.copy(), m.copy(), v.copy(), g, 1, lr=0.01)
    mm = 0.1 * g
    vv = 0.001 * g * g
    want = w - 0.01 * (mm / 0.1) / (np.sqrt(vv / 0.001) + 1e-8)
    assert np.allclose(w2, want, rtol=1e-14) and np.allclose(m2, mm) and np.allclose(v2, vv)
    # minimises a quadratic
    c = rng.standard_normal(50)
    w = np.zeros(50); m = np.zeros(50); v = np.zeros(50)
    for t in range(1, 3001):
        w, m, v = O.adam_step(w, m, v, 2 * (w - c), t, lr=0.01)
    assert np.max(np.abs(w - c)) < 1e-3


def test_adam_training_lowers_the_loss():
    m = rand_net(13)
    s, dims, a = rand_inputs(14, 6)
    state = {k: (np.zeros_like(m[k]), np.zeros_like(m[k])) for k in m}
    l0, _ = O.mlp_loss_grad(m, s, dims, a)
    for t in range(1, 31):
        _, g = O.mlp_loss_grad(m, s, dims, a)
        for k in m:
            w, mm, vv = O.adam_step(m[k], state[k][0], state[k][1], g[k], t, lr=1e-3)
            m[k], state[k] = w, (mm, vv)
    l1, _ = O.mlp_loss_grad(m, s, dims, a)
    assert l1 < 0.7 * l0


def test_swarm_seed_rebuilt_from_the_stream():
    P, d = 12, 9
    rng = np.random.default_rng(15)
    mu = rng.standard_normal(d).astype(np.float32)
    rho = rng.uniform(0, 1, P).astype(np.float32)
    pos = O.swarm_seed(77, 5, P, d, mu, rho)
    u = O.swarm_uniforms(77, 5, 0, P, d, O.PURPOSE_SEED)
    u = (np.float32(2) * u - np.float32(1)).astype(np.float32)
    sigma = np.sqrt(d / 3.0)  # expected norm of a uniform start in [-1, 1)^d
    u_plain = O.swarm_uniforms(77, 5, 0, 4000, d, O.PURPOSE_INIT_X) * 2 - 1
    assert np.linalg.norm(u_plain, axis=1).mean() == pytest.approx(sigma, rel=0.03)
    for i in range(P):
        nrm = np.float32(np.sqrt((u[i].astype(np.float64) ** 2).sum()))
        want = (sigma * (mu + rho[i] * (u[i] / nrm))).astype(np.float32)
        assert np.allclose(pos[i], want, rtol=2e-6, atol=2e-6)
        assert np.linalg.norm(pos[i].astype(np.float64) / sigma - mu) == pytest.approx(
            rho[i], rel=1e-5)
