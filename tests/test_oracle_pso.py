"""Pins for the oracle's swarm update (Eq. pso-1) and search (Algorithm 1)."""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W


@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
def test_single_update_by_hand(precision):
    # omega=0.5, c1=2, c2=4; x=0.5, v=0.25, pB=1, gB=-1, r1=0.5, r2=0.25:
    # v' = 0.5*0.25 + 2*0.5*(1-0.5) + 4*0.25*(-1-0.5) = 0.125 + 0.5 - 1.5 = -0.875
    # x' = x + v' = -0.375   (all values exact in binary)
    p = O.make_params(inertia=0.5, c1=2.0, c2=4.0, precision=precision)
    x, v = O.pso_step(p, [[0.5]], [[0.25]], [[1.0]], [-1.0], [[0.5]], [[0.25]])
    assert v[0, 0] == -0.875 and x[0, 0] == -0.375
    # at pB = gB = x only inertia acts
    x, v = O.pso_step(p, [[2.0, -4.0]], [[1.0, 8.0]], [[2.0, -4.0]], [2.0, -4.0],
                      [[0.3, 0.9]], [[0.7, 0.1]])
    assert v.tolist() == [[0.5, 4.0]] and x.tolist() == [[2.5, 0.0]]


def test_update_converges_on_sphere():
    """The update rule alone (no SLM loss) must drive a swarm to the minimum
    of f(x) = ||x - c||^2: a sign or index slip in any term makes it wander."""
    rng = np.random.default_rng(0)
    P, d, T = 24, 4, 300
    c = np.array([0.3, -0.6, 0.1, 0.8])
    p = O.make_params(inertia=0.7, c1=1.5, c2=1.5, precision=O.F64)
    # the textbook-stable setting omega=0.7, c1=c2=1.5 converges
    x = rng.uniform(-1, 1, (P, d))
    v = 0.1 * rng.uniform(-1, 1, (P, d))
    f = lambda z: ((z - c) ** 2).sum(axis=1)
    pb, pf = x.copy(), f(x)
    g = pb[np.argmin(pf)].copy()
    for t in range(1, T + 1):
        r1 = O.swarm_uniforms(5, 0, t, P, d, O.PURPOSE_R1).astype(np.float64)
        r2 = O.swarm_uniforms(5, 0, t, P, d, O.PURPOSE_R2).astype(np.float64)
        x, v = O.pso_step(p, x, v, pb, g, r1, r2)
        fx = f(x)
        imp = fx < pf
        pb[imp], pf[imp] = x[imp], fx[imp]
        g = pb[np.argmin(pf)].copy()
    assert np.linalg.norm(g - c) < 1e-4


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_recovers_planted_hyperplane(seed):
    """Labels = side of w . x = 0 with 5 % flips: the Bayes direction is w and
    the best attainable weighted entropy is near H(0.05) = 0.1985 nats."""
    wl = W.single_node(seed=seed)
    p = O.make_params("entropy", 2, 32, 50, 64, min_leaf=1, precision=O.F64)
    r = O.node_split(p, wl.X, wl.labels)
    assert abs(r.direction @ wl.meta["w"]) >= 0.99
    assert np.linalg.norm(r.direction) == pytest.approx(1.0, abs=1e-12)
    assert 0.15 < r.split["loss"] < 0.30
    h = -(0.05 * np.log(0.05) + 0.95 * np.log(0.95))
    assert r.split["loss"] > h - 0.05


def test_recovers_lda_direction():
    """Two Gaussians with a shared covariance: the Bayes boundary is normal to
    Sigma^{-1}(mu1 - mu0)."""
    wl = W.two_gaussians(20_000, 4, seed=3)
    p = O.make_params("gini", 2, 32, 60, 128, min_leaf=1, precision=O.F64)
    r = O.node_split(p, wl.X, wl.labels)
    assert abs(r.direction @ wl.meta["lda"]) > 0.999


def test_matches_angle_sweep_in_2d():
    """In d=2 every direction is an angle: a dense sweep lower-bounds the loss
    any direction can reach, and PSO must come within 1e-3 of it."""
    wl = W.gmm(3000, 2, 3, seed=4)
    p = O.make_params("gini", 3, 24, 60, 64, min_leaf=5, precision=O.F64)
    r = O.node_split(p, wl.X, wl.labels)
    th = np.linspace(0.0, np.pi, 20_000, endpoint=False)
    pos = np.stack([np.cos(th), np.sin(th)], axis=1)
    sweep = min(e["loss"] for e in O.eval_swarm(p, wl.X, wl.labels, None, pos)[0])
    assert r.split["loss"] <= sweep + 1e-3


@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
def test_trace_and_result_consistency(precision):
    wl = W.gmm(2000, 8, 4, seed=6)
    p = O.make_params("gini", 4, 16, 30, 32, min_leaf=5, precision=precision)
    r = O.node_split(p, wl.X, wl.labels, node_uid=12345)
    tl = r.trace_loss
    assert np.all(np.diff(tl) <= 0.0)            # gbest never gets worse
    it = r.split["iter_of_best"]
    assert tl[it] == r.split["loss"] and (it == 0 or tl[it - 1] > tl[it])
    # re-scoring the returned gbest reproduces the reported split exactly
    e = O.eval_swarm(p, wl.X, wl.labels, None, r.gbest[None, :])[0][0]
    for k in ("loss", "bin", "zmin", "inv_w", "n_left", "n_right", "q_num", "q_den"):
        assert e[k] == r.split[k]
    # the search is deterministic in (seed, node uid) and changes with either
    assert O.node_split(p, wl.X, wl.labels, node_uid=12345).split == r.split
    r2 = O.node_split(p, wl.X, wl.labels, node_uid=12346)
    assert not np.array_equal(r2.gbest, r.gbest)


def test_zero_iterations_scores_initial_swarm():
    wl = W.gmm(500, 4, 2, seed=8)
    p = O.make_params("gini", 2, 10, 0, 16, precision=O.F32_MIRROR)
    r = O.node_split(p, wl.X, wl.labels, node_uid=9)
    u = O.swarm_uniforms(p.seed, 9, 0, 10, 4, O.PURPOSE_INIT_X)
    x0 = (2.0 * u - 1.0).astype(np.float64)
    ev = O.eval_swarm(p, wl.X, wl.labels, None, x0)[0]
    best = min(range(10), key=lambda i: (-ev[i]["q_num"] / ev[i]["q_den"], i))
    assert r.split["particle"] == best and np.array_equal(r.gbest, x0[best])


@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
def test_one_iteration_follows_documented_streams(precision):
    """T=1 by hand: x0 = 2u-1 (purpose INIT_X), v0 = 0.1(2u-1) (INIT_V), score,
    pbest = x0, gbest = best; then r1 (R1), r2 (R2) at t=1, one synchronous
    update, score, strict-< bests. The oracle's search must agree."""
    wl = W.gmm(800, 5, 3, seed=10)
    P, d, uid = 12, 5, 4242
    p = O.make_params("gini", 3, P, 1, 32, min_leaf=3, precision=precision)
    r = O.node_split(p, wl.X, wl.labels, node_uid=uid)

    def key(e):
        return (0, -e["q_num"] / e["q_den"]) if e["valid"] else (1, 0.0)

    x = (2.0 * O.swarm_uniforms(p.seed, uid, 0, P, d, O.PURPOSE_INIT_X) - 1.0).astype(np.float64)
    u = (2.0 * O.swarm_uniforms(p.seed, uid, 0, P, d, O.PURPOSE_INIT_V) - 1.0)
    v = (np.float32(0.1) * u).astype(np.float64) if precision == O.F32_MIRROR else 0.1 * u.astype(np.float64)
    ev = O.eval_swarm(p, wl.X, wl.labels, None, x)[0]
    pb, pe = x.copy(), list(ev)
    g = min(range(P), key=lambda i: (key(ev[i]), i))
    gb, ge = x[g].copy(), ev[g]
    r1 = O.swarm_uniforms(p.seed, uid, 1, P, d, O.PURPOSE_R1).astype(np.float64)
    r2 = O.swarm_uniforms(p.seed, uid, 1, P, d, O.PURPOSE_R2).astype(np.float64)
    x, v = O.pso_step(p, x, v, pb, gb, r1, r2)
    ev = O.eval_swarm(p, wl.X, wl.labels, None, x)[0]
    for i in range(P):
        if ev[i]["valid"] and (not pe[i]["valid"] or
                               ev[i]["q_num"] * pe[i]["q_den"] > pe[i]["q_num"] * ev[i]["q_den"]):
            pe[i] = ev[i]
            if not ge["valid"] or ev[i]["q_num"] * ge["q_den"] > ge["q_num"] * ev[i]["q_den"]:
                gb, ge, g = x[i].copy(), ev[i], i
    assert np.array_equal(r.gbest, gb)
    assert r.split["particle"] == g and r.split["loss"] == ge["loss"]


def test_search_from_given_start_equals_search_from_its_own_draws():
    """A search started from the positions the uniform draws give is the
    plain search; a different start changes the trajectory."""
    import oracle as O
    from paper_2208_07023_gb300 import workloads as W
    wl = W.gmm(800, 6, 3, seed=4)
    p = O.make_params("gini", 3, n_particles=12, n_iters=8, n_bins=32, min_leaf=3,
                      precision=O.F32_MIRROR, seed=5)
    u = O.swarm_uniforms(5, 7, 0, 12, 6, 1)
    x0 = (2.0 * u - 1.0).astype(np.float32)
    a = O.node_split(p, wl.X, wl.labels, node_uid=7)
    b = O.node_split_from(p, wl.X, x0, wl.labels, node_uid=7)
    assert np.array_equal(a.trace_loss, b.trace_loss) and np.array_equal(a.gbest, b.gbest)
    c = O.node_split_from(p, wl.X, -x0, wl.labels, node_uid=7)
    assert not np.array_equal(c.gbest, a.gbest)
