"""Pins for the oracle's adaptive PSO (Sec. III-B; the published rules of the
cited APSO method).

* the evolutionary factor against closed forms: three particles on a line at
  0, a, 1 have mean distances (1 + a)/2, 1/2, (2 - a)/2, so the particle at
  0 gives f = a / (1 - a) (a < 1/2), the one at a gives 0, the one at 1 gives
  1; four particles at 0, 1, 2, 10 give f = 1/8 for the first;
* the state of hand-chosen f values, away from and inside the overlaps of
  the membership functions, against the ring rule for every previous state;
* the learning-factor steps, clamping and normalisation, and the inertia's
  end values 1 / 2.5 and 1 / (1 + 1.5 e^-2.6);
* elitist learning: the candidate differs from gB in exactly one coordinate,
  whose index is uniform over the features (chi-square) and whose step is
  Gaussian (Kolmogorov-Smirnov) with a standard deviation falling linearly
  from 2 (the initial range's width) to 0.2 over the search; the acceptance
  rule on hand-built swarms: a strictly better candidate becomes gB and the
  gB particle's personal best, a tie or worse one replaces the worst particle
  (invalid counts as worst, ties to the lower index) and its personal best
  only when better;
* end to end: the planted hyperplane is found, the trajectory differs from
  plain PSO, apso = 0 is plain PSO, and elite candidates are scored in the
  convergence state, some of them accepted.
"""
import numpy as np
import pytest

import oracle as O

EXP, EXT, CON, JMP = O.APSO_EXPLORE, O.APSO_EXPLOIT, O.APSO_CONVERGE, O.APSO_JUMPOUT


def line(*xs):
    return np.array(xs, dtype=np.float64)[:, None]


@pytest.mark.parametrize("a", [0.1, 0.2, 1 / 3, 0.4])
def test_evolutionary_factor_closed_form(a):
    x = line(0.0, a, 1.0)
    r = O.apso_step(x, 0, EXP, 2.0, 2.0, 0.05)
    assert r["f"] == pytest.approx(a / (1 - a), rel=1e-6)
    assert O.apso_step(x, 1, EXP, 2.0, 2.0, 0.05)["f"] == 0.0
    assert O.apso_step(x, 2, EXP, 2.0, 2.0, 0.05)["f"] == 1.0


def test_evolutionary_factor_four_points_and_distances_in_d():
    assert O.apso_step(line(0, 1, 2, 10), 0, EXP, 2.0, 2.0, 0.05)["f"] == pytest.approx(0.125)
    # the same configuration rotated into 3 dimensions: distances unchanged
    rng = np.random.default_rng(1)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    x = np.zeros((4, 3))
    x[:, 0] = [0, 1, 2, 10]
    assert O.apso_step(x @ q.T, 0, EXP, 2.0, 2.0, 0.05)["f"] == pytest.approx(0.125, rel=1e-5)


def f_config(f):
    """Three particles whose first particle has evolutionary factor f."""
    a = f / (1 + f)
    return line(0.0, a, 1.0)


# (f, previous state) -> state, from the membership functions: convergence on
# [0, 0.3), exploitation on (0.2, 0.6), exploration on (0.4, 0.8),
# jumping out on (0.7, 1]; overlaps resolved by keeping the previous state,
# else the next in the ring 1 -> 2 -> 3 -> 4 -> 1, else the larger membership
CASES = [
    (0.05, EXP, CON), (0.05, JMP, CON), (0.35, CON, EXT), (0.65, CON, EXP), (0.95, EXT, JMP),
    (0.25, EXT, EXT), (0.25, CON, CON), (0.25, EXP, EXT), (0.25, JMP, EXT),
    (0.5, EXP, EXP), (0.5, EXT, EXT), (0.5, JMP, EXP), (0.45, CON, EXT), (0.55, CON, EXP),
    (0.75, EXP, EXP), (0.75, JMP, JMP), (0.75, CON, JMP), (0.75, EXT, EXP),
]


@pytest.mark.parametrize("f,prev,want", CASES)
def test_state_rule(f, prev, want):
    r = O.apso_step(f_config(f), 0, prev, 2.0, 2.0, 0.08)
    assert r["f"] == pytest.approx(f, rel=1e-5)
    assert r["state"] == want


def test_learning_factor_steps():
    # exploration at f = 0.65 (from convergence: no overlap)
    r = O.apso_step(f_config(0.65), 0, CON, 2.0, 2.0, 0.1)
    assert (r["c1"], r["c2"]) == pytest.approx((2.1, 1.9), abs=1e-6)
    r = O.apso_step(f_config(0.35), 0, CON, 2.0, 2.0, 0.1)   # exploitation
    assert (r["c1"], r["c2"]) == pytest.approx((2.05, 1.95), abs=1e-6)
    r = O.apso_step(f_config(0.05), 0, EXP, 1.8, 1.9, 0.1)   # convergence
    assert (r["c1"], r["c2"]) == pytest.approx((1.85, 1.95), abs=1e-6)
    r = O.apso_step(f_config(0.95), 0, EXP, 2.0, 2.0, 0.1)   # jumping out
    assert (r["c1"], r["c2"]) == pytest.approx((1.9, 2.1), abs=1e-6)
    # clamped to [1.5, 2.5]
    r = O.apso_step(f_config(0.65), 0, CON, 2.45, 1.55, 0.1)
    assert (r["c1"], r["c2"]) == (2.5, 1.5)
    # normalised to a sum of 4
    r = O.apso_step(f_config(0.05), 0, EXP, 2.4, 2.0, 0.1)
    assert (r["c1"], r["c2"]) == pytest.approx((4 * 2.45 / 4.5, 4 * 2.05 / 4.5), abs=1e-6)
    assert r["c1"] + r["c2"] == pytest.approx(4.0, abs=1e-6)


def test_inertia_end_values():
    assert O.apso_step(line(0.0, 0.3, 1.0), 1, EXP, 2.0, 2.0, 0.05)["w"] == \
        pytest.approx(1 / 2.5, rel=1e-7)
    assert O.apso_step(line(0.0, 0.3, 1.0), 2, EXP, 2.0, 2.0, 0.05)["w"] == \
        pytest.approx(1 / (1 + 1.5 * np.exp(-2.6)), rel=1e-7)


def test_apso_search_end_to_end():
    rng = np.random.default_rng(2)
    n, d = 3000, 8
    X = rng.standard_normal((n, d)).astype(np.float32)
    w = rng.standard_normal(d)
    w /= np.linalg.norm(w)
    labels = (X.astype(np.float64) @ w >= 0).astype(np.int32)
    labels[rng.random(n) < 0.05] ^= 1
    pa = O.make_params("entropy", 2, 32, 50, 64, min_leaf=1, apso=True)
    pp = O.make_params("entropy", 2, 32, 50, 64, min_leaf=1)
    a = O.node_split(pa, X, labels)
    b = O.node_split(pp, X, labels)
    assert abs(a.direction @ w) > 0.99
    assert not np.array_equal(a.trace_loss, b.trace_loss)
    assert a.trace_loss[0] == b.trace_loss[0]  # the same initial swarm
    assert a.split["loss"] < 0.24
    c = O.node_split(O.make_params("entropy", 2, 32, 50, 64, min_leaf=1, apso=False), X, labels)
    assert np.array_equal(c.trace_loss, b.trace_loss)


def test_elite_candidate_moves_one_coordinate():
    rng = np.random.default_rng(3)
    gb = rng.standard_normal(12)
    for uid in range(50):
        e, k = O.elite_candidate(9, uid, 4, 20, gb)
        diff = np.flatnonzero(e != gb)
        assert 0 <= k < 12 and set(diff.tolist()) <= {k}
        assert np.array_equal(np.delete(e, k), np.delete(gb, k))


def test_elite_candidate_index_is_uniform():
    from scipy import stats
    d = 10
    ks = [O.elite_candidate(5, uid, 0, 10, np.zeros(d))[1] for uid in range(5000)]
    counts = np.bincount(ks, minlength=d)
    assert stats.chisquare(counts).pvalue > 1e-3


@pytest.mark.parametrize("t,T,sd", [(0, 10, 2.0), (5, 10, 2.0 * 0.55), (9, 9, 0.2)])
def test_elite_step_is_gaussian_with_linear_schedule(t, T, sd):
    from scipy import stats
    steps = []
    for uid in range(4000):
        e, k = O.elite_candidate(7, uid, t, T, np.zeros(4))
        steps.append(e[k])
    steps = np.array(steps)
    assert stats.kstest(steps / sd, "norm").pvalue > 1e-3
    assert np.std(steps) == pytest.approx(sd, rel=0.05)
    # the float-mode candidate is rounded once per operation, as float
    assert np.array_equal(steps, steps.astype(np.float32).astype(np.float64))


def swarm(P=5, d=3):
    x = np.arange(P * d, dtype=np.float64).reshape(P, d)
    pb = x + 100.0
    return x, pb


def test_elite_better_becomes_gbest_and_gbest_particles_pbest():
    x, pb = swarm()
    cur = np.array([0.5, 0.3, 0.9, 0.2, 0.4])
    pbl = np.array([0.4, 0.3, 0.8, 0.2, 0.4])
    gb = pb[3].copy()
    el = np.array([-1.0, -2.0, -3.0])
    r = O.elite_apply(x, pb, cur, pbl, 0.2, 3, gb, el, 0.1)
    assert r["accepted"] and r["g_loss"] == 0.1
    assert np.array_equal(r["gb"], el) and np.array_equal(r["pb"][3], el)
    assert r["pb_loss"][3] == 0.1
    assert np.array_equal(r["x"], x) and np.array_equal(r["cur_loss"], cur)
    assert np.array_equal(np.delete(r["pb"], 3, axis=0), np.delete(pb, 3, axis=0))


@pytest.mark.parametrize("e_loss,pb_replaced", [(0.2, True), (0.5, True), (0.8, False), (0.85, False)])
def test_elite_not_better_replaces_the_worst_particle(e_loss, pb_replaced):
    x, pb = swarm()
    cur = np.array([0.5, 0.3, 0.9, 0.2, 0.4])
    pbl = np.array([0.4, 0.3, 0.8, 0.2, 0.4])
    gb = pb[3].copy()
    el = np.array([-1.0, -2.0, -3.0])
    r = O.elite_apply(x, pb, cur, pbl, 0.2, 3, gb, el, e_loss)
    assert not r["accepted"] and r["worst"] == 2 and r["g_loss"] == 0.2
    assert np.array_equal(r["x"][2], el) and r["cur_loss"][2] == e_loss
    assert np.array_equal(np.delete(r["x"], 2, axis=0), np.delete(x, 2, axis=0))
    assert np.array_equal(r["gb"], gb)
    assert np.array_equal(r["pb"][2], el if pb_replaced else pb[2])
    assert r["pb_loss"][2] == (e_loss if pb_replaced else 0.8)


def test_elite_worst_ties_and_invalid():
    x, pb = swarm(4, 2)
    el = np.array([7.0, 8.0])
    # equal worst losses: the lower index
    r = O.elite_apply(x, pb, np.array([0.6, 0.1, 0.6, 0.3]), np.full(4, 0.1), 0.1, 1,
                      pb[1].copy(), el, 0.7)
    assert r["worst"] == 0
    # an invalid particle is the worst; an invalid candidate never becomes a pbest
    r = O.elite_apply(x, pb, np.array([0.6, 0.1, np.inf, 0.3]), np.full(4, np.inf), 0.1, 1,
                      pb[1].copy(), el, np.inf)
    assert r["worst"] == 2 and not r["accepted"]
    assert np.array_equal(r["x"][2], el) and np.array_equal(r["pb"][2], pb[2])


def test_elite_learning_runs_in_the_search():
    rng = np.random.default_rng(2)
    n, d = 3000, 8
    X = rng.standard_normal((n, d)).astype(np.float32)
    w = rng.standard_normal(d)
    w /= np.linalg.norm(w)
    labels = (X.astype(np.float64) @ w >= 0).astype(np.int32)
    labels[rng.random(n) < 0.05] ^= 1
    tries = accepts = 0
    for seed in range(1, 6):
        r = O.node_split(O.make_params("gini", 2, 32, 50, 64, min_leaf=1, apso=True, seed=seed),
                         X, labels)
        assert abs(r.direction @ w) > 0.99
        assert np.all(np.diff(r.trace_loss) <= 0)
        tries += r.split["elite_tries"]
        accepts += r.split["elite_accepts"]
        plain = O.node_split(O.make_params("gini", 2, 32, 50, 64, min_leaf=1, seed=seed),
                             X, labels)
        assert plain.split["elite_tries"] == 0
    assert tries > 0 and 0 < accepts < tries
