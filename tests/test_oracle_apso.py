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
* end to end: the planted hyperplane is found, the trajectory differs from
  plain PSO, and apso = 0 is plain PSO.
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
