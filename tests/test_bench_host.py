"""Host-side arithmetic of the benchmark: the tree loss it reports."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_leaf_gini_against_a_loop():
    import bench
    rng = np.random.default_rng(3)
    n, K = 5000, 7
    leaf = rng.integers(0, 40, n) * 3 + 1  # sparse heap indices
    labels = rng.integers(0, K, n).astype(np.int32)
    want = 0.0
    for h in np.unique(leaf):
        c = np.bincount(labels[leaf == h], minlength=K).astype(np.float64)
        want += c.sum() * (1.0 - ((c / c.sum()) ** 2).sum())
    assert bench.leaf_gini(leaf, labels, K) == np.float64(want / n).item() or \
        abs(bench.leaf_gini(leaf, labels, K) - want / n) < 1e-12


def test_leaf_gini_special_cases():
    import bench
    labels = np.array([0, 0, 1, 1], np.int32)
    assert bench.leaf_gini(np.array([0, 0, 0, 0]), labels, 2) == 0.5
    assert bench.leaf_gini(np.array([1, 1, 2, 2]), labels, 2) == 0.0


def test_oracle_targets_of_boosting_workloads():
    # a boosting run's first root search fits residuals: y minus its mean, or
    # class 0's one-hot minus 1/K; other workloads search the targets as given
    import bench
    from paper_2208_07023_gb300 import workloads as W

    class WL:
        pass
    rng = np.random.default_rng(1)
    w = WL()
    w.y, w.labels, w.n_classes = rng.standard_normal(100).astype(np.float32), None, 0
    lab, y = bench.oracle_targets({"rounds": 3}, w)
    assert lab is None and abs(float(np.mean(y.astype(np.float64)))) < 1e-6
    assert np.allclose(y, w.y - np.float32(np.mean(w.y.astype(np.float64))), atol=1e-6)
    w2 = WL()
    w2.y, w2.labels, w2.n_classes = None, rng.integers(0, 4, 100).astype(np.int32), 4
    lab, y = bench.oracle_targets({"rounds": 3}, w2)
    assert lab is None and set(np.unique(y).tolist()) <= {np.float32(0.75), np.float32(-0.25)}
    assert np.array_equal(y > 0, w2.labels == 0)
    assert bench.oracle_targets({}, w2) == (w2.labels, None)
    # every boosting workload names its rounds and learning rate
    for name, cfg in W.SETTINGS.items():
        if cfg.get("rounds"):
            assert cfg["criterion"] == "mse" and 0 < cfg["lr"] <= 1 and cfg["n_trees"] == 1


def test_clock_sampler_keeps_the_marked_region():
    import datetime

    import bench
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(ms, mhz, power_cap="Not Active", thermal="Not Active"):
        ts = (base + datetime.timedelta(milliseconds=ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.0, 0x0, Not Active, Not Active, {thermal}, {power_cap}"

    s = bench.ClockSampler("GPU-x")
    s.out = "\n".join([line(0, 1000, thermal="Active"), line(50, 2070), line(100, 2040),
                       line(150, 2070, power_cap="Active"), line(200, 900)])
    t = base.timestamp()
    s.t0, s.t1 = t + 0.04, t + 0.16  # samples at 50, 100, 150 ms fall inside
    r = s.summary()
    assert r["samples"] == 3 and r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]  # the thermal sample lies outside
    s.t0, s.t1 = t + 0.060, t + 0.070  # shorter than a period: within the slack
    assert s.summary()["samples"] == 1
    s.t0, s.t1 = t + 1.0, t + 1.1  # no sample near: the closest one, flagged
    r = s.summary()
    assert r["samples"] == 1 and r["sm_mhz"] == 900 and r["nearest_sample_outside_region"]
