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
