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
