"""Seeded synthetic inputs for SLM split search and tree training.

This module only draws input data (feature matrices, labels, targets). It holds
none of the method's arithmetic: no projection, binning, criterion or swarm
update lives here, so both the CUDA path and the CPU oracle can take their
inputs from it without sharing any of the computation they are compared on.

The paper's 15 benchmark datasets (Sec. V) are not used. Each workload below is
a synthetic stand-in with the sizes and structure of one evaluation setting:

* ``single_node``   n=2000, d=16, 2 classes labelled by the side of a random
                    hyperplane through the origin, 5 % of labels flipped.
* ``gmm``           K-class Gaussian mixture: uniform class priors, class
                    means ~ N(0, 2 I), one shared covariance Q diag(lam) Q^T
                    with Q Haar-random and lam log-uniform in [0.1, 10].
* ``tanh_regression`` X ~ N(0, I); y = sum_{j<8} tanh(w_j . x) + N(0, 0.1^2)
                    with w_j ~ N(0, I/d).

All draws use numpy's PCG64 generator seeded explicitly, so every platform
produces the same bytes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    X: np.ndarray                    # [n, d] float32, row-major
    labels: Optional[np.ndarray]     # [n] int32 in [0, K) (classification)
    y: Optional[np.ndarray]          # [n] float32 (regression)
    n_classes: int                   # 0 for regression
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])


def single_node(n: int = 2000, d: int = 16, flip: float = 0.05,
                seed: int = 1) -> Workload:
    """Two classes split by a random hyperplane through the origin.

    w is a random unit vector; label = [w . x >= 0], then each label is flipped
    independently with probability ``flip``. The Bayes direction is w.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x51A1]))
    w = rng.standard_normal(d)
    w /= np.linalg.norm(w)
    X = rng.standard_normal((n, d)).astype(np.float32)
    side = (X.astype(np.float64) @ w >= 0.0).astype(np.int32)
    flips = rng.random(n) < flip
    labels = np.where(flips, 1 - side, side).astype(np.int32)
    return Workload("single_node", np.ascontiguousarray(X), labels, None, 2,
                    {"w": w, "flip": flip, "seed": seed})


def haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian with sign fix."""
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def gmm(n: int, d: int, n_classes: int, seed: int = 1,
        mean_var: float = 2.0, lam_lo: float = 0.1,
        lam_hi: float = 10.0, sample_seed=None) -> Workload:
    """Gaussian mixture with a shared, randomly rotated covariance.

    `seed` draws the mixture (means, rotation, spectrum) and, by default, the
    samples too; a `sample_seed` draws the samples from a stream of their own,
    so that independent sample sets of one mixture can be drawn."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x6A11]))
    means = rng.normal(0.0, np.sqrt(mean_var), (n_classes, d))
    q = haar_orthogonal(rng, d)
    lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), d))
    if sample_seed is not None:
        rng = np.random.default_rng(np.random.SeedSequence([seed, sample_seed, 0x5A3]))
    labels = rng.integers(0, n_classes, n).astype(np.int32)
    z = rng.standard_normal((n, d))
    X = means[labels] + (z * np.sqrt(lam)[None, :]) @ q.T
    return Workload("gmm", np.ascontiguousarray(X.astype(np.float32)),
                    labels, None, n_classes,
                    {"means": means, "q": q, "lam": lam, "seed": seed})


def two_gaussians(n: int, d: int, seed: int = 1) -> Workload:
    """Two classes with a shared covariance: the LDA direction is
    Sigma^{-1} (mu_1 - mu_0)."""
    wl = gmm(n, d, 2, seed=seed)
    m = wl.meta
    sigma = (m["q"] * m["lam"][None, :]) @ m["q"].T
    lda = np.linalg.solve(sigma, m["means"][1] - m["means"][0])
    wl.meta["lda"] = lda / np.linalg.norm(lda)
    wl.meta["sigma"] = sigma
    wl.name = "two_gaussians"
    return wl


def tanh_regression(n: int, d: int, n_terms: int = 8, noise: float = 0.1,
                    seed: int = 1) -> Workload:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x7A9E]))
    W = rng.normal(0.0, 1.0 / np.sqrt(d), (n_terms, d))
    X = rng.standard_normal((n, d)).astype(np.float32)
    y = np.tanh(X.astype(np.float64) @ W.T).sum(axis=1)
    y = y + rng.normal(0.0, noise, n)
    return Workload("tanh_regression", np.ascontiguousarray(X), None,
                    y.astype(np.float32), 0, {"W": W, "seed": seed})


# --- named evaluation settings --------------------------------------------
# Each entry: workload builder + the PSO / tree hyper-parameters it runs with.
# omega=0.7, c1=c2=1.5 throughout; min_leaf=20 for the tree settings.

SETTINGS = {
    # one node, plain method
    "node_n2000_d16": dict(
        builder=lambda seed=1: single_node(2000, 16, 0.05, seed),
        criterion="entropy", n_particles=32, n_iters=50, n_bins=64,
        max_depth=1, min_leaf=1, n_trees=1),
    # the same node searched with 1024 independent seeds in one batch (1024
    # depth-1 trees without bootstrap: each root has its own swarm stream)
    "node_n2000_d16_x1024": dict(
        builder=lambda seed=1: single_node(2000, 16, 0.05, seed),
        criterion="entropy", n_particles=32, n_iters=50, n_bins=64,
        max_depth=1, min_leaf=1, n_trees=1024, bootstrap=False),
    # full classification tree, FP32 projection, all nodes of a level batched
    "tree_n50k_d64_k10": dict(
        builder=lambda seed=1: gmm(50_000, 64, 10, seed),
        criterion="gini", n_particles=64, n_iters=100, n_bins=128,
        max_depth=8, min_leaf=20, n_trees=1),
    # the classification tree with the per-node feature pre-screen: the swarm
    # searches the subspace of each node's 16 best features
    "tree_n50k_d64_k10_top16": dict(
        builder=lambda seed=1: gmm(50_000, 64, 10, seed),
        criterion="gini", n_particles=64, n_iters=100, n_bins=128,
        max_depth=8, min_leaf=20, n_trees=1, top_n=16),
    # regression tree
    "regtree_n200k_d128": dict(
        builder=lambda seed=1: tanh_regression(200_000, 128, 8, 0.1, seed),
        criterion="mse", n_particles=64, n_iters=80, n_bins=256,
        max_depth=10, min_leaf=20, n_trees=1, proj="bf16", topk=8),
    # learned proposal evaluated on a large mixture: PSO iterations to reach
    # the plain search's split loss over the nodes of the first four levels
    "proposal_n1m_d256_k20": dict(
        builder=lambda seed=1: gmm(1_000_000, 256, 20, seed),
        criterion="gini", n_particles=64, n_iters=80, n_bins=128,
        max_depth=12, min_leaf=20, n_trees=1, proj="bf16", topk=8),
    # SLR Boost: 10 rounds of depth-6 SLR trees fitted to the residuals of
    # the regression target, learning rate 0.3
    "boost_n200k_d128_r10": dict(
        builder=lambda seed=1: tanh_regression(200_000, 128, 8, 0.1, seed),
        criterion="mse", n_particles=64, n_iters=40, n_bins=256,
        max_depth=6, min_leaf=20, n_trees=1, rounds=10, lr=0.3),
    # SLM Boost: 5 rounds of 10 depth-4 SLR trees (one per class) fitted to
    # the softmax residuals of the classification mixture, learning rate 0.5
    "slmboost_n50k_d64_k10_r5": dict(
        builder=lambda seed=1: gmm(50_000, 64, 10, seed),
        criterion="mse", n_particles=64, n_iters=40, n_bins=128,
        max_depth=4, min_leaf=20, n_trees=1, rounds=5, lr=0.5, classes=10),
    # bagged forest of 64 trees; every level of all trees searched as one
    # graph-captured launch
    "forest64_n100k_d32_k5": dict(
        builder=lambda seed=1: gmm(100_000, 32, 5, seed),
        criterion="gini", n_particles=48, n_iters=60, n_bins=128,
        max_depth=8, min_leaf=20, n_trees=64, graphs=True),
}
