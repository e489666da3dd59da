"""Shared helpers of the GPU parity tests."""
import numpy as np
import pytest


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def context():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2208_07023_gb300 import binding
    return binding.Context(0)


def oracle_params(O, crit, K, P, T, B, min_leaf=1, seed=1, max_depth=8,
                  precision=None):
    return O.make_params(crit, K, P, T, B, min_leaf=min_leaf, seed=seed,
                         max_depth=max_depth,
                         precision=O.F32_MIRROR if precision is None else precision)


def gpu_params(S, crit, K, P, T, B, min_leaf=1, seed=1, max_depth=8, n_trees=1,
               bootstrap=False):
    return S.make_params(crit, K, n_particles=P, n_iters=T, n_bins=B,
                         min_leaf=min_leaf, seed=seed, max_depth=max_depth,
                         n_trees=n_trees, bootstrap=bootstrap)


def edge_distance(z, zmin, zmax, B):
    """Distance of each z to the nearest interior bin edge (fp64)."""
    edges = zmin + (zmax - zmin) * np.arange(1, B) / B
    return np.min(np.abs(z[:, None] - edges[None, :]), axis=1)
