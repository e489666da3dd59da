"""A forest split across processes (Sec. V, SLM Forest): growing trees
r, r + N, ... with slm_set_tree_ids(r, N) gives, tree for tree, the trees of
the whole forest grown at once (same bootstrap draws, same swarm streams),
here for N = 2 and 3 on one GPU; ids past 65535 are refused."""
import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("crit", ["gini", "entropy"])
def test_interleaved_parts_equal_the_whole_forest(crit):
    from paper_2208_07023_gb300 import binding as S
    ctx = context()
    wl = W.gmm(12000, 16, 5, seed=8)
    n_trees = 7
    p = gpu_params(S, crit, 5, 24, 6, 64, min_leaf=10, max_depth=5, seed=4, n_trees=n_trees,
                   bootstrap=True)
    whole = ctx.train_tree(p, wl.X, labels=wl.labels)
    ref = [whole.export(t) for t in range(n_trees)]
    whole.free()
    for world in (2, 3):
        for r in range(world):
            ids = list(range(r, n_trees, world))
            ctx.set_tree_ids(r, world)
            q = gpu_params(S, crit, 5, 24, 6, 64, min_leaf=10, max_depth=5, seed=4,
                           n_trees=len(ids), bootstrap=True)
            part = ctx.train_tree(q, wl.X, labels=wl.labels)
            for t, gid in enumerate(ids):
                got = part.export(t)
                for k in got:
                    assert np.array_equal(got[k], ref[gid][k]), (world, r, gid, k)
            part.free()
    ctx.set_tree_ids(65535, 1)
    q = gpu_params(S, crit, 5, 24, 6, 64, min_leaf=10, max_depth=5, seed=4, n_trees=2,
                   bootstrap=True)
    with pytest.raises(S.SlmError) as e:
        ctx.train_tree(q, wl.X, labels=wl.labels)
    assert e.value.status == S.SLM_EINVAL
    ctx.set_tree_ids()
    ctx.close()
