"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2).

Trees are independent units: every rank grows its own trees on its own data
and the ranks meet only to report, so the job's throughput is the evaluations
of all ranks over the time of the slowest one. These tests run two gloo ranks
as processes and check that reduction, that the ranks' workloads differ, and
that the reference arm's extra ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = [12.5, 30.0][rank]
        evals = [1000, 2500][rank]
        out[rank] = bench.reduce_over_ranks(ms, evals, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(rank_main, args=(2, free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    # every rank sees the slowest rank's time and the sum of all evaluations
    assert res[0] == res[1] == (30.0, 3500.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.0, 11, 1, "cpu") == (7.0, 11.0)


def test_ranks_train_on_their_own_data():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2208_07023_gb300 import workloads as W
    seeds = [bench.rank_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8
    a = W.SETTINGS["node_n2000_d16"]["builder"](seeds[0])
    b = W.SETTINGS["node_n2000_d16"]["builder"](seeds[1])
    assert a.X.shape == b.X.shape and not (a.X == b.X).all()


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_bench_line_keys_of_reference_arm():
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys (a short run on the smallest workload)."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "node_n2000_d16", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in j, k
    assert j["impl"] == "reference" and j["value"] > 0
    assert j["config"]["workload"] == "node_n2000_d16"


def forest_rank_main(rank, world, port, out):
    """Rank r grows trees r, r + N, ... of one small bagged forest with the
    oracle (every tree keyed by its global id) and the ranks gather them."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle as O
    from paper_2208_07023_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        wl = W.gmm(600, 4, 3, seed=5)
        p = O.make_params("gini", 3, n_particles=8, n_iters=4, n_bins=16, max_depth=3,
                          min_leaf=5, precision=O.F32_MIRROR)
        first, stride, count = bench.rank_forest_share(5, rank, world)
        mine = []
        for t in range(count):
            tid = first + t * stride
            tr = O.train_tree(p, wl.X, wl.labels, tree_id=tid, bootstrap=True)
            mine.append((tid, {k: np.asarray(getattr(tr, k)).tolist()
                               for k in ("kind", "bin", "leaf_class", "weight", "dir")}))
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        out[rank] = sorted(kv for part in parts for kv in part)
    finally:
        dist.destroy_process_group()


def test_forest_split_across_two_gloo_ranks_equals_one_rank():
    import numpy as np

    import oracle as O
    from paper_2208_07023_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(forest_rank_main, args=(2, free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        got = out[0]
        assert out[1] == got
    assert [tid for tid, _ in got] == [0, 1, 2, 3, 4]
    wl = W.gmm(600, 4, 3, seed=5)
    p = O.make_params("gini", 3, n_particles=8, n_iters=4, n_bins=16, max_depth=3,
                      min_leaf=5, precision=O.F32_MIRROR)
    for tid, arrays in got:
        ref = O.train_tree(p, wl.X, wl.labels, tree_id=tid, bootstrap=True)
        for k, v in arrays.items():
            assert np.array_equal(np.asarray(v), np.asarray(getattr(ref, k))), (tid, k)


def test_forest_share_covers_every_tree_once():
    sys.path.insert(0, ROOT)
    import bench
    for n_trees in (1, 5, 64):
        for world in (1, 2, 3, 8):
            ids = []
            for r in range(world):
                first, stride, count = bench.rank_forest_share(n_trees, r, world)
                ids += [first + t * stride for t in range(count)]
            assert sorted(ids) == list(range(n_trees))
