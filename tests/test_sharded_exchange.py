"""The sample-sharded exchange of a node search, emulated on two CPU ranks
(gloo). A node's samples are split between the ranks; each projects its own
samples (the oracle's fp32-mirror projection), the ranks all-reduce the
per-particle ranges (min / max: exact), bin with the global range, and
all-reduce their per-bin class counts or fixed-point moments (integer sums:
exact in any order). The result is the unsharded node's: the same range, the
same bins, the same histograms, so every rank's threshold scan and argmins
see identical inputs, and the swarm update needs no broadcast because both
ranks draw the same counter-based random streams. (The GPU path here runs on
one device; this pins the exchange it would add.)"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P, B, K, SEED, UID = 12, 64, 4, 5, 77
FIX_BITS = 40  # fixed-point step of the MSE moments: 2^-40 of the target's scale


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def node_data():
    sys.path.insert(0, ROOT)
    from paper_2208_07023_gb300 import workloads as W
    wl = W.gmm(4001, 9, K, seed=3)
    rng = np.random.default_rng(4)
    pos = rng.uniform(-1, 1, (P, 9)).astype(np.float32).astype(np.float64)
    y = (wl.X[:, 0] * 2.5 + rng.standard_normal(wl.n)).astype(np.float32)
    return wl.X, wl.labels, y, pos


def bins_of(z, zmin, zmax):
    # the binning of the mirror arithmetic: float32, one rounding per operation
    z32, lo, hi = np.float32(z), np.float32(zmin), np.float32(zmax)
    inv_w = np.float32(B) / (hi - lo)
    b = np.floor((z32 - lo[:, None]) * inv_w[:, None]).astype(np.int64)
    return np.minimum(b, B - 1)


def fixed_point(y, scale):
    return np.rint(y.astype(np.float64) * scale).astype(np.int64)


def rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import oracle as O
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        X, labels, y, pos = node_data()
        n = len(labels)
        shard = np.arange(rank, n, world, dtype=np.int32)  # interleaved shards
        p = O.make_params("gini", K, P, 0, B, min_leaf=1)
        _, _, z = O.eval_swarm(p, X, labels, None, pos, idx=shard, want_z=True)
        lo = torch.from_numpy(z.min(axis=1).copy())
        hi = torch.from_numpy(z.max(axis=1).copy())
        dist.all_reduce(lo, op=dist.ReduceOp.MIN)
        dist.all_reduce(hi, op=dist.ReduceOp.MAX)
        bins = bins_of(z, lo.numpy(), hi.numpy())
        cnt = np.zeros((P, B, K), np.int64)
        for q in range(P):
            np.add.at(cnt[q], (bins[q], labels[shard]), 1)
        c = torch.from_numpy(cnt)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        # regression moments: a shared scale from the all-reduced target range
        ymax = torch.tensor([float(np.abs(y[shard]).max())], dtype=torch.float64)
        dist.all_reduce(ymax, op=dist.ReduceOp.MAX)
        scale = 2.0 ** FIX_BITS / ymax.item()
        m1 = np.zeros((P, B), np.int64)
        for q in range(P):
            np.add.at(m1[q], bins[q], fixed_point(y[shard], scale))
        s1 = torch.from_numpy(m1)
        dist.all_reduce(s1, op=dist.ReduceOp.SUM)
        u = np.empty(P * 9, np.float32)
        O.lib().ora_swarm_uniforms(SEED, UID, 1, P, 9, O.PURPOSE_R1, O._ptr(u))
        out[rank] = dict(lo=lo.numpy(), hi=hi.numpy(), cnt=c.numpy(), m1=s1.numpy(),
                         bins=bins, shard=shard, scale=scale, r1=u)
    finally:
        dist.destroy_process_group()


def test_sharded_node_equals_unsharded_node():
    import oracle as O
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.start_processes(rank_main, args=(2, free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    X, labels, y, pos = node_data()
    n = len(labels)
    p = O.make_params("gini", K, P, 0, B, min_leaf=1)
    ev, bins_full, z_full = O.eval_swarm(p, X, labels, None, pos, want_bins=True, want_z=True)
    # the exchanged ranges are the node's
    for r in (0, 1):
        assert np.array_equal(res[r]["lo"], z_full.min(axis=1))
        assert np.array_equal(res[r]["hi"], z_full.max(axis=1))
        assert np.array_equal(res[r]["r1"], res[0]["r1"])  # one random stream
    # every sample's bin is the oracle's unsharded bin
    for r in (0, 1):
        assert np.array_equal(res[r]["bins"], bins_full[:, res[r]["shard"]])
    # the all-reduced histograms are the node's, on both ranks
    want = np.zeros((P, B, K), np.int64)
    for q in range(P):
        np.add.at(want[q], (bins_full[q], labels), 1)
    assert np.array_equal(res[0]["cnt"], want) and np.array_equal(res[1]["cnt"], want)
    scale = res[0]["scale"]
    want_m1 = np.zeros((P, B), np.int64)
    for q in range(P):
        np.add.at(want_m1[q], bins_full[q], fixed_point(y, scale))
    assert np.array_equal(res[0]["m1"], want_m1) and np.array_equal(res[1]["m1"], want_m1)
    # and the node's score follows from those bins alone
    for q in (0, P - 1):
        s = O.score_bins(p, labels, None, bins_full[q])
        assert (s["bin"], s["q_num"], s["q_den"]) == (ev[q]["bin"], ev[q]["q_num"],
                                                      ev[q]["q_den"])
