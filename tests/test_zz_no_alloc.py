"""The no-allocation scoring entry point (slm_evaluate_swarm_noalloc).

Some callers cannot allocate device memory while they run -- their memory is
reserved up front and handed out by their own pool, or the allocator is not
available where they run -- so this entry point keeps all its scratch in one
fixed device array inside the library. These checks call it through the C
ABI with caller-owned device buffers and compare its scores with those of
slm_evaluate_swarm on the same inputs:
  * Gini, entropy (which reads the c ln c table) and MSE scores;
  * bootstrap multiplicities (the weighted path);
  * the same call twice in a row, and a smaller call after a larger one of
    the same criterion, so that stale contents of the shared array from the
    earlier call would show;
and that it refuses what it cannot do without a launch: the tensor-core
form, an unknown projection mode and host pointers. The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params


def _noalloc(S, torch, params, X, labels=None, y=None, idx=None, positions=None,
             weights=None, host_X=False):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None
    Xd, Ld, Yd, Id, Pd, Wd = (dev(X), dev(labels), dev(y), dev(idx), dev(positions),
                              dev(weights))
    Xh = np.ascontiguousarray(X) if host_X else None
    out = torch.zeros(positions.shape[0] * ctypes.sizeof(S.slm_eval), dtype=torch.uint8,
                      device="cuda")
    torch.cuda.synchronize()
    n, d = X.shape
    n_idx = n if idx is None else idx.shape[0]
    ptr = lambda t: t.data_ptr() if t is not None else None
    st = S.lib().slm_evaluate_swarm_noalloc(
        0, None, ctypes.byref(params), Xh.ctypes.data if host_X else Xd.data_ptr(), n, d,
        ptr(Ld), ptr(Yd), ptr(Id), ptr(Wd), n_idx, Pd.data_ptr(), positions.shape[0],
        out.data_ptr())
    host = out.cpu().numpy().tobytes()
    res = (S.slm_eval * positions.shape[0]).from_buffer_copy(host)
    return st, [{k: getattr(e, k) for k, _ in e._fields_} for e in res]


def _same(crit, got, ref):
    for g, r in zip(got, ref):
        assert (g["valid"], g["bin"], g["n_left"], g["n_right"]) == \
            (r["valid"], r["bin"], r["n_left"], r["n_right"])
        assert (g["zmin"], g["inv_w"]) == (r["zmin"], r["inv_w"])
        if crit == "gini":
            assert (g["q_num"], g["q_den"], g["loss"]) == (r["q_num"], r["q_den"], r["loss"])
        else:
            # entropy and MSE: the same kernels on the same bins; 1e-9 is the
            # parity bar of the double-precision criteria
            assert g["loss"] == pytest.approx(r["loss"], rel=1e-9)


@pytest.mark.gpu
def test_noalloc_matches_evaluate_swarm():
    torch = pytest.importorskip("torch")
    ctx = context()
    from paper_2208_07023_gb300 import binding as S
    rng = np.random.default_rng(3)
    big = W.gmm(9000, 24, 6, seed=31)
    small = W.gmm(1500, 24, 6, seed=33)
    boot = np.bincount(rng.integers(0, 5000, 5000), minlength=5000).astype(np.uint32)
    cases = [
        # (criterion, workload, particles, bins, sample subset, multiplicities)
        ("gini", big, 48, 64, rng.choice(9000, 7001, replace=False), None),
        ("gini", big, 48, 64, None, None),       # the same criterion, larger
        ("gini", big, 48, 64, None, None),       # ... and the same call again
        ("gini", small, 16, 32, None, None),     # smaller after larger
        ("entropy", W.gmm(5000, 12, 3, seed=34), 32, 64, None, None),
        ("gini", W.gmm(5000, 12, 3, seed=35), 24, 128, None, boot),
        ("mse", W.tanh_regression(6000, 16, seed=32), 20, 128, None, None),
        ("mse", W.tanh_regression(2000, 16, seed=36), 8, 64, None, None),
    ]
    for crit, wl, P, B, idx, wts in cases:
        idx = None if idx is None else idx.astype(np.int32)
        pos = rng.uniform(-1, 1, (P, wl.d)).astype(np.float32)
        gp = gpu_params(S, crit, wl.n_classes, P, 0, B, min_leaf=5)
        ref, _ = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y, sample_idx=idx,
                                    weights=wts)
        st, got = _noalloc(S, torch, gp, wl.X, wl.labels, wl.y, idx, pos, weights=wts)
        assert st == S.SLM_OK, (crit, P, B)
        _same(crit, got, ref)
    ctx.close()


@pytest.mark.gpu
def test_noalloc_rejects_what_it_cannot_do():
    torch = pytest.importorskip("torch")
    from paper_2208_07023_gb300 import binding as S
    X = np.zeros((200_000, 64), np.float32)
    pos = np.zeros((64, 64), np.float32)
    gp = gpu_params(S, "gini", 2, 64, 0, 16)
    st, _ = _noalloc(S, torch, gp, X, np.zeros(200_000, np.int32), None, None, pos)
    assert st == S.SLM_EUNSUPPORTED  # beyond the fixed array
    wl = W.gmm(1000, 8, 2, seed=37)
    pos = np.ones((16, 8), np.float32)
    gp = gpu_params(S, "gini", 2, 16, 0, 16)
    gp.proj = S.SLM_PROJ_BF16_TOPK
    st, _ = _noalloc(S, torch, gp, wl.X, wl.labels, None, None, pos)
    assert st == S.SLM_EUNSUPPORTED  # the FP32 form only
    gp.proj = 7
    st, _ = _noalloc(S, torch, gp, wl.X, wl.labels, None, None, pos)
    assert st == S.SLM_EINVAL
    gp = gpu_params(S, "gini", 2, 16, 0, 16)
    st, _ = _noalloc(S, torch, gp, wl.X, wl.labels, None, None, pos, host_X=True)
    assert st == S.SLM_EINVAL  # rows in host memory are refused before any launch
    st, got = _noalloc(S, torch, gp, wl.X, wl.labels, None, None, pos)
    assert st == S.SLM_OK and got[0]["valid"] in (0, 1)
