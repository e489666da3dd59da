"""The no-allocation scoring entry point (slm_evaluate_swarm_noalloc).

Some callers cannot allocate device memory while they run -- their memory is
reserved up front and handed out by their own pool -- so this entry point
keeps all its scratch in one fixed device array inside the library. These
checks call it through the C ABI with caller-owned device buffers and compare
its scores with those of slm_evaluate_swarm, twice in a row (the second call
must not see anything of the first). The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params


def _noalloc(S, torch, params, X, labels=None, y=None, idx=None, positions=None):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None
    Xd, Ld, Yd, Id, Pd = dev(X), dev(labels), dev(y), dev(idx), dev(positions)
    out = torch.zeros(positions.shape[0] * ctypes.sizeof(S.slm_eval), dtype=torch.uint8,
                      device="cuda")
    torch.cuda.synchronize()
    n, d = X.shape
    n_idx = n if idx is None else idx.shape[0]
    st = S.lib().slm_evaluate_swarm_noalloc(
        0, None, ctypes.byref(params), Xd.data_ptr(), n, d,
        Ld.data_ptr() if Ld is not None else None, Yd.data_ptr() if Yd is not None else None,
        Id.data_ptr() if Id is not None else None, None, n_idx, Pd.data_ptr(),
        positions.shape[0], out.data_ptr())
    host = out.cpu().numpy().tobytes()
    res = (S.slm_eval * positions.shape[0]).from_buffer_copy(host)
    return st, [{k: getattr(e, k) for k, _ in e._fields_} for e in res]


@pytest.mark.gpu
def test_noalloc_matches_evaluate_swarm_twice():
    torch = pytest.importorskip("torch")
    ctx = context()
    from paper_2208_07023_gb300 import binding as S
    rng = np.random.default_rng(3)
    cases = [
        ("gini", W.gmm(9000, 24, 6, seed=31), 48, 64, rng.choice(9000, 7001, replace=False)),
        ("mse", W.tanh_regression(6000, 16, seed=32), 20, 128, None),
    ]
    for crit, wl, P, B, idx in cases:
        idx = None if idx is None else idx.astype(np.int32)
        pos = rng.uniform(-1, 1, (P, wl.d)).astype(np.float32)
        gp = gpu_params(S, crit, wl.n_classes, P, 0, B, min_leaf=5)
        ref, _ = ctx.evaluate_swarm(gp, wl.X, pos, labels=wl.labels, y=wl.y, sample_idx=idx)
        st, got = _noalloc(S, torch, gp, wl.X, wl.labels, wl.y, idx, pos)
        assert st == S.SLM_OK
        for g, r in zip(got, ref):
            assert (g["valid"], g["bin"], g["n_left"], g["n_right"]) == \
                (r["valid"], r["bin"], r["n_left"], r["n_right"])
            assert (g["zmin"], g["inv_w"]) == (r["zmin"], r["inv_w"])
            if crit == "gini":
                assert (g["q_num"], g["q_den"], g["loss"]) == (r["q_num"], r["q_den"], r["loss"])
            else:
                assert g["loss"] == pytest.approx(r["loss"], rel=1e-9)
    ctx.close()


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    from paper_2208_07023_gb300 import binding as S
    X = np.zeros((200_000, 64), np.float32)
    pos = np.zeros((64, 64), np.float32)
    gp = gpu_params(S, "gini", 2, 64, 0, 16)
    st, _ = _noalloc(S, torch, gp, X, np.zeros(200_000, np.int32), None, None, pos)
    assert st == S.SLM_EUNSUPPORTED
