"""ctypes binding of libslm (include/slm.h).

Argument marshalling only: every step of the computation runs inside
libslm.so. Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
their raw pointers go to the C ABI, which stages host arrays itself. If the
library is missing or cannot be loaded the import of a Context fails loudly;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

SLM_OK, SLM_EINVAL, SLM_ENOMEM, SLM_ECUDA, SLM_ETIMEOUT, SLM_EUNSUPPORTED = range(6)
SLM_GINI, SLM_ENTROPY, SLM_MSE = 0, 1, 2
SLM_PROJ_FP32, SLM_PROJ_BF16_TOPK = 0, 1
CRITERIA = {"gini": SLM_GINI, "entropy": SLM_ENTROPY, "mse": SLM_MSE}
PURPOSE_INIT_X, PURPOSE_INIT_V, PURPOSE_R1, PURPOSE_R2 = 1, 2, 3, 4
KERNELS = ["project", "hist_scan", "move", "swarm_init", "node_stats",
           "partition", "compact", "gather", "other", "project_mma", "topk", "proposal",
           "node_search"]


class slm_params(C.Structure):
    _fields_ = [
        ("criterion", C.c_int32), ("n_classes", C.c_int32),
        ("n_particles", C.c_int32), ("n_iters", C.c_int32),
        ("n_bins", C.c_int32), ("topk", C.c_int32), ("inertia", C.c_float),
        ("c1", C.c_float), ("c2", C.c_float), ("max_depth", C.c_int32),
        ("min_leaf", C.c_int32), ("proj", C.c_int32), ("n_trees", C.c_int32),
        ("bootstrap", C.c_int32), ("seeded", C.c_int32), ("top_n", C.c_int32),
        ("apso", C.c_int32), ("seed", C.c_uint64),
    ]


class slm_eval(C.Structure):
    _fields_ = [
        ("loss", C.c_double), ("q_num", C.c_uint64), ("q_den", C.c_uint64),
        ("zmin", C.c_float), ("inv_w", C.c_float), ("bin", C.c_int32),
        ("valid", C.c_int32), ("n_left", C.c_int64), ("n_right", C.c_int64),
    ]


class slm_split(C.Structure):
    _fields_ = [
        ("eval", slm_eval), ("particle", C.c_int32),
        ("iter_of_best", C.c_int32), ("threshold", C.c_float),
        ("norm", C.c_float),
    ]


class slm_prob(C.Structure):
    _fields_ = [
        ("n_candidates", C.c_int32), ("R", C.c_int32), ("gamma", C.c_double),
        ("alpha0", C.c_double), ("alpha", C.c_double), ("batch", C.c_int32),
        ("q", C.c_int32), ("cos_num", C.c_int32), ("cos_den", C.c_int32),
    ]


def make_prob(n_candidates=1000, R=4, gamma=0.8, alpha0=8.0, alpha=0.05, batch=64, q=4,
              cos_num=9, cos_den=10) -> slm_prob:
    """Parameters of the probabilistic search (Sec. II-B): candidates, ranks
    chosen per candidate, the rank weight ratio gamma, the coefficient range
    alpha0 exp(-alpha r), candidates per scoring batch, vectors kept by the
    cosine pruning and its threshold cos_num / cos_den."""
    return slm_prob(n_candidates, R, gamma, alpha0, alpha, batch, q, cos_num, cos_den)


class SlmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libslm status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Loads libslm.so (building it first if stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libslm.so not found at {path}")
        L = C.CDLL(path)
        vp, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        P = C.POINTER
        sig = {
            "slm_status_string": ([C.c_int], C.c_char_p),
            "slm_create": ([P(vp), C.c_int, vp], C.c_int),
            "slm_destroy": ([vp], None),
            "slm_last_error": ([vp, C.c_char_p, C.c_size_t], C.c_int),
            "slm_swarm_uniforms": ([vp, u64, u32, u32, i32, i32, i32, vp], C.c_int),
            "slm_bootstrap": ([vp, u64, u32, i64, vp], C.c_int),
            "slm_evaluate_swarm": ([vp, P(slm_params), vp, i64, i32, vp, vp, vp, vp,
                                    i64, vp, i32, vp, vp], C.c_int),
            "slm_node_split": ([vp, P(slm_params), vp, i64, i32, vp, vp, vp, vp, i64,
                                u32, vp, vp, P(slm_split), vp], C.c_int),
            "slm_prob_search": ([vp, P(slm_params), P(slm_prob), vp, i64, i32, vp, vp, vp, vp,
                                 i64, u32, vp, vp, P(slm_split), vp, vp, vp, P(i32)], C.c_int),
            "slm_forest_begin": ([vp, P(slm_params), vp, i64, i32, vp, vp, P(vp)], C.c_int),
            "slm_grow_level": ([vp, vp, P(i32)], C.c_int),
            "slm_train_tree": ([vp, P(slm_params), vp, i64, i32, vp, vp, P(vp)], C.c_int),
            "slm_forest_free": ([vp], None),
            "slm_forest_info": ([vp, P(i32), P(i32), P(i32), P(i64)], C.c_int),
            "slm_forest_export": ([vp, vp, i32] + [vp] * 11, C.c_int),
            "slm_predict": ([vp, vp, vp, i64, i32, vp, vp, vp], C.c_int),
            "slm_profile": ([vp, C.c_int], C.c_int),
            "slm_kernel_stats": ([vp, i32, P(i64), P(C.c_double), P(C.c_double)], C.c_int),
            "slm_launch_count": ([vp, P(i64)], C.c_int),
            "slm_set_graphs": ([vp, i32], C.c_int),
            "slm_set_projection_tma": ([vp, i32], C.c_int),
            "slm_set_fused_step": ([vp, i32, P(i64)], C.c_int),
            "slm_set_class_hist": ([vp, i32, i32], C.c_int),
            "slm_set_tree_ids": ([vp, i64, i64], C.c_int),
            "slm_set_step_shape": ([vp, i32, P(i32)], C.c_int),
            "slm_seeded_start": ([vp, P(slm_params), vp, i64, i32, vp, vp, vp, vp, i64, u32,
                                  vp], C.c_int),
            "slm_measure_peaks": ([C.c_int, vp, P(C.c_double), P(C.c_double)], C.c_int),
            "slm_set_tuning": ([vp, i32], C.c_int),
            "slm_set_small_nodes": ([vp, i32, i64], C.c_int),
            "slm_set_node_search": ([vp, i32], C.c_int),
            "slm_test_hooks": ([vp, i32, i64], C.c_int),
            "slm_last_node_search": ([vp, P(i32)], C.c_int),
            "slm_force_tiles": ([vp, i32, i32, i32], C.c_int),
            "slm_tuning_stats": ([vp, P(i64), P(i32), P(i32), P(i32)], C.c_int),
            "slm_tuned_shapes": ([vp, i32, P(i32), vp, vp, vp, vp, vp, vp, vp], C.c_int),
            "slm_graph_stats": ([vp, P(i64), P(i64), P(i64), P(i64)], C.c_int),
            "slm_evaluate_swarm_noalloc": ([C.c_int, vp, P(slm_params), vp, i64, i32, vp, vp,
                                            vp, vp, i64, vp, i32, vp], C.c_int),
            "slm_node_stats": ([vp, vp, i64, i32, vp, i32, vp, vp, vp, i64, vp], C.c_int),
            "slm_proposal_create": ([vp, u64, P(vp)], C.c_int),
            "slm_proposal_free": ([vp], None),
            "slm_proposal_set": ([vp, vp] + [vp] * 6, C.c_int),
            "slm_proposal_get": ([vp, vp] + [vp] * 6, C.c_int),
            "slm_proposal_forward": ([vp, vp, vp, i32, vp], C.c_int),
            "slm_proposal_loss_grad": ([vp, vp, vp, vp, vp, i32, P(C.c_double)] + [vp] * 6,
                                       C.c_int),
            "slm_proposal_train": ([vp, vp, vp, vp, vp, i32, i32, i32, C.c_float, u64, vp],
                                   C.c_int),
            "slm_use_proposal": ([vp, vp], C.c_int),
            "slm_swarm_seed": ([vp, u64, u32, i32, i32, vp, vp, vp], C.c_int),
            "slm_train_boost": ([vp, P(slm_params), vp, i64, i32, vp, vp, i32, C.c_float,
                                 vp, P(vp)], C.c_int),
            "slm_boost_predict": ([vp, vp, vp, i64, i32, vp, vp], C.c_int),
            "slm_boost_info": ([vp, P(i32), P(i32), P(C.c_float), P(C.c_float)], C.c_int),
            "slm_boost_tree": ([vp, i32], vp),
            "slm_boost_free": ([vp], None),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def measure_peaks(device: int = 0, stream=None) -> dict:
    """slm_measure_peaks: measured FP32 FFMA throughput (TFLOP/s) and L2 read
    bandwidth (GB/s) of `device`."""
    f, g = C.c_double(), C.c_double()
    st = lib().slm_measure_peaks(device, stream, C.byref(f), C.byref(g))
    if st != SLM_OK:
        raise SlmError(st, "slm_measure_peaks")
    return {"ffma_tflops": f.value, "l2_read_gbs": g.value}


def make_params(criterion="gini", n_classes=2, n_particles=32, n_iters=50,
                n_bins=64, inertia=0.7, c1=1.5, c2=1.5, max_depth=8, min_leaf=1,
                seed=1, n_trees=1, bootstrap=False, proj=SLM_PROJ_FP32,
                topk=8, seeded=False, top_n=0, apso=False) -> slm_params:
    crit = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    return slm_params(crit, 0 if crit == SLM_MSE else n_classes, n_particles,
                      n_iters, n_bins, topk, inertia, c1, c2, max_depth, min_leaf,
                      proj, n_trees, 1 if bootstrap else 0, 1 if seeded else 0, top_n,
                      1 if apso else 0, seed)


def _ptr(a) -> Optional[int]:
    """Raw pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _as(a, dtype):
    if a is None or not isinstance(a, (list, tuple, np.ndarray)):
        return a
    return np.ascontiguousarray(a, dtype=dtype)


class Forest:
    def __init__(self, ctx: "Context", handle: int):
        self.ctx = ctx
        self.handle = C.c_void_p(handle)

    def info(self):
        """slm_forest_info: trees, heap size, features and evaluations so far."""
        nt, hs, d, ev = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        self.ctx._check(lib().slm_forest_info(self.handle, C.byref(nt), C.byref(hs),
                                              C.byref(d), C.byref(ev)))
        return {"n_trees": nt.value, "heap_size": hs.value, "d": d.value,
                "evaluations": ev.value}

    def grow_level(self) -> int:
        """slm_grow_level: grows every tree one level; returns the nodes split."""
        n = C.c_int32()
        self.ctx._check(lib().slm_grow_level(self.ctx.handle, self.handle, C.byref(n)))
        return n.value

    def export(self, tree: int = 0) -> dict:
        """slm_forest_export: tree `tree`'s heap arrays as numpy arrays."""
        inf = self.info()
        H, d = inf["heap_size"], inf["d"]
        out = {"kind": np.empty(H, np.int32), "dir": np.empty((H, d), np.float32),
               "zmin": np.empty(H, np.float32), "inv_w": np.empty(H, np.float32),
               "bin": np.empty(H, np.int32), "leaf_class": np.empty(H, np.int32),
               "leaf_value": np.empty(H, np.float64), "weight": np.empty(H, np.int64),
               "loss": np.empty(H, np.float64), "n_left": np.empty(H, np.int64),
               "n_right": np.empty(H, np.int64)}
        self.ctx._check(lib().slm_forest_export(
            self.ctx.handle, self.handle, tree,
            *[_ptr(out[k]) for k in ("kind", "dir", "zmin", "inv_w", "bin", "leaf_class",
                                     "leaf_value", "weight", "loss", "n_left", "n_right")]))
        return out

    def free(self):
        """slm_forest_free (idempotent)."""
        if self.handle:
            lib().slm_forest_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _RoundTree(Forest):
    """A boosting round's tree: owned by its Boost, never freed here."""

    def __init__(self, ctx, handle, owner):
        super().__init__(ctx, handle)
        self._owner = owner  # keeps the boost alive while the tree is used

    def free(self):
        """The boost owns its trees: nothing to free here."""
        self.handle = C.c_void_p(None)


class Boost:
    """SLR / SLM Boost: trees fitted to residuals, owned by the library.
    train_loss: training MSE (regression) or cross-entropy after each round."""

    def __init__(self, ctx: "Context", handle, train_loss):
        self.ctx, self.handle = ctx, C.c_void_p(handle)
        self.train_loss = train_loss
        self.train_mse = train_loss

    def info(self) -> dict:
        """slm_boost_info: rounds, outputs, base and learning rate."""
        m, k, b, lr = C.c_int32(), C.c_int32(), C.c_float(), C.c_float()
        self.ctx._check(lib().slm_boost_info(self.handle, C.byref(m), C.byref(k), C.byref(b),
                                             C.byref(lr)))
        return {"n_rounds": m.value, "n_outputs": k.value, "base": b.value,
                "learning_rate": lr.value}

    def tree(self, t: int) -> Forest:
        """Tree t = round * n_outputs + output."""
        h = lib().slm_boost_tree(self.handle, t)
        if not h:
            raise IndexError(t)
        return _RoundTree(self.ctx, h, self)

    def predict(self, X, want_class=False):
        """Scores [n] (regression) or [n, K]; with want_class also the argmax."""
        X = _as(X, np.float32)
        n, d = X.shape
        K = self.info()["n_outputs"]
        out = np.empty((n, K) if K > 1 else n, np.float32)
        cls = np.empty(n, np.int32) if want_class else None
        self.ctx._check(lib().slm_boost_predict(self.ctx.handle, self.handle, _ptr(X), n, d,
                                                _ptr(out), _ptr(cls)))
        return (out, cls) if want_class else out

    def free(self):
        """slm_boost_free (idempotent)."""
        if self.handle:
            lib().slm_boost_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


PROP_D, PROP_K, PROP_H, PROP_P = 256, 20, 512, 64
PROP_IN, PROP_OUT = PROP_D * (PROP_K + 1), PROP_D + PROP_P
PROP_SHAPES = {"W1": (PROP_IN, PROP_H), "b1": (PROP_H,), "W2": (PROP_H, PROP_H),
               "b2": (PROP_H,), "W3": (PROP_H, PROP_OUT), "b3": (PROP_OUT,)}
_PROP_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


class Proposal:
    """A learned swarm proposal (network) owned by the library."""

    def __init__(self, ctx: "Context", handle):
        self.ctx, self.handle = ctx, handle

    def free(self):
        """slm_proposal_free (idempotent)."""
        if self.handle:
            lib().slm_proposal_free(self.handle)
            self.handle = C.c_void_p(None)

    def set(self, params: dict):
        """slm_proposal_set: the network's weights from numpy arrays."""
        arrs = [_as(np.ascontiguousarray(params[k], dtype=np.float32), np.float32)
                for k in _PROP_ORDER]
        self.ctx._check(lib().slm_proposal_set(self.ctx.handle, self.handle,
                                               *[_ptr(a) for a in arrs]))

    def get(self) -> dict:
        """slm_proposal_get: the network's weights as numpy arrays."""
        out = {k: np.empty(PROP_SHAPES[k], np.float32) for k in _PROP_ORDER}
        self.ctx._check(lib().slm_proposal_get(self.ctx.handle, self.handle,
                                               *[_ptr(out[k]) for k in _PROP_ORDER]))
        return out

    def forward(self, stats) -> np.ndarray:
        """slm_proposal_forward: outputs for a batch of node statistics."""
        stats = np.ascontiguousarray(stats, dtype=np.float32).reshape(-1, PROP_IN)
        out = np.empty((stats.shape[0], PROP_OUT), np.float32)
        self.ctx._check(lib().slm_proposal_forward(self.ctx.handle, self.handle, _ptr(stats),
                                                   stats.shape[0], _ptr(out)))
        return out

    def loss_grad(self, stats, dims, targets):
        """slm_proposal_loss_grad: loss and gradients of a batch."""
        stats = np.ascontiguousarray(stats, dtype=np.float32).reshape(-1, PROP_IN)
        n = stats.shape[0]
        dims = np.ascontiguousarray(dims, dtype=np.int32)
        targets = np.ascontiguousarray(targets, dtype=np.float32).reshape(n, PROP_D)
        g = {k: np.empty(PROP_SHAPES[k], np.float32) for k in _PROP_ORDER}
        loss = C.c_double()
        self.ctx._check(lib().slm_proposal_loss_grad(
            self.ctx.handle, self.handle, _ptr(stats), _ptr(dims), _ptr(targets), n,
            C.byref(loss), *[_ptr(g[k]) for k in _PROP_ORDER]))
        return loss.value, g

    def train(self, stats, dims, targets, epochs=10, batch=64, lr=1e-3, seed=1):
        """slm_proposal_train: Adam steps on (statistics, direction) pairs."""
        stats = _as(stats, np.float32)
        dims = _as(dims, np.int32)
        targets = _as(targets, np.float32)
        n = int(dims.shape[0])
        losses = np.zeros(epochs, np.float64)
        self.ctx._check(lib().slm_proposal_train(
            self.ctx.handle, self.handle, _ptr(stats), _ptr(dims), _ptr(targets), n, epochs,
            batch, lr, seed, _ptr(losses)))
        return losses


class Context:
    """One libslm context (device + stream)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        h = C.c_void_p()
        st = lib().slm_create(C.byref(h), device, stream)
        if st != SLM_OK:
            raise SlmError(st, "slm_create failed")
        self.handle = h

    def _check(self, st: int):
        if st != SLM_OK:
            buf = C.create_string_buffer(512)
            lib().slm_last_error(self.handle, buf, 512)
            raise SlmError(st, buf.value.decode(errors="replace"))

    def close(self):
        """slm_destroy (idempotent)."""
        if self.handle:
            lib().slm_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- learned proposal ---------------------------------------------------
    def node_stats(self, X, labels=None, n_classes=0, y=None, sample_idx=None, weights=None):
        """slm_node_stats: the proposal network's input statistics of nodes."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        sample_idx, weights = _as(sample_idx, np.int32), _as(weights, np.uint32)
        n, d = X.shape
        n_idx = n if sample_idx is None else sample_idx.shape[0]
        out = np.empty(PROP_IN, np.float32)
        self._check(lib().slm_node_stats(self.handle, _ptr(X), n, d, _ptr(labels), n_classes,
                                         _ptr(y), _ptr(sample_idx), _ptr(weights), n_idx,
                                         _ptr(out)))
        return out

    def proposal(self, seed: int = 1) -> Proposal:
        """slm_proposal_create: a network with Glorot-initialised weights."""
        h = C.c_void_p()
        self._check(lib().slm_proposal_create(self.handle, seed, C.byref(h)))
        return Proposal(self, h)

    def use_proposal(self, prop: Optional[Proposal]):
        """slm_use_proposal: the network seeded searches use."""
        self._check(lib().slm_use_proposal(self.handle, prop.handle if prop else None))

    def swarm_seed(self, seed, node_uid, n_particles, d, mu_hat, rho) -> np.ndarray:
        """slm_swarm_seed: seeded starting positions of one swarm."""
        mu_hat = np.ascontiguousarray(mu_hat, dtype=np.float32)
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        pos = np.empty((n_particles, d), np.float32)
        self._check(lib().slm_swarm_seed(self.handle, seed, node_uid, n_particles, d,
                                         _ptr(mu_hat), _ptr(rho), _ptr(pos)))
        return pos

    # -- diagnostics -------------------------------------------------------
    def profile(self, on: bool):
        """slm_profile: per-launch timing with CUDA events on or off."""
        self._check(lib().slm_profile(self.handle, 1 if on else 0))

    def kernel_stats(self) -> dict:
        """slm_kernel_stats: launches, pairs and milliseconds per kernel class."""
        out = {}
        for k, name in enumerate(KERNELS):
            n, ms, pairs = C.c_int64(), C.c_double(), C.c_double()
            self._check(lib().slm_kernel_stats(self.handle, k, C.byref(n), C.byref(ms),
                                               C.byref(pairs)))
            out[name] = {"launches": n.value, "ms": ms.value, "pairs": pairs.value}
        return out

    def launch_count(self) -> int:
        """slm_launch_count: kernels launched by this context."""
        n = C.c_int64()
        self._check(lib().slm_launch_count(self.handle, C.byref(n)))
        return n.value

    def test_hooks(self, first_wait_polls: int = -1, fail_alloc_after: int = 0):
        """slm_test_hooks: forced wait limit and allocation failure (tests only)."""
        self._check(lib().slm_test_hooks(self.handle, first_wait_polls, fail_alloc_after))

    def set_node_search(self, on: bool):
        """slm_set_node_search: persistent whole-search kernel for small nodes."""
        self._check(lib().slm_set_node_search(self.handle, 1 if on else 0))

    def last_node_search(self) -> int:
        """slm_last_node_search: CTAs per node of the last persistent search."""
        n = C.c_int32()
        self._check(lib().slm_last_node_search(self.handle, C.byref(n)))
        return n.value

    def set_small_nodes(self, max_entries: int = 4096, min_pairs: int = -1):
        """slm_set_small_nodes: the warp-per-particle histogram's thresholds."""
        self._check(lib().slm_set_small_nodes(self.handle, max_entries, min_pairs))

    def set_tuning(self, on: bool):
        """slm_set_tuning: projection tile and histogram cluster tuning on/off."""
        self._check(lib().slm_set_tuning(self.handle, 1 if on else 0))

    def force_tiles(self, pg: int = 0, ctas_per_sm: int = 0, gather: bool = False):
        """slm_force_tiles: fixed projection tiles (pg = 0 releases them)."""
        self._check(lib().slm_force_tiles(self.handle, pg, ctas_per_sm, 1 if gather else 0))

    def tuning_stats(self) -> dict:
        """slm_tuning_stats: tuner passes and the last tiles and cluster size."""
        n, pg, cps, hc = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        self._check(lib().slm_tuning_stats(self.handle, C.byref(n), C.byref(pg), C.byref(cps),
                                           C.byref(hc)))
        return {"shapes": n.value, "last_pg": pg.value, "last_ctas_per_sm": cps.value,
                "last_hist_cluster": hc.value}

    def tuned_shapes(self) -> list:
        """slm_tuned_shapes: every tuned shape and its choice."""
        n = C.c_int32()
        self._check(lib().slm_tuned_shapes(self.handle, 0, C.byref(n), None, None, None, None,
                                           None, None, None))
        m = n.value
        cols = [np.zeros(m, np.int32) for _ in range(6)] + [np.zeros(m, np.float32)]
        self._check(lib().slm_tuned_shapes(self.handle, m, C.byref(n),
                                           *[_ptr(a) for a in cols]))
        names = ("d", "padded_p", "tiles_log2", "pg", "ctas_per_sm", "gather", "ms")
        return [{k: (float(a[i]) if k == "ms" else int(a[i])) for k, a in zip(names, cols)}
                for i in range(m)]

    def set_graphs(self, on: bool):
        """slm_set_graphs: CUDA-graph capture of the search loops."""
        self._check(lib().slm_set_graphs(self.handle, 1 if on else 0))

    def set_projection_tma(self, on: bool):
        """slm_set_projection_tma: tensor-map staging as a tuned candidate."""
        self._check(lib().slm_set_projection_tma(self.handle, 1 if on else 0))

    def set_fused_step(self, on: bool = True, always: bool = False) -> int:
        """slm_set_fused_step: fold the swarm move into the projection (plain FP32
        searches) where the level's projection is short, or (always) wherever
        possible; returns the searches run folded so far."""
        n = C.c_int64()
        mode = 0 if not on else (2 if always else 1)
        self._check(lib().slm_set_fused_step(self.handle, mode, C.byref(n)))
        return n.value

    def set_step_shape(self, shape: int = -1) -> int:
        """slm_set_step_shape: tile shape of the folded projection (-1: chosen
        per batch); returns the shape of the last folded batch."""
        last = C.c_int32()
        self._check(lib().slm_set_step_shape(self.handle, shape, C.byref(last)))
        return last.value

    def set_tree_ids(self, first: int = 0, stride: int = 1):
        """slm_set_tree_ids: local tree t of later forests is global tree
        first + t * stride (bootstrap draw and node uids)."""
        self._check(lib().slm_set_tree_ids(self.handle, first, stride))

    def set_class_hist(self, on: bool, node_step: bool = True):
        """slm_set_class_hist: the latency-oriented classification histogram kernel,
        and whether its last block per node takes the gbest step and the move."""
        self._check(lib().slm_set_class_hist(self.handle, 1 if on else 0, 1 if node_step else 0))

    def graph_stats(self) -> dict:
        """slm_graph_stats: graph launches, reuses, updates, instantiations."""
        a, r, b, c = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(lib().slm_graph_stats(self.handle, C.byref(a), C.byref(r), C.byref(b),
                                          C.byref(c)))
        return {"launches": a.value, "reuses": r.value, "updates": b.value,
                "instantiations": c.value}

    # -- raw draws -------------------------------------------------------
    def swarm_uniforms(self, seed, node_uid, t, n_particles, d, purpose):
        """slm_swarm_uniforms: one swarm stream's uniforms [P, d]."""
        u = np.empty((n_particles, d), np.float32)
        self._check(lib().slm_swarm_uniforms(self.handle, seed, node_uid, t,
                                             n_particles, d, purpose, _ptr(u)))
        return u

    def bootstrap(self, seed, tree_id, n):
        """slm_bootstrap: tree `tree_id`'s bootstrap multiplicities [n]."""
        w = np.empty(n, np.uint32)
        self._check(lib().slm_bootstrap(self.handle, seed, tree_id, n, _ptr(w)))
        return w

    # -- scoring and search ------------------------------------------------
    def evaluate_swarm(self, params, X, positions, labels=None, y=None,
                       sample_idx=None, weights=None, want_bins=False):
        """slm_evaluate_swarm: scores (and optionally bins) of given projections."""
        X = _as(X, np.float32)
        positions = _as(positions, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        sample_idx, weights = _as(sample_idx, np.int32), _as(weights, np.uint32)
        n, d = X.shape
        n_pos = positions.shape[0]
        n_idx = n if sample_idx is None else sample_idx.shape[0]
        out = (slm_eval * n_pos)()
        bins = np.empty((n_pos, n_idx), np.int32) if want_bins else None
        self._check(lib().slm_evaluate_swarm(
            self.handle, C.byref(params), _ptr(X), n, d, _ptr(labels), _ptr(y),
            _ptr(sample_idx), _ptr(weights), n_idx, _ptr(positions), n_pos, out,
            _ptr(bins)))
        return [_eval_dict(e) for e in out], bins

    def seeded_start(self, params, X, labels=None, y=None, sample_idx=None, weights=None,
                     node_uid=0):
        """slm_seeded_start: the initial positions [P, d] a seeded search of this
        node starts from."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        sample_idx, weights = _as(sample_idx, np.int32), _as(weights, np.uint32)
        n, d = X.shape
        n_idx = n if sample_idx is None else sample_idx.shape[0]
        pos = np.empty((params.n_particles, d), np.float32)
        self._check(lib().slm_seeded_start(
            self.handle, C.byref(params), _ptr(X), n, d, _ptr(labels), _ptr(y),
            _ptr(sample_idx), _ptr(weights), n_idx, node_uid, _ptr(pos)))
        return pos

    def node_split(self, params, X, labels=None, y=None, sample_idx=None,
                   weights=None, node_uid=0, want_trace=False):
        """slm_node_split: one node's swarm search; a dict of the split, gB, direction
        and (want_trace) the gbest loss after every iteration."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        sample_idx, weights = _as(sample_idx, np.int32), _as(weights, np.uint32)
        n, d = X.shape
        n_idx = n if sample_idx is None else sample_idx.shape[0]
        direction = np.empty(d, np.float32)
        gbest = np.empty(d, np.float32)
        trace = np.empty(params.n_iters + 1, np.float64) if want_trace else None
        sp = slm_split()
        self._check(lib().slm_node_split(
            self.handle, C.byref(params), _ptr(X), n, d, _ptr(labels), _ptr(y),
            _ptr(sample_idx), _ptr(weights), n_idx, node_uid, _ptr(direction),
            _ptr(gbest), C.byref(sp), _ptr(trace)))
        res = _eval_dict(sp.eval)
        res.update(particle=sp.particle, iter_of_best=sp.iter_of_best,
                   threshold=sp.threshold, norm=sp.norm, direction=direction,
                   gbest=gbest, trace=trace)
        return res

    def prob_search(self, params, prob, X, labels=None, y=None, sample_idx=None,
                    weights=None, node_uid=0):
        """slm_prob_search: the probabilistic search on one node; a dict of the
        best candidate's split, its vector (\"best\") and direction, the best
        loss after each batch, the feature ranking and the pruning's kept
        candidates."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        sample_idx, weights = _as(sample_idx, np.int32), _as(weights, np.uint32)
        n, d = X.shape
        n_idx = n if sample_idx is None else sample_idx.shape[0]
        direction = np.empty(d, np.float32)
        best = np.empty(d, np.float32)
        # arguments out of range are rejected by the call before it writes
        ok = 1 <= prob.n_candidates <= 1 << 20 and prob.batch >= 1
        trace = np.empty(-(-prob.n_candidates // prob.batch) if ok else 1, np.float64)
        rank_feat = np.empty(d, np.int32)
        kept = np.empty(max(prob.q, 1), np.int32)
        n_kept = C.c_int32(0)
        sp = slm_split()
        self._check(lib().slm_prob_search(
            self.handle, C.byref(params), C.byref(prob), _ptr(X), n, d, _ptr(labels), _ptr(y),
            _ptr(sample_idx), _ptr(weights), n_idx, node_uid, _ptr(direction), _ptr(best),
            C.byref(sp), _ptr(trace), _ptr(rank_feat), _ptr(kept), C.byref(n_kept)))
        res = _eval_dict(sp.eval)
        res.update(particle=sp.particle, iter_of_best=sp.iter_of_best,
                   threshold=sp.threshold, norm=sp.norm, direction=direction, best=best,
                   trace=trace, rank_feat=rank_feat, kept=kept[:n_kept.value])
        return res

    def forest_begin(self, params, X, labels=None, y=None) -> Forest:
        """slm_forest_begin: a forest at its root level (grow with grow_level)."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        n, d = X.shape
        h = C.c_void_p()
        self._check(lib().slm_forest_begin(self.handle, C.byref(params), _ptr(X), n, d,
                                           _ptr(labels), _ptr(y), C.byref(h)))
        return Forest(self, h.value)

    def train_tree(self, params, X, labels=None, y=None) -> Forest:
        """slm_train_tree: trees (params.n_trees) grown to completion."""
        X = _as(X, np.float32)
        labels, y = _as(labels, np.int32), _as(y, np.float32)
        n, d = X.shape
        h = C.c_void_p()
        self._check(lib().slm_train_tree(self.handle, C.byref(params), _ptr(X), n, d,
                                         _ptr(labels), _ptr(y), C.byref(h)))
        return Forest(self, h.value)

    def train_boost(self, params, X, y=None, n_rounds: int = 10, learning_rate: float = 0.3,
                    labels=None, n_classes=None) -> Boost:
        """SLR Boost (y) or SLM Boost (labels; n_classes, else params.n_classes
        when >= 2, else the largest label + 1)."""
        X, y, labels = _as(X, np.float32), _as(y, np.float32), _as(labels, np.int32)
        n, d = X.shape
        if labels is not None:
            params = slm_params.from_buffer_copy(params)
            if n_classes is None:
                n_classes = (params.n_classes if params.n_classes >= 2
                             else int(labels.max()) + 1)
            params.n_classes = n_classes
        loss = np.empty(max(1, n_rounds), np.float64)
        h = C.c_void_p()
        self._check(lib().slm_train_boost(self.handle, C.byref(params), _ptr(X), n, d,
                                          _ptr(labels), _ptr(y), n_rounds, learning_rate,
                                          _ptr(loss), C.byref(h)))
        return Boost(self, h.value, loss[:n_rounds])

    def predict(self, forest: Forest, X, want_leaf=False):
        """slm_predict: classes (vote), values (mean) and optionally leaf ids."""
        X = _as(X, np.float32)
        n, d = X.shape
        nt = forest.info()["n_trees"]
        cls = np.empty(n, np.int32)
        val = np.empty(n, np.float64)
        leaf = np.empty((n, nt), np.int32) if want_leaf else None
        self._check(lib().slm_predict(self.handle, forest.handle, _ptr(X), n, d,
                                      _ptr(cls), _ptr(val), _ptr(leaf)))
        return cls, val, leaf


def _eval_dict(e: slm_eval) -> dict:
    return {name: getattr(e, name) for name, _ in e._fields_}
