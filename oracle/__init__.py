"""CPU oracle for SLM split search with PSO (arXiv 2208.07023).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs import this package; the product
path (``paper_2208_07023_gb300``) never does, and the two share no code.

The arithmetic lives in ``slm_oracle.c`` (plain C, gcc, OpenMP over particles);
this module builds it with ``gcc -O2 -ffp-contract=off`` and wraps it with
ctypes. Every function takes and returns numpy arrays in host memory.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "slm_oracle.c")
_HDR = os.path.join(_HERE, "slm_oracle.h")

GINI, ENTROPY, MSE = 0, 1, 2
F64, F32_MIRROR, BF16_TOPK = 0, 1, 2
PURPOSE_INIT_X, PURPOSE_INIT_V, PURPOSE_R1, PURPOSE_R2, PURPOSE_BOOTSTRAP = 1, 2, 3, 4, 5
CRITERIA = {"gini": GINI, "entropy": ENTROPY, "mse": MSE}


class Params(C.Structure):
    _fields_ = [
        ("criterion", C.c_int32), ("n_classes", C.c_int32),
        ("n_particles", C.c_int32), ("n_iters", C.c_int32),
        ("n_bins", C.c_int32), ("inertia", C.c_float), ("c1", C.c_float),
        ("c2", C.c_float), ("max_depth", C.c_int32), ("min_leaf", C.c_int32),
        ("seed", C.c_uint64), ("precision", C.c_int32),
        ("n_threads", C.c_int32), ("topk", C.c_int32), ("top_n", C.c_int32),
        ("apso", C.c_int32),
    ]


class Apso(C.Structure):
    _fields_ = [("f", C.c_float), ("state", C.c_int32), ("c1", C.c_float), ("c2", C.c_float),
                ("w", C.c_float)]


class Eval(C.Structure):
    _fields_ = [
        ("zmin", C.c_double), ("zmax", C.c_double), ("inv_w", C.c_double),
        ("valid", C.c_int32), ("bin", C.c_int32), ("loss", C.c_double),
        ("q_num", C.c_uint64), ("q_den", C.c_uint64),
        ("n_left", C.c_double), ("n_right", C.c_double),
    ]


class Split(C.Structure):
    _fields_ = [
        ("valid", C.c_int32), ("particle", C.c_int32),
        ("iter_of_best", C.c_int32), ("bin", C.c_int32),
        ("zmin", C.c_double), ("inv_w", C.c_double),
        ("threshold", C.c_double), ("loss", C.c_double),
        ("q_num", C.c_uint64), ("q_den", C.c_uint64),
        ("n_left", C.c_double), ("n_right", C.c_double),
        ("first_near_tie", C.c_int32), ("elite_tries", C.c_int32),
        ("elite_accepts", C.c_int32),
    ]


class _Mlp(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in ("W1", "b1", "W2", "b2", "W3", "b3")]


MLP_D, MLP_K, MLP_H, MLP_P = 256, 20, 512, 64
MLP_IN, MLP_OUT = MLP_D * (MLP_K + 1), MLP_D + MLP_P
MLP_SHAPES = {"W1": (MLP_IN, MLP_H), "b1": (MLP_H,), "W2": (MLP_H, MLP_H), "b2": (MLP_H,),
              "W3": (MLP_H, MLP_OUT), "b3": (MLP_OUT,)}
PURPOSE_SEED = 6


class Prob(C.Structure):
    _fields_ = [("n_candidates", C.c_int32), ("R", C.c_int32), ("gamma", C.c_double),
                ("alpha0", C.c_double), ("alpha", C.c_double), ("batch", C.c_int32),
                ("q", C.c_int32), ("cos_num", C.c_int32), ("cos_den", C.c_int32)]


class _Tree(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in (
        "kind", "dir", "zmin", "inv_w", "bin", "leaf_class", "leaf_value",
        "weight", "loss", "n_left", "n_right")]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain gcc; no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH) or
             os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                               os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            L.ora_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.ora_swarm_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32,
                                             C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
            L.ora_bootstrap.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_void_p]
            L.ora_pso_step.argtypes = [P(Params), C.c_int32, C.c_int32] + [C.c_void_p] * 6
            L.ora_eval_swarm.argtypes = [P(Params), C.c_void_p, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
            L.ora_eval_swarm.restype = C.c_int
            L.ora_score_bins.argtypes = [P(Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_int64, C.c_void_p, P(Eval)]
            L.ora_score_bins.restype = C.c_int
            L.ora_bf16_round.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
            L.ora_node_stats.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.c_void_p]
            L.ora_node_stats.restype = C.c_int
            L.ora_mlp_forward.argtypes = [P(_Mlp), C.c_void_p, C.c_int32, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            L.ora_mlp_forward.restype = C.c_int
            L.ora_mlp_loss_grad.argtypes = [P(_Mlp), C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int32, C.c_int32, P(C.c_double)] + \
                [C.c_void_p] * 6
            L.ora_mlp_loss_grad.restype = C.c_int
            L.ora_adam_step.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_int32, C.c_double,
                                                           C.c_double, C.c_double, C.c_double]
            L.ora_swarm_seed.argtypes = [C.c_uint64, C.c_uint32, C.c_int32, C.c_int32,
                                         C.c_void_p, C.c_void_p, C.c_void_p]
            L.ora_node_split.argtypes = [P(Params), C.c_void_p, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.c_uint32, C.c_void_p, C.c_void_p, P(Split),
                                         C.c_void_p, C.c_void_p]
            L.ora_node_split.restype = C.c_int
            L.ora_node_split_from.argtypes = [P(Params), C.c_void_p, C.c_int32, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                              P(Split), C.c_void_p, C.c_void_p]
            L.ora_node_split_from.restype = C.c_int
            L.ora_prob_candidate.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32,
                                             C.c_void_p, P(Prob), C.c_void_p]
            L.ora_prob_candidate.restype = None
            L.ora_prob_search.argtypes = [P(Params), P(Prob), C.c_void_p, C.c_int32, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_uint32, C.c_void_p, P(Split), C.c_void_p,
                                          C.c_void_p, C.c_void_p, P(C.c_int32)]
            L.ora_prob_search.restype = C.c_int
            L.ora_select_features.argtypes = [P(Params), C.c_void_p, C.c_int32, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.c_int32, C.c_void_p, C.c_void_p,
                                              C.c_void_p]
            L.ora_select_features.restype = C.c_int
            L.ora_apso_step.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                        C.c_float, C.c_float, C.c_float, P(Apso)]
            L.ora_apso_step.restype = None
            L.ora_elite_candidate.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32,
                                              C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                              P(C.c_int32)]
            L.ora_elite_candidate.restype = None
            L.ora_elite_apply.argtypes = [C.c_int32, C.c_int32] + [C.c_void_p] * 4 + [
                P(C.c_double), C.c_int32, C.c_void_p, C.c_void_p, C.c_double, P(C.c_int32)]
            L.ora_elite_apply.restype = C.c_int32
            L.ora_train_boost.argtypes = [P(Params), C.c_void_p, C.c_int64, C.c_int32,
                                          C.c_void_p, C.c_int32, C.c_float, P(_Tree),
                                          P(C.c_float), C.c_void_p, C.c_void_p]
            L.ora_softmax_residuals.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                                C.c_void_p]
            L.ora_softmax_residuals.restype = None
            L.ora_train_boost_cls.argtypes = [P(Params), C.c_void_p, C.c_int64, C.c_int32,
                                              C.c_void_p, C.c_int32, C.c_int32, C.c_float,
                                              P(_Tree), C.c_void_p, C.c_void_p]
            L.ora_boost_predict_cls.argtypes = [P(Params), P(_Tree), C.c_int32, C.c_int32,
                                                C.c_float, C.c_void_p, C.c_int64, C.c_int32,
                                                C.c_void_p, C.c_void_p]
            L.ora_boost_predict.argtypes = [P(Params), P(_Tree), C.c_int32, C.c_float,
                                            C.c_float, C.c_void_p, C.c_int64, C.c_int32,
                                            C.c_void_p]
            L.ora_train_tree.argtypes = [P(Params), C.c_void_p, C.c_int64, C.c_int32,
                                         C.c_void_p, C.c_void_p, C.c_uint32, C.c_int32,
                                         P(_Tree)]
            L.ora_train_tree.restype = C.c_int
            L.ora_predict.argtypes = [P(Params), P(_Tree), C.c_void_p, C.c_int64,
                                      C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
            L.ora_predict.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(criterion="gini", n_classes=2, n_particles=32, n_iters=50,
                n_bins=64, inertia=0.7, c1=1.5, c2=1.5, max_depth=8,
                min_leaf=1, seed=1, precision=F32_MIRROR, n_threads=0,
                topk=0, top_n=0, apso=False) -> Params:
    crit = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    return Params(crit, 0 if crit == MSE else n_classes, n_particles, n_iters,
                  n_bins, inertia, c1, c2, max_depth, min_leaf, seed, precision,
                  n_threads, topk, top_n, 1 if apso else 0)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def swarm_uniforms(seed, node_uid, t, n_particles, d, purpose) -> np.ndarray:
    u = np.empty((n_particles, d), dtype=np.float32)
    lib().ora_swarm_uniforms(seed, node_uid, t, n_particles, d, purpose, _ptr(u))
    return u


def bootstrap(seed, tree_id, n) -> np.ndarray:
    w = np.empty(n, dtype=np.uint32)
    lib().ora_bootstrap(seed, tree_id, n, _ptr(w))
    return w


def pso_step(params: Params, x, v, pbest, gbest, r1, r2):
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    pbest = np.ascontiguousarray(pbest, dtype=np.float64)
    gbest = np.ascontiguousarray(gbest, dtype=np.float64)
    r1 = np.ascontiguousarray(r1, dtype=np.float64)
    r2 = np.ascontiguousarray(r2, dtype=np.float64)
    P, d = x.shape
    lib().ora_pso_step(C.byref(params), P, d, _ptr(x), _ptr(v), _ptr(pbest),
                       _ptr(gbest), _ptr(r1), _ptr(r2))
    return x, v


def _node_arrays(X, labels, y, idx, wts):
    X = np.ascontiguousarray(X, dtype=np.float32)
    n = X.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
    y = None if y is None else np.ascontiguousarray(y, dtype=np.float32)
    wts = None if wts is None else np.ascontiguousarray(wts, dtype=np.uint32)
    return X, labels, y, idx, wts


def eval_swarm(params: Params, X, labels, y, pos, idx=None, wts=None,
               want_bins=False, want_z=False):
    """Score each row of pos[P, d] on the node idx. Returns (list of dict,
    bins[P, n_idx] or None, z[P, n_idx] or None)."""
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    P, d = pos.shape
    out = (Eval * P)()
    bins = np.empty((P, idx.size), dtype=np.int32) if want_bins else None
    z = np.empty((P, idx.size), dtype=np.float64) if want_z else None
    rc = lib().ora_eval_swarm(C.byref(params), _ptr(X), d, _ptr(labels), _ptr(y),
                              _ptr(idx), _ptr(wts), idx.size, _ptr(pos), P, out,
                              _ptr(bins), _ptr(z))
    if rc:
        raise ValueError(f"ora_eval_swarm failed: {rc}")
    return [_struct_dict(e) for e in out], bins, z


APSO_EXPLORE, APSO_EXPLOIT, APSO_CONVERGE, APSO_JUMPOUT = 1, 2, 3, 4
PURPOSE_APSO = 7


def apso_step(x, gpart, prev_state, c1, c2, delta) -> dict:
    """One adaptive-PSO state update from positions x[P, d]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    P, d = x.shape
    out = Apso()
    lib().ora_apso_step(P, d, _ptr(x), gpart, prev_state, c1, c2, delta, C.byref(out))
    return {name: getattr(out, name) for name, _ in out._fields_}


def elite_candidate(seed, node_uid, t, T, gb, precision=F32_MIRROR):
    """Elitist-learning candidate of the adaptive PSO: (e[d], k)."""
    gb = np.ascontiguousarray(gb, dtype=np.float64)
    e = np.empty_like(gb)
    k = C.c_int32(0)
    lib().ora_elite_candidate(seed, node_uid, t, T, gb.size, _ptr(gb), precision, _ptr(e),
                              C.byref(k))
    return e, k.value


def elite_apply(x, pb, cur_loss, pb_loss, g_loss, gpart, gb, elite, e_loss):
    """Elitist-learning acceptance on losses (inf: invalid). Arrays are
    updated in place; returns (accepted, worst, new gB loss)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    P, d = x.shape
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (pb, cur_loss, pb_loss, gb,
                                                                  elite)]
    g = C.c_double(g_loss)
    w = C.c_int32(-2)
    rc = lib().ora_elite_apply(P, d, _ptr(x), _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                               C.byref(g), gpart, _ptr(arrs[3]), _ptr(arrs[4]), e_loss,
                               C.byref(w))
    if rc < 0:
        raise ValueError(f"ora_elite_apply failed: {rc}")
    return dict(accepted=bool(rc), worst=w.value, g_loss=g.value, x=x, pb=arrs[0],
                cur_loss=arrs[1], pb_loss=arrs[2], gb=arrs[3])


def select_features(params: Params, X, labels, y, n, idx=None, wts=None):
    """The node's n best features by their own split loss (increasing
    feature order), every feature's score, and whether the n-th and the
    (n+1)-th best are a near-tie."""
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    d = X.shape[1]
    feat = np.empty(n, dtype=np.int32)
    ev = (Eval * d)()
    tie = C.c_int32(0)
    rc = lib().ora_select_features(C.byref(params), _ptr(X), d, _ptr(labels), _ptr(y),
                                   _ptr(idx), _ptr(wts), idx.size, n, _ptr(feat), ev,
                                   C.byref(tie))
    if rc:
        raise ValueError(f"ora_select_features failed: {rc}")
    return feat, [_struct_dict(e) for e in ev], bool(tie.value)


def score_bins(params: Params, labels, y, bins, idx=None, wts=None) -> dict:
    """Histogram + threshold scan of given bins[n_idx] of the node idx."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    n_idx = bins.size
    idx = np.arange(n_idx, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, dtype=np.int32)
    labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
    y = None if y is None else np.ascontiguousarray(y, dtype=np.float32)
    wts = None if wts is None else np.ascontiguousarray(wts, dtype=np.uint32)
    e = Eval()
    rc = lib().ora_score_bins(C.byref(params), _ptr(labels), _ptr(y), _ptr(idx), _ptr(wts),
                              n_idx, _ptr(bins), C.byref(e))
    if rc:
        raise ValueError(f"ora_score_bins failed: {rc}")
    return _struct_dict(e)


def bf16_round(a) -> np.ndarray:
    """Nearest bfloat16 of each float32 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    lib().ora_bf16_round(_ptr(a), _ptr(out), a.size)
    return out


def _struct_dict(s) -> dict:
    return {name: getattr(s, name) for name, _ in s._fields_}


@dataclass
class SplitResult:
    split: dict
    gbest: np.ndarray
    direction: np.ndarray
    trace_loss: np.ndarray
    trace_particle: np.ndarray


def node_split(params: Params, X, labels=None, y=None, idx=None, wts=None,
               node_uid=0) -> SplitResult:
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    d = X.shape[1]
    gb = np.zeros(d, dtype=np.float64)
    dr = np.zeros(d, dtype=np.float64)
    T = params.n_iters
    tl = np.zeros(T + 1, dtype=np.float64)
    tp = np.zeros(T + 1, dtype=np.int32)
    sp = Split()
    rc = lib().ora_node_split(C.byref(params), _ptr(X), d, _ptr(labels), _ptr(y),
                              _ptr(idx), _ptr(wts), idx.size, node_uid, _ptr(gb),
                              _ptr(dr), C.byref(sp), _ptr(tl), _ptr(tp))
    if rc:
        raise ValueError(f"ora_node_split failed: {rc}")
    return SplitResult(_struct_dict(sp), gb, dr, tl, tp)


def node_split_from(params: Params, X, init_x, labels=None, y=None, idx=None, wts=None,
                    node_uid=0) -> SplitResult:
    """node_split starting from the positions init_x[P, d] (float32) instead of
    the uniform draws (a learned seed's start); velocities as usual."""
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    d = X.shape[1]
    init_x = np.ascontiguousarray(init_x, dtype=np.float32)
    if init_x.shape != (params.n_particles, d):
        raise ValueError("init_x must be [n_particles, d]")
    gb = np.zeros(d, dtype=np.float64)
    dr = np.zeros(d, dtype=np.float64)
    T = params.n_iters
    tl = np.zeros(T + 1, dtype=np.float64)
    tp = np.zeros(T + 1, dtype=np.int32)
    sp = Split()
    rc = lib().ora_node_split_from(C.byref(params), _ptr(X), d, _ptr(labels), _ptr(y),
                                   _ptr(idx), _ptr(wts), idx.size, node_uid, _ptr(init_x),
                                   _ptr(gb), _ptr(dr), C.byref(sp), _ptr(tl), _ptr(tp))
    if rc:
        raise ValueError(f"ora_node_split_from failed: {rc}")
    return SplitResult(_struct_dict(sp), gb, dr, tl, tp)


def make_prob(n_candidates=1000, R=4, gamma=0.8, alpha0=8.0, alpha=0.05, batch=64, q=4,
              cos_num=9, cos_den=10) -> Prob:
    return Prob(n_candidates, R, gamma, alpha0, alpha, batch, q, cos_num, cos_den)


def prob_candidate(seed, node_uid, c, rank_feat, pp: Prob) -> np.ndarray:
    rank_feat = np.ascontiguousarray(rank_feat, dtype=np.int32)
    a = np.zeros(rank_feat.size, np.float64)
    lib().ora_prob_candidate(seed, node_uid, c, rank_feat.size, _ptr(rank_feat), C.byref(pp),
                             _ptr(a))
    return a


@dataclass
class ProbResult:
    split: dict
    best: np.ndarray
    trace_loss: np.ndarray
    rank_feat: np.ndarray
    kept: np.ndarray


def prob_search(params: Params, pp: Prob, X, labels=None, y=None, idx=None, wts=None,
                node_uid=0) -> ProbResult:
    """The probabilistic search of the original SLM on one node (Sec. II-B)."""
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    d = X.shape[1]
    best = np.zeros(d, np.float64)
    nb = (pp.n_candidates + pp.batch - 1) // pp.batch
    tl = np.zeros(nb, np.float64)
    rf = np.zeros(d, np.int32)
    kept = np.zeros(max(1, pp.q), np.int32)
    nk = C.c_int32()
    sp = Split()
    rc = lib().ora_prob_search(C.byref(params), C.byref(pp), _ptr(X), d, _ptr(labels), _ptr(y),
                               _ptr(idx), _ptr(wts), idx.size, node_uid, _ptr(best),
                               C.byref(sp), _ptr(tl), _ptr(rf), _ptr(kept), C.byref(nk))
    if rc:
        raise ValueError(f"ora_prob_search failed: {rc}")
    return ProbResult(_struct_dict(sp), best, tl, rf, kept[:nk.value].copy())


@dataclass
class Tree:
    max_depth: int
    d: int
    kind: np.ndarray
    dir: np.ndarray
    zmin: np.ndarray
    inv_w: np.ndarray
    bin: np.ndarray
    leaf_class: np.ndarray
    leaf_value: np.ndarray
    weight: np.ndarray
    loss: np.ndarray
    n_left: np.ndarray
    n_right: np.ndarray

    def _cstruct(self):
        return _Tree(*[_ptr(getattr(self, f)) for f, _ in _Tree._fields_])


def _empty_tree(max_depth, d) -> Tree:
    H = (1 << (max_depth + 1)) - 1
    return Tree(max_depth, d, np.zeros(H, np.int32), np.zeros((H, d), np.float64),
                np.zeros(H), np.zeros(H), np.zeros(H, np.int32),
                np.zeros(H, np.int32), np.zeros(H), np.zeros(H), np.zeros(H),
                np.zeros(H), np.zeros(H))


def train_tree(params: Params, X, labels=None, y=None, tree_id=0,
               bootstrap=False) -> Tree:
    X, labels, y, _, _ = _node_arrays(X, labels, y, None, None)
    n, d = X.shape
    t = _empty_tree(params.max_depth, d)
    cs = t._cstruct()
    rc = lib().ora_train_tree(C.byref(params), _ptr(X), n, d, _ptr(labels), _ptr(y),
                              tree_id, 1 if bootstrap else 0, C.byref(cs))
    if rc:
        raise ValueError(f"ora_train_tree failed: {rc}")
    return t


@dataclass
class Boost:
    trees: list
    base: float
    learning_rate: float
    F: np.ndarray          # final boosted predictions of the training rows
    train_mse: np.ndarray  # after each round


def train_boost(params: Params, X, y, n_rounds, learning_rate) -> Boost:
    """SLR Boost: least-squares gradient boosting of SLR trees."""
    X, _, y, _, _ = _node_arrays(X, None, y, None, None)
    n, d = X.shape
    trees = [_empty_tree(params.max_depth, d) for _ in range(n_rounds)]
    arr = (_Tree * max(1, n_rounds))(*[t._cstruct() for t in trees])
    base = C.c_float(0.0)
    F = np.empty(n, np.float32)
    mse = np.empty(max(1, n_rounds), np.float64)
    rc = lib().ora_train_boost(C.byref(params), _ptr(X), n, d, _ptr(y), n_rounds,
                               learning_rate, arr, C.byref(base), _ptr(F), _ptr(mse))
    if rc:
        raise ValueError(f"ora_train_boost failed: {rc}")
    return Boost(trees, base.value, learning_rate, F, mse[:n_rounds])


def boost_predict(params: Params, boost: Boost, X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    M = len(boost.trees)
    arr = (_Tree * max(1, M))(*[t._cstruct() for t in boost.trees])
    out = np.empty(n, np.float32)
    rc = lib().ora_boost_predict(C.byref(params), arr, M, boost.base, boost.learning_rate,
                                 _ptr(X), n, d, _ptr(out))
    if rc:
        raise ValueError(f"ora_boost_predict failed: {rc}")
    return out


@dataclass
class BoostCls:
    trees: list            # [round * K + class]
    n_classes: int
    learning_rate: float
    F: np.ndarray          # [n, K] final scores of the training rows
    train_loss: np.ndarray  # mean cross-entropy after each round


def train_boost_cls(params: Params, X, labels, n_classes, n_rounds, learning_rate) -> BoostCls:
    """SLM Boost: K-class softmax gradient boosting with SLR trees."""
    X, labels, _, _, _ = _node_arrays(X, labels, None, None, None)
    n, d = X.shape
    K = n_classes
    trees = [_empty_tree(params.max_depth, d) for _ in range(n_rounds * K)]
    arr = (_Tree * max(1, len(trees)))(*[t._cstruct() for t in trees])
    F = np.empty((n, K), np.float32)
    loss = np.empty(max(1, n_rounds), np.float64)
    rc = lib().ora_train_boost_cls(C.byref(params), _ptr(X), n, d, _ptr(labels), K, n_rounds,
                                   learning_rate, arr, _ptr(F), _ptr(loss))
    if rc:
        raise ValueError(f"ora_train_boost_cls failed: {rc}")
    return BoostCls(trees, K, learning_rate, F, loss[:n_rounds])


def softmax_residuals(F, labels, n_classes) -> np.ndarray:
    """One round's residuals R[k, i] of the scores F[n, K]."""
    F = np.ascontiguousarray(F, dtype=np.float32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = labels.size
    R = np.empty((n_classes, n), np.float32)
    lib().ora_softmax_residuals(_ptr(F), _ptr(labels), n, n_classes, _ptr(R))
    return R


def boost_predict_cls(params: Params, boost: BoostCls, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    K = boost.n_classes
    M = len(boost.trees) // K
    arr = (_Tree * max(1, len(boost.trees)))(*[t._cstruct() for t in boost.trees])
    F = np.empty((n, K), np.float32)
    cls = np.empty(n, np.int32)
    rc = lib().ora_boost_predict_cls(C.byref(params), arr, M, K, boost.learning_rate,
                                     _ptr(X), n, d, _ptr(F), _ptr(cls))
    if rc:
        raise ValueError(f"ora_boost_predict_cls failed: {rc}")
    return F, cls


def predict(params: Params, tree: Tree, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    cls = np.empty(n, np.int32)
    val = np.empty(n, np.float64)
    leaf = np.empty(n, np.int32)
    cs = tree._cstruct()
    rc = lib().ora_predict(C.byref(params), C.byref(cs), _ptr(X), n, d, _ptr(cls),
                           _ptr(val), _ptr(leaf))
    if rc:
        raise ValueError(f"ora_predict failed: {rc}")
    return cls, val, leaf


# ---- learned swarm proposal ----------------------------------------------------

def node_stats(X, labels=None, n_classes=0, y=None, idx=None, wts=None) -> np.ndarray:
    """The network input of one node: class-mean offsets and variances."""
    X, labels, y, idx, wts = _node_arrays(X, labels, y, idx, wts)
    out = np.zeros(MLP_IN, np.float64)
    rc = lib().ora_node_stats(_ptr(X), X.shape[1], _ptr(labels), n_classes, _ptr(y),
                              _ptr(idx), _ptr(wts), idx.size, _ptr(out))
    if rc:
        raise ValueError(f"ora_node_stats failed: {rc}")
    return out


def _mlp_struct(m: dict):
    arrs = {k: np.ascontiguousarray(m[k], dtype=np.float64).reshape(MLP_SHAPES[k])
            for k in MLP_SHAPES}
    return _Mlp(*[_ptr(arrs[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]), arrs


def mlp_forward(m: dict, s, bf16=True):
    """Returns (out[n, OUT], h1[n, H], h2[n, H])."""
    st, keep = _mlp_struct(m)
    s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, MLP_IN)
    n = s.shape[0]
    out = np.empty((n, MLP_OUT)); h1 = np.empty((n, MLP_H)); h2 = np.empty((n, MLP_H))
    rc = lib().ora_mlp_forward(C.byref(st), _ptr(s), n, 1 if bf16 else 0, _ptr(h1),
                               _ptr(h2), _ptr(out))
    if rc:
        raise ValueError(f"ora_mlp_forward failed: {rc}")
    return out, h1, h2


def mlp_loss_grad(m: dict, s, dims, a, bf16=True):
    """Mean loss and the gradient of every parameter (dict like m)."""
    st, keep = _mlp_struct(m)
    s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, MLP_IN)
    n = s.shape[0]
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(n, MLP_D)
    g = {k: np.empty(MLP_SHAPES[k]) for k in MLP_SHAPES}
    loss = C.c_double()
    rc = lib().ora_mlp_loss_grad(C.byref(st), _ptr(s), _ptr(dims), _ptr(a), n,
                                 1 if bf16 else 0, C.byref(loss),
                                 *[_ptr(g[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    if rc:
        raise ValueError(f"ora_mlp_loss_grad failed: {rc}")
    return loss.value, g


def adam_step(w, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on float64 arrays, in place; returns (w, m, v)."""
    w, m, v = (np.ascontiguousarray(x, dtype=np.float64) for x in (w, m, v))
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().ora_adam_step(_ptr(w), _ptr(m), _ptr(v), _ptr(g), w.size, t, lr, beta1, beta2, eps)
    return w, m, v


def swarm_seed(seed, node_uid, n_particles, d, mu_hat, rho) -> np.ndarray:
    mu_hat = np.ascontiguousarray(mu_hat, dtype=np.float32)
    rho = np.ascontiguousarray(rho, dtype=np.float32)
    pos = np.empty((n_particles, d), np.float32)
    lib().ora_swarm_seed(seed, node_uid, n_particles, d, _ptr(mu_hat), _ptr(rho), _ptr(pos))
    return pos
