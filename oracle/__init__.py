"""Plain FP64 CPU oracle for Background SHAP / Banzhaf values on tree ensembles.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA path and never consumes anything the CUDA path
produced.  The arithmetic lives in ``woodelf_oracle.c`` (see its header for the
three tiers O0 / O1 / O2 and the paper passages each one follows); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "woodelf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SHAPLEY = 0
BANZHAF = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ens_args(ens):
    return [ctypes.c_int32(ens.n_trees), _p(ens.tree_offset), _p(ens.feature), _p(ens.threshold),
            _p(ens.left), _p(ens.right), _p(ens.value)]


def _rows(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    return x, x.shape[0], x.shape[1]


def threads() -> int:
    return int(_load().orc_num_threads())


def predict(ens, X) -> np.ndarray:
    lib = _load()
    X, n, ld = _rows(X)
    out = np.zeros(n, dtype=np.float64)
    lib.orc_predict(*_ens_args(ens), _p(X), ctypes.c_int64(n), ctypes.c_int64(ld), _p(out))
    return out


def leaf_table(ens):
    """(tree, local node, depth, count offset) of every leaf, tree by tree, depth first."""
    lib = _load()
    lib.orc_leaf_count.restype = ctypes.c_int64
    lib.orc_leaf_table.restype = ctypes.c_int64
    nl = lib.orc_leaf_count(*_ens_args(ens))
    if nl < 0:
        raise ValueError("malformed ensemble")
    tree = np.zeros(nl, np.int32); node = np.zeros(nl, np.int32)
    depth = np.zeros(nl, np.int32); hoff = np.zeros(nl, np.int64)
    hs = lib.orc_leaf_table(*_ens_args(ens), _p(tree), _p(node), _p(depth), _p(hoff))
    return tree, node, depth, hoff, int(hs)


def bg_hist(ens, B) -> np.ndarray:
    """Exact per-leaf background pattern counts (uint64), leaf_table order."""
    lib = _load()
    lib.orc_hist_size.restype = ctypes.c_int64
    hs = lib.orc_hist_size(*_ens_args(ens))
    B, m, ld = _rows(B)
    counts = np.zeros(hs, dtype=np.uint64)
    rc = lib.orc_bg_hist(*_ens_args(ens), _p(B), ctypes.c_int64(m), ctypes.c_int64(ld), _p(counts))
    if rc:
        raise RuntimeError("orc_bg_hist failed")
    return counts


def values_hist(ens, counts, m, C, metric=SHAPLEY) -> np.ndarray:
    """O2: values from exact background counts (Eq. bg_shap_derivation (c)-(d))."""
    lib = _load()
    C, n, ld = _rows(C)
    F = ens.n_features
    phi = np.zeros((n, F), dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    rc = lib.orc_values_hist(*_ens_args(ens), ctypes.c_int32(F), _p(counts), ctypes.c_int64(m),
                             _p(C), ctypes.c_int64(n), ctypes.c_int64(ld), ctypes.c_int32(metric), _p(phi))
    if rc:
        raise RuntimeError("orc_values_hist failed")
    return phi


def base_from_hist(ens, counts, m) -> float:
    lib = _load()
    out = ctypes.c_double(0.0)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    lib.orc_base_from_hist(*_ens_args(ens), _p(counts), ctypes.c_int64(m), ctypes.byref(out))
    return out.value


def values_pairs(ens, C, B, metric=SHAPLEY):
    """O1: Eq. trival_bg, one cube per (consumer, background row, leaf).  Returns (phi, base)."""
    lib = _load()
    C, n, ldc = _rows(C)
    B, m, ldb = _rows(B)
    F = ens.n_features
    phi = np.zeros((n, F), dtype=np.float64)
    base = ctypes.c_double(0.0)
    rc = lib.orc_values_pairs(*_ens_args(ens), ctypes.c_int32(F), _p(C), ctypes.c_int64(n), ctypes.c_int64(ldc),
                              _p(B), ctypes.c_int64(m), ctypes.c_int64(ldb), ctypes.c_int32(metric), _p(phi),
                              ctypes.byref(base))
    if rc:
        raise RuntimeError("orc_values_pairs failed")
    return phi, base.value


def values_bruteforce(ens, C, B, metric=SHAPLEY):
    """O0: the game definition over all 2^F coalitions.  Returns (phi, v_empty per consumer)."""
    lib = _load()
    C, n, ldc = _rows(C)
    B, m, ldb = _rows(B)
    F = ens.n_features
    phi = np.zeros((n, F), dtype=np.float64)
    vempty = np.zeros(n, dtype=np.float64)
    rc = lib.orc_values_bruteforce(*_ens_args(ens), ctypes.c_int32(F), _p(C), ctypes.c_int64(n), ctypes.c_int64(ldc),
                                   _p(B), ctypes.c_int64(m), ctypes.c_int64(ldb), ctypes.c_int32(metric),
                                   _p(phi), _p(vempty))
    if rc:
        raise RuntimeError("orc_values_bruteforce failed")
    return phi, vempty


def _wdnf_arrays(cubes):
    """cubes: list of (weight, [(var, negated), ...])."""
    w = np.array([c[0] for c in cubes], dtype=np.float64)
    off = np.zeros(len(cubes) + 1, dtype=np.int64)
    var, neg = [], []
    for k, (_, lits) in enumerate(cubes):
        for v, ng in lits:
            var.append(v); neg.append(1 if ng else 0)
        off[k + 1] = len(var)
    return w, off, np.array(var, dtype=np.int32), np.array(neg, dtype=np.uint8)


def wdnf_eval(h, cubes, x) -> float:
    lib = _load()
    w, off, var, neg = _wdnf_arrays(cubes)
    xv = np.ascontiguousarray(x, dtype=np.uint8)
    out = ctypes.c_double(0.0)
    lib.orc_wdnf_eval(ctypes.c_int32(h), ctypes.c_int32(len(cubes)), _p(w), _p(off), _p(var), _p(neg), _p(xv),
                      ctypes.byref(out))
    return out.value


def wdnf_values(h, cubes, metric=SHAPLEY) -> np.ndarray:
    lib = _load()
    w, off, var, neg = _wdnf_arrays(cubes)
    phi = np.zeros(h, dtype=np.float64)
    rc = lib.orc_wdnf_values(ctypes.c_int32(h), ctypes.c_int32(len(cubes)), _p(w), _p(off), _p(var), _p(neg),
                             ctypes.c_int32(metric), _p(phi))
    if rc:
        raise RuntimeError("orc_wdnf_values failed")
    return phi


def wdnf_values_bruteforce(h, cubes, metric=SHAPLEY) -> np.ndarray:
    lib = _load()
    w, off, var, neg = _wdnf_arrays(cubes)
    phi = np.zeros(h, dtype=np.float64)
    rc = lib.orc_wdnf_values_bruteforce(ctypes.c_int32(h), ctypes.c_int32(len(cubes)), _p(w), _p(off), _p(var),
                                        _p(neg), ctypes.c_int32(metric), _p(phi))
    if rc:
        raise RuntimeError("orc_wdnf_values_bruteforce failed")
    return phi


def path_cube(feats, pc, pb, n_out, metric=SHAPLEY):
    """Unit-weight value of the cube of pattern pair (pc, pb) on a path; (ok, per-feature values)."""
    lib = _load()
    f = np.ascontiguousarray(feats, dtype=np.int32)
    out = np.zeros(n_out, dtype=np.float64)
    rc = lib.orc_path_cube(ctypes.c_int32(len(f)), _p(f), ctypes.c_uint64(pc), ctypes.c_uint64(pb),
                           ctypes.c_int32(metric), _p(out), ctypes.c_int32(n_out))
    if rc < 0:
        raise ValueError("feature id out of range")
    return bool(rc), out


def _cover(ens, cover):
    cv = np.ascontiguousarray(cover, dtype=np.float64)
    if cv.shape[0] != ens.n_nodes:
        raise ValueError("one cover per node")
    return cv


def pd_values_bruteforce(ens, cover, C, metric=SHAPLEY):
    """O0 of the path-dependent game.  Returns (phi, v_empty per consumer)."""
    lib = _load()
    C, n, ldc = _rows(C)
    F = ens.n_features
    phi = np.zeros((n, F), dtype=np.float64)
    vempty = np.zeros(n, dtype=np.float64)
    cv = _cover(ens, cover)
    rc = lib.orc_pd_values_bruteforce(*_ens_args(ens), _p(cv), ctypes.c_int32(F), _p(C), ctypes.c_int64(n),
                                      ctypes.c_int64(ldc), ctypes.c_int32(metric), _p(phi), _p(vempty))
    if rc:
        raise RuntimeError("orc_pd_values_bruteforce failed")
    return phi, vempty


def pd_values(ens, cover, C, metric=SHAPLEY):
    """O2 of the path-dependent game (Eq. path_dependent_estimation).  Returns (phi, base)."""
    lib = _load()
    C, n, ldc = _rows(C)
    F = ens.n_features
    phi = np.zeros((n, F), dtype=np.float64)
    base = ctypes.c_double(0.0)
    cv = _cover(ens, cover)
    rc = lib.orc_pd_values(*_ens_args(ens), _p(cv), ctypes.c_int32(F), _p(C), ctypes.c_int64(n), ctypes.c_int64(ldc),
                           ctypes.c_int32(metric), _p(phi), ctypes.byref(base))
    if rc:
        raise RuntimeError("orc_pd_values failed")
    return phi, base.value


def pd_freq(ens, cover) -> np.ndarray:
    """Path-dependent frequencies of every leaf's baseline patterns, leaf_table order."""
    lib = _load()
    lib.orc_hist_size.restype = ctypes.c_int64
    hs = lib.orc_hist_size(*_ens_args(ens))
    out = np.zeros(hs, dtype=np.float64)
    lib.orc_pd_freq(*_ens_args(ens), _p(_cover(ens, cover)), _p(out))
    return out


def wdnf_iv(h, cubes, metric=SHAPLEY) -> np.ndarray:
    """Interaction values of a WDNF by the per-cube closed forms (h x h, diagonal 0)."""
    lib = _load()
    w, off, var, neg = _wdnf_arrays(cubes)
    out = np.zeros((h, h), dtype=np.float64)
    rc = lib.orc_wdnf_iv(ctypes.c_int32(h), ctypes.c_int32(len(cubes)), _p(w), _p(off), _p(var), _p(neg),
                         ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_wdnf_iv failed")
    return out


def wdnf_iv_bruteforce(h, cubes, metric=SHAPLEY) -> np.ndarray:
    """Interaction values of a WDNF by the definitions (all assignments of the others)."""
    lib = _load()
    w, off, var, neg = _wdnf_arrays(cubes)
    out = np.zeros((h, h), dtype=np.float64)
    rc = lib.orc_wdnf_iv_bruteforce(ctypes.c_int32(h), ctypes.c_int32(len(cubes)), _p(w), _p(off), _p(var),
                                    _p(neg), ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_wdnf_iv_bruteforce failed")
    return out


def iv_bruteforce(ens, C, B, metric=SHAPLEY) -> np.ndarray:
    """Interaction values of the background game by the definitions (n x F x F)."""
    lib = _load()
    C, n, ldc = _rows(C)
    B, m, ldb = _rows(B)
    F = ens.n_features
    out = np.zeros((n, F, F), dtype=np.float64)
    rc = lib.orc_iv_bruteforce(*_ens_args(ens), ctypes.c_int32(F), _p(C), ctypes.c_int64(n), ctypes.c_int64(ldc),
                               _p(B), ctypes.c_int64(m), ctypes.c_int64(ldb), ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_iv_bruteforce failed")
    return out


def iv_hist(ens, counts, m, C, metric=SHAPLEY) -> np.ndarray:
    """Interaction values from exact background counts (n x F x F)."""
    lib = _load()
    C, n, ld = _rows(C)
    F = ens.n_features
    out = np.zeros((n, F, F), dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    rc = lib.orc_iv_hist(*_ens_args(ens), ctypes.c_int32(F), _p(counts), ctypes.c_int64(m),
                         _p(C), ctypes.c_int64(n), ctypes.c_int64(ld), ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_iv_hist failed")
    return out


def pd_iv(ens, cover, C, metric=SHAPLEY) -> np.ndarray:
    """Path-dependent interaction values, frequency form (n x F x F)."""
    lib = _load()
    C, n, ld = _rows(C)
    F = ens.n_features
    out = np.zeros((n, F, F), dtype=np.float64)
    rc = lib.orc_pd_iv(*_ens_args(ens), _p(_cover(ens, cover)), ctypes.c_int32(F), _p(C), ctypes.c_int64(n),
                       ctypes.c_int64(ld), ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_pd_iv failed")
    return out


def pd_iv_bruteforce(ens, cover, C, metric=SHAPLEY) -> np.ndarray:
    """Path-dependent interaction values by the definitions over all coalitions (n x F x F)."""
    lib = _load()
    C, n, ld = _rows(C)
    F = ens.n_features
    out = np.zeros((n, F, F), dtype=np.float64)
    rc = lib.orc_pd_iv_bruteforce(*_ens_args(ens), _p(_cover(ens, cover)), ctypes.c_int32(F), _p(C),
                                  ctypes.c_int64(n), ctypes.c_int64(ld), ctypes.c_int32(metric), _p(out))
    if rc:
        raise RuntimeError("orc_pd_iv_bruteforce failed")
    return out
