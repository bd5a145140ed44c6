"""Seeded synthetic workloads shaped like the paper's experiments.

The paper measures on XGBoost regressors of 100 trees of depth 6 trained on the
IEEE-CIS and KDD-Cup-99 tables (section "Experimental Results").  Neither the
datasets nor the trained models are available, so this module draws stand-ins of
the same shape: float32 feature matrices (Gaussian columns plus small integer
category codes stored as float) and random binary decision-tree ensembles whose
thresholds sit at background quantiles.

This module holds none of the method's arithmetic.  It only draws inputs; the CPU
oracle and the CUDA path both consume what it returns.

Tree format (shared by every consumer of an ensemble): trees are stored back to
back; ``tree_offset[t]`` is the index of tree ``t``'s root in the flat node arrays
and ``tree_offset[T]`` the total node count.  Per node: ``feature`` (int32, -1 for a
leaf), ``threshold`` (float32), ``left`` / ``right`` (int32 child indices local to
the tree, -1 for a leaf) and ``value`` (float32 leaf output, 0 for inner nodes).
A row goes left at a node when ``x[feature] < threshold`` (strict).
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

SEED_BASE = 20251109

# Rows of the background used to place thresholds at quantiles.  Sorting every
# column of a multi-million-row background would dominate generation time; the
# first rows of the background are an unbiased sample of the same distribution.
QUANTILE_ROWS = 65536


@dataclasses.dataclass
class Ensemble:
    n_features: int
    tree_offset: np.ndarray  # int64 [T+1]
    feature: np.ndarray      # int32 [N]
    threshold: np.ndarray    # float32 [N]
    left: np.ndarray         # int32 [N]
    right: np.ndarray        # int32 [N]
    value: np.ndarray        # float32 [N]

    @property
    def n_trees(self) -> int:
        return int(self.tree_offset.shape[0] - 1)

    @property
    def n_nodes(self) -> int:
        return int(self.tree_offset[-1])

    def max_depth(self) -> int:
        best = 0
        for t in range(self.n_trees):
            o = int(self.tree_offset[t])
            stack = [(0, 0)]
            while stack:
                v, d = stack.pop()
                if self.feature[o + v] < 0:
                    best = max(best, d)
                else:
                    stack.append((int(self.left[o + v]), d + 1))
                    stack.append((int(self.right[o + v]), d + 1))
        return best


@dataclasses.dataclass
class Workload:
    name: str
    seed: int
    n_consumers: int
    n_background: int
    n_features: int
    n_gauss: int
    n_trees: int
    depth: int
    leaf_std: float
    early_leaf_p: float
    complete: bool


def draw_features(rng: np.random.Generator, rows: int, n_features: int, n_gauss: int) -> np.ndarray:
    """Row-major float32 matrix: ``n_gauss`` N(0,1) columns, then integer codes 0..15."""
    x = np.empty((rows, n_features), dtype=np.float32)
    if n_gauss > 0:
        x[:, :n_gauss] = rng.standard_normal((rows, n_gauss), dtype=np.float32)
    if n_features > n_gauss:
        x[:, n_gauss:] = rng.integers(0, 16, size=(rows, n_features - n_gauss), dtype=np.int32).astype(np.float32)
    return x


def draw_ensemble(rng: np.random.Generator, background: np.ndarray, n_trees: int, depth: int,
                  leaf_std: float, early_leaf_p: float = 0.0, complete: bool = True) -> Ensemble:
    """Random ensemble.  Each inner node splits on a uniform feature at the value found
    at a uniform quantile of that background column.  Nodes are numbered breadth first.
    When ``complete`` is false, a node at depth 1..depth-1 becomes a leaf early with
    probability ``early_leaf_p`` (the root always splits), so leaf depths are ragged.
    """
    n_features = background.shape[1]
    q = min(background.shape[0], QUANTILE_ROWS)
    sorted_cols = np.sort(background[:q], axis=0)
    offs = [0]
    feats, thrs, lefts, rights, vals = [], [], [], [], []
    for _ in range(n_trees):
        f_t, th_t, l_t, r_t, v_t, d_t = [], [], [], [], [], []
        f_t.append(0); th_t.append(0.0); l_t.append(-1); r_t.append(-1); v_t.append(0.0); d_t.append(0)
        head = 0
        while head < len(f_t):
            d = d_t[head]
            leaf = d >= depth or (not complete and d >= 1 and rng.random() < early_leaf_p)
            if leaf:
                f_t[head] = -1
                v_t[head] = float(rng.normal(0.0, leaf_std))
            else:
                f = int(rng.integers(0, n_features))
                u = float(rng.random())
                f_t[head] = f
                th_t[head] = float(sorted_cols[min(int(u * q), q - 1), f])
                for side in (0, 1):
                    child = len(f_t)
                    f_t.append(-1); th_t.append(0.0); l_t.append(-1); r_t.append(-1); v_t.append(0.0)
                    d_t.append(d + 1)
                    if side == 0:
                        l_t[head] = child
                    else:
                        r_t[head] = child
            head += 1
        feats += f_t; thrs += th_t; lefts += l_t; rights += r_t; vals += v_t
        offs.append(offs[-1] + len(f_t))
    return Ensemble(
        n_features=n_features,
        tree_offset=np.asarray(offs, dtype=np.int64),
        feature=np.asarray(feats, dtype=np.int32),
        threshold=np.asarray(thrs, dtype=np.float32),
        left=np.asarray(lefts, dtype=np.int32),
        right=np.asarray(rights, dtype=np.int32),
        value=np.asarray(vals, dtype=np.float32),
    )


# The workloads: k = 1 tiny (complete depth 3, 8 Gaussian features), k = 2 mid and
# k = 3 large (127 features shaped like KDD-Cup-99 after one-hot encoding: 90 Gaussian
# columns and 37 integer codes; ragged depth-6 trees as XGBoost's default depth).
WORKLOADS = {
    "tiny": Workload("tiny", SEED_BASE + 1, 100, 200, 8, 8, 10, 3, 1.0, 0.0, True),
    "mid": Workload("mid", SEED_BASE + 2, 100_000, 100_000, 127, 90, 100, 6, 0.1, 0.1, False),
    "large": Workload("large", SEED_BASE + 3, 3_000_000, 5_000_000, 127, 90, 200, 6, 0.1, 0.1, False),
}


def make(w: Workload | str, n_consumers: int | None = None, n_background: int | None = None,
         n_trees: int | None = None):
    """Draw (ensemble, consumers C, background B) for a workload.

    Overriding the row counts keeps every other draw identical: the ensemble, the
    background and the consumers come from independent child streams of the seed, and
    the first rows drawn for a smaller request equal the first rows of a larger one.
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    n = w.n_consumers if n_consumers is None else n_consumers
    m = w.n_background if n_background is None else n_background
    T = w.n_trees if n_trees is None else n_trees
    s_tree, s_bg, s_cons = np.random.SeedSequence(w.seed).spawn(3)
    B = draw_rows(s_bg, m, w.n_features, w.n_gauss)
    C = draw_rows(s_cons, n, w.n_features, w.n_gauss)
    qsrc = B if m >= QUANTILE_ROWS else draw_rows(s_bg, QUANTILE_ROWS, w.n_features, w.n_gauss)
    ens = draw_ensemble(np.random.Generator(np.random.PCG64(s_tree)), qsrc, T, w.depth,
                        w.leaf_std, w.early_leaf_p, w.complete)
    return ens, C, B


def consumers(w: Workload | str, n: int) -> np.ndarray:
    """The first n consumer rows of a workload: the rows make(w, n_consumers=n) returns,
    without drawing the ensemble or the background."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    _, _, s_cons = np.random.SeedSequence(w.seed).spawn(3)
    return draw_rows(s_cons, n, w.n_features, w.n_gauss)


def node_covers(ens: Ensemble, X: np.ndarray) -> np.ndarray:
    """Cover of every node: how many rows of X reach it (what a trained model records
    for its training rows), indexed like the node arrays, as float64."""
    cover = np.zeros(ens.n_nodes, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float32)
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        node = np.zeros(X.shape[0], dtype=np.int64)
        active = np.ones(X.shape[0], dtype=bool)
        while active.any():
            idx = np.nonzero(active)[0]
            np.add.at(cover, o + node[idx], 1.0)
            f = ens.feature[o + node[idx]]
            leaf = f < 0
            active[idx[leaf]] = False
            inner = idx[~leaf]
            if inner.size == 0:
                break
            fi = ens.feature[o + node[inner]]
            go_left = X[inner, fi] < ens.threshold[o + node[inner]]
            node[inner] = np.where(go_left, ens.left[o + node[inner]], ens.right[o + node[inner]])
    return cover


def _log_uniform(rng, lo, hi):
    return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))


def ragged_specs(seed: int = SEED_BASE + 4, count: int = 64):
    """The ragged batch: `count` ensembles with trees log-uniform in [10, 500], depth
    uniform in 2..8, features uniform in [20, 300] (71 % Gaussian, the rest integer codes,
    the KDD mix), consumers log-uniform in [1e3, 2e5] and background rows log-uniform in
    [1e4, 1e6]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        T = int(round(_log_uniform(rng, 10, 500)))
        D = int(rng.integers(2, 9))
        F = int(rng.integers(20, 301))
        n = int(round(_log_uniform(rng, 1e3, 2e5)))
        m = int(round(_log_uniform(rng, 1e4, 1e6)))
        out.append(Workload(f"ragged{i}", seed * 1000 + i, n, m, F, int(round(0.71 * F)), T, D, 0.1, 0.1, False))
    return out


def serving_specs(seed: int = SEED_BASE + 5):
    """The serving set: four resident ensembles (50, 200, 500, 1000 trees of depths 4, 6, 7,
    8), features drawn uniformly in [50, 500], 1e6-row backgrounds."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (T, D) in enumerate([(50, 4), (200, 6), (500, 7), (1000, 8)]):
        F = int(rng.integers(50, 501))
        out.append(Workload(f"serve{i}", seed * 1000 + i, 0, 1_000_000, F, int(round(0.71 * F)), T, D, 0.1, 0.1,
                            False))
    return out


def request_stream(seed: int, rate_per_s: float, duration_s: float, n_ensembles: int, n_lo=1, n_hi=100_000):
    """Poisson arrivals: (arrival time in s, ensemble index, consumer rows log-uniform)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            return out
        out.append((t, int(rng.integers(0, n_ensembles)), int(round(_log_uniform(rng, n_lo, n_hi)))))


_CHUNK = 1 << 16


def draw_rows(seed_seq: np.random.SeedSequence, rows: int, n_features: int, n_gauss: int) -> np.ndarray:
    """Rows drawn in fixed chunks of 65,536 from per-chunk child streams, so a prefix
    of a long draw equals a short draw and the chunks are drawn in parallel threads
    (numpy's generators release the GIL while filling arrays)."""
    out = np.empty((rows, n_features), dtype=np.float32)
    n_chunks = max(1, math.ceil(rows / _CHUNK))
    kids = np.random.SeedSequence(seed_seq.entropy, spawn_key=seed_seq.spawn_key).spawn(n_chunks)

    def chunk(i):
        lo, hi = i * _CHUNK, min(rows, (i + 1) * _CHUNK)
        if hi > lo:
            out[lo:hi] = draw_features(np.random.Generator(np.random.PCG64(kids[i])), hi - lo, n_features, n_gauss)

    if n_chunks == 1:
        chunk(0)
    else:
        with ThreadPoolExecutor(max_workers=min(n_chunks, os.cpu_count() or 1, 16)) as ex:
            list(ex.map(chunk, range(n_chunks)))
    return out
