"""Pins for the CPU oracle: it is checked against what the paper prints and what the
mathematics fixes, never against itself.

* the worked WDNF example of Appendix B (Tables banzhaf_calc_example and
  shapley_calc_example), per cube and in total, and the equivalent WDNF printed after
  Corollary robust_DNF;
* the exponential definitions (Eq. PB_shap / PB_banzhaf) against the linear-time
  formulas on random WDNFs with repeated and contradictory literals;
* on tree ensembles: the three tiers O0 (coalition brute force), O1 (per pair) and O2
  (per counted background pattern) against each other, the efficiency property, the
  closed form of a stump, the null player, symmetry, consumer == background, m = 1;
* the background counts against a direct evaluation of Def. decision_pattern, their
  sums, the sibling property, and the root-first bit order of the path-dependent
  example.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _cubes(spec):
    return [(float(w), [(int(v), bool(n)) for v, n in lits]) for w, lits in spec]


def _frac(pairs):
    return np.array([float(Fraction(a, b)) for a, b in pairs])


# ------------------------------------------------------------------ WDNF level

def test_worked_example_shapley_total_and_per_cube():
    g = _gold("wdnf_worked_example.json")
    psi = _cubes(g["psi"])
    np.testing.assert_allclose(oracle.wdnf_values(3, psi, oracle.SHAPLEY), _frac(g["shapley_total"]), rtol=0, atol=1e-15)
    for k, cube in enumerate(psi):
        np.testing.assert_allclose(oracle.wdnf_values(3, [cube], oracle.SHAPLEY), _frac(g["shapley_per_cube"][k]),
                                   rtol=0, atol=1e-15)
    # efficiency as printed under the Shapley table
    assert oracle.wdnf_values(3, psi).sum() == pytest.approx(float(Fraction(*g["psi_all_ones_minus_all_zeros"])), abs=1e-14)


def test_worked_example_banzhaf_total_and_per_cube():
    g = _gold("wdnf_worked_example.json")
    psi = _cubes(g["psi"])
    np.testing.assert_allclose(oracle.wdnf_values(3, psi, oracle.BANZHAF), _frac(g["banzhaf_total"]), rtol=0, atol=1e-15)
    for k, cube in enumerate(psi):
        np.testing.assert_allclose(oracle.wdnf_values(3, [cube], oracle.BANZHAF), _frac(g["banzhaf_per_cube"][k]),
                                   rtol=0, atol=1e-15)


def test_exponential_definitions_reproduce_the_tables():
    g = _gold("wdnf_worked_example.json")
    psi = _cubes(g["psi"])
    np.testing.assert_allclose(oracle.wdnf_values_bruteforce(3, psi, oracle.SHAPLEY), _frac(g["shapley_total"]), atol=1e-14)
    np.testing.assert_allclose(oracle.wdnf_values_bruteforce(3, psi, oracle.BANZHAF), _frac(g["banzhaf_total"]), atol=1e-14)


def test_equivalent_wdnf_is_robust():
    g = _gold("wdnf_worked_example.json")
    psi, alt = _cubes(g["psi"]), _cubes(g["psi_equivalent"])
    for a in range(8):
        x = [(a >> i) & 1 for i in range(3)]
        assert oracle.wdnf_eval(3, psi, x) == oracle.wdnf_eval(3, alt, x)
    for metric, key in ((oracle.SHAPLEY, "shapley_total"), (oracle.BANZHAF, "banzhaf_total")):
        np.testing.assert_allclose(oracle.wdnf_values(3, alt, metric), _frac(g[key]), atol=1e-14)


def test_wdnf_evaluation_example():
    g = _gold("wdnf_worked_example.json")["eval_example"]
    assert oracle.wdnf_eval(3, _cubes(g["cubes"]), g["x"]) == g["value"]


@pytest.mark.parametrize("seed", range(6))
def test_linear_formulas_equal_definitions_on_random_wdnf(seed):
    rng = np.random.default_rng(1000 + seed)
    h = 7
    cubes = []
    for _ in range(12):
        k = int(rng.integers(0, 6))
        lits = [(int(rng.integers(0, h)), bool(rng.integers(0, 2))) for _ in range(k)]
        cubes.append((float(rng.normal()), lits))
    for metric in (oracle.SHAPLEY, oracle.BANZHAF):
        np.testing.assert_allclose(oracle.wdnf_values(h, cubes, metric), oracle.wdnf_values_bruteforce(h, cubes, metric),
                                   rtol=0, atol=1e-12)


# ------------------------------------------------------------------ pattern-pair cubes

@pytest.mark.parametrize("D", [3, 6])
def test_pair_cube_counts_and_per_cube_efficiency(D):
    feats = list(range(10, 10 + D))
    n_ok = n_nz = 0
    for pc in range(1 << D):
        for pb in range(1 << D):
            ok, vals = oracle.path_cube(feats, pc, pb, 10 + D)
            has_bottom = ((pc | pb) != (1 << D) - 1)
            assert ok == (not has_bottom)
            if not ok:
                assert not vals.any()
                continue
            n_ok += 1
            n_nz += int(np.count_nonzero(vals))
            s_plus = any(((pc >> i) & 1) and not ((pb >> i) & 1) for i in range(D))
            s_minus = any(not ((pc >> i) & 1) and ((pb >> i) & 1) for i in range(D))
            assert vals.sum() == pytest.approx(float(not s_minus) - float(not s_plus), abs=1e-14)
    assert n_ok == 3 ** D
    assert n_nz == 2 * D * 3 ** (D - 1)


def test_pair_cube_repeated_feature_is_a_set():
    # path features (5, 7, 5); bits root first
    ok, v = oracle.path_cube([5, 7, 5], 0b101, 0b011, 8)   # (1,0) f5, (0,1) f7, (1,1)
    assert ok and v[5] == 0.5 and v[7] == -0.5
    ok, v = oracle.path_cube([5, 7, 5], 0b110, 0b011, 8)   # +5, (1,1), then (0,1) on 5 -> contradiction
    assert not ok and not v.any()
    ok, v = oracle.path_cube([5, 7, 5], 0b111, 0b010, 8)   # +5 twice -> S+ = {5}
    assert ok and v[5] == 1.0 and np.count_nonzero(v) == 1


# ------------------------------------------------------------------ tree ensembles

def _ensemble(F, trees):
    """trees: list of node lists (feature, threshold, left, right, value), root first."""
    offs, f, th, l, r, v = [0], [], [], [], [], []
    for nodes in trees:
        for (a, b, c, d, e) in nodes:
            f.append(a); th.append(b); l.append(c); r.append(d); v.append(e)
        offs.append(offs[-1] + len(nodes))
    return synth.Ensemble(F, np.array(offs, np.int64), np.array(f, np.int32), np.array(th, np.float32),
                          np.array(l, np.int32), np.array(r, np.int32), np.array(v, np.float32))


@pytest.fixture(scope="module")
def tiny():
    return synth.make("tiny")


def test_three_tiers_agree_on_tiny(tiny):
    ens, C, B = tiny
    p0, v0 = oracle.values_bruteforce(ens, C, B)
    p1, base = oracle.values_pairs(ens, C, B)
    counts = oracle.bg_hist(ens, B)
    p2 = oracle.values_hist(ens, counts, B.shape[0], C)
    np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p2, p0, rtol=0, atol=1e-12)
    fb = oracle.predict(ens, B).mean()
    assert base == pytest.approx(fb, abs=1e-12)
    assert oracle.base_from_hist(ens, counts, B.shape[0]) == pytest.approx(fb, abs=1e-12)
    np.testing.assert_allclose(v0, fb, atol=1e-12)


@pytest.mark.parametrize("metric", [oracle.SHAPLEY, oracle.BANZHAF])
def test_efficiency_and_banzhaf_brute_force(tiny, metric):
    ens, C, B = tiny
    B3 = B[:3]  # the paper checks Banzhaf on 100 consumers x 3 background rows
    p0, _ = oracle.values_bruteforce(ens, C, B3, metric)
    p2 = oracle.values_hist(ens, oracle.bg_hist(ens, B3), 3, C, metric)
    np.testing.assert_allclose(p2, p0, rtol=0, atol=1e-12)
    if metric == oracle.SHAPLEY:
        eff = oracle.predict(ens, C) - oracle.predict(ens, B3).mean()
        np.testing.assert_allclose(p2.sum(axis=1), eff, atol=1e-9)


def test_efficiency_mid_slice():
    ens, C, B = synth.make("mid", n_consumers=40, n_background=3000, n_trees=30)
    counts = oracle.bg_hist(ens, B)
    p2 = oracle.values_hist(ens, counts, B.shape[0], C)
    p1, base = oracle.values_pairs(ens, C, B)
    np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-12)
    eff = oracle.predict(ens, C) - base
    np.testing.assert_allclose(p2.sum(axis=1), eff, atol=1e-9)


def test_stump_closed_form():
    theta, wl, wr = 0.25, 1.5, -0.75
    ens = _ensemble(3, [[(1, theta, 1, 2, 0.0), (-1, 0, -1, -1, wl), (-1, 0, -1, -1, wr)]])
    rng = np.random.default_rng(7)
    B = rng.standard_normal((50, 3)).astype(np.float32)
    B[:5, 1] = theta  # ties go right
    C = rng.standard_normal((20, 3)).astype(np.float32)
    C[0, 1] = theta
    qL = float(np.mean(B[:, 1] < theta)); qR = 1.0 - qL
    want = wl * ((C[:, 1] < theta) - qL) + wr * ((C[:, 1] >= theta) - qR)
    p2 = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    np.testing.assert_allclose(p2[:, 1], want, atol=1e-12)
    assert not p2[:, [0, 2]].any()


def test_null_player_consumer_equals_background_and_single_baseline(tiny):
    ens, C, B = tiny
    F = ens.n_features
    used = set(int(f) for f in ens.feature if f >= 0)
    # a feature no tree splits on gets exactly zero
    ens2 = _ensemble(F + 2, [[(0, 0.0, 1, 2, 0.0), (-1, 0, -1, -1, 1.0), (3, 0.5, 3, 4, 0.0),
                              (-1, 0, -1, -1, -2.0), (-1, 0, -1, -1, 0.5)]])
    rng = np.random.default_rng(3)
    C2 = rng.standard_normal((10, F + 2)).astype(np.float32)
    B2 = rng.standard_normal((30, F + 2)).astype(np.float32)
    p = oracle.values_hist(ens2, oracle.bg_hist(ens2, B2), 30, C2)
    assert not p[:, [1, 2] + list(range(4, F + 2))].any()
    # consumer identical to every background row: nothing to attribute
    Bc = np.repeat(C[:1], 7, axis=0)
    p = oracle.values_hist(ens, oracle.bg_hist(ens, Bc), 7, C[:1])
    assert np.abs(p).max() < 1e-14
    # m = 1 is Baseline SHAP, compared with the coalition definition
    p0, _ = oracle.values_bruteforce(ens, C[:10], B[:1])
    p2 = oracle.values_hist(ens, oracle.bg_hist(ens, B[:1]), 1, C[:10])
    np.testing.assert_allclose(p2, p0, atol=1e-12)
    assert used  # the tiny ensemble does split


def test_symmetric_players_get_equal_values():
    t1 = [(0, 0.0, 1, 2, 0.0), (1, 0.5, 3, 4, 0.0), (-1, 0, -1, -1, 3.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, -2.0)]
    t2 = [(1, 0.0, 1, 2, 0.0), (0, 0.5, 3, 4, 0.0), (-1, 0, -1, -1, 3.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, -2.0)]
    ens = _ensemble(3, [t1, t2])
    rng = np.random.default_rng(11)
    half = rng.standard_normal((40, 3)).astype(np.float32)
    B = np.concatenate([half, half[:, [1, 0, 2]]])
    C = rng.standard_normal((15, 3)).astype(np.float32)
    C[:, 1] = C[:, 0]
    p = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    np.testing.assert_allclose(p[:, 0], p[:, 1], atol=1e-13)
    assert np.abs(p[:, 0]).max() > 1e-3


# ------------------------------------------------------------------ background counts

def _paths(ens):
    out = []
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        stack = [(0, [], [])]
        while stack:
            v, nodes, left = stack.pop()
            if ens.feature[o + v] < 0:
                out.append((t, v, nodes, left))
            else:
                stack.append((int(ens.right[o + v]), nodes + [v], left + [0]))
                stack.append((int(ens.left[o + v]), nodes + [v], left + [1]))
    return out


def test_counts_match_direct_decision_patterns(tiny):
    ens, _, B = tiny
    tree, node, depth, hoff, hs = oracle.leaf_table(ens)
    counts = oracle.bg_hist(ens, B)
    index = {(int(t), int(v)): (int(d), int(h)) for t, v, d, h in zip(tree, node, depth, hoff)}
    for (t, v, nodes, left) in _paths(ens):
        o = int(ens.tree_offset[t])
        D, h = index[(t, v)]
        want = np.zeros(1 << D, np.uint64)
        for b in B:
            p = 0
            for n, gl in zip(nodes, left):  # Def. decision_pattern, root first
                goes_left = bool(b[ens.feature[o + n]] < ens.threshold[o + n])
                p = (p << 1) | int(goes_left == bool(gl))
            want[p] += 1
        np.testing.assert_array_equal(counts[h:h + (1 << D)], want)


def test_count_sums_and_siblings():
    ens, _, B = synth.make("mid", n_consumers=1, n_background=5000, n_trees=20)
    tree, node, depth, hoff, hs = oracle.leaf_table(ens)
    counts = oracle.bg_hist(ens, B)
    m = B.shape[0]
    reach = np.zeros(ens.n_trees, np.int64)
    by_node = {}
    for t, v, d, h in zip(tree, node, depth, hoff):
        c = counts[h:h + (1 << d)]
        assert int(c.sum()) == m
        reach[t] += int(c[(1 << d) - 1])
        by_node[(int(t), int(v))] = c
    assert (reach == m).all()
    n_pairs = 0
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        for v in range(int(ens.tree_offset[t + 1] - o)):
            if ens.feature[o + v] < 0:
                continue
            a, b = int(ens.left[o + v]), int(ens.right[o + v])
            if (t, a) in by_node and (t, b) in by_node:
                ca, cb = by_node[(t, a)], by_node[(t, b)]
                np.testing.assert_array_equal(cb, ca[np.arange(ca.size) ^ 1])
                n_pairs += 1
    assert n_pairs > 100


def test_pattern_bit_order_root_first():
    g = _gold("path_dependent_pattern_example.json")
    # path n1 -> n2 (left of n1) -> n3 (right of n2) -> n4 (left of n3, the leaf)
    nodes = [(0, 0.0, 1, 2, 0.0),           # n1
             (1, 0.0, 3, 4, 0.0),           # n2 = n1.left
             (-1, 0, -1, -1, 0.0),
             (-1, 0, -1, -1, 0.0),
             (2, 0.0, 5, 6, 0.0),           # n3 = n2.right
             (-1, 0, -1, -1, 1.0),          # n4 = n3.left
             (-1, 0, -1, -1, 0.0)]
    ens = _ensemble(3, [nodes])
    # follows at n1 (goes left), leaves at n2 (goes left, not right), follows at n3 (goes left)
    row = np.array([[-1.0, -1.0, -1.0]], np.float32)
    tree, node, depth, hoff, hs = oracle.leaf_table(ens)
    k = [i for i in range(len(node)) if node[i] == 5][0]
    assert depth[k] == g["depth"]
    counts = oracle.bg_hist(ens, row)
    assert counts[hoff[k] + g["pattern"]] == 1
    assert int(counts[hoff[k]:hoff[k] + 8].sum()) == 1
