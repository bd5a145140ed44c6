"""Pins for the oracle's path-dependent tiers (section "Efficient Path-Dependent SHAP
Equation"): the worked pattern-5 example of Eq. path_dependent_estimation, the
coalition brute force of the cover-weighted game against the frequency form, and the
efficiency property."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ensemble(F, trees):
    offs, f, th, l, r, v = [0], [], [], [], [], []
    for nodes in trees:
        for (a, b, c, d, e) in nodes:
            f.append(a); th.append(b); l.append(c); r.append(d); v.append(e)
        offs.append(offs[-1] + len(nodes))
    return synth.Ensemble(F, np.array(offs, np.int64), np.array(f, np.int32), np.array(th, np.float32),
                          np.array(l, np.int32), np.array(r, np.int32), np.array(v, np.float32))


def test_pattern_five_example():
    g = json.load(open(os.path.join(GOLD, "path_dependent_pattern_example.json")))
    # n1 -> n2 (left of n1) -> n3 (right of n2) -> n4 (left of n3, the leaf)
    nodes = [(0, 0.0, 1, 2, 0.0), (1, 0.0, 3, 4, 0.0), (-1, 0, -1, -1, 0.0), (-1, 0, -1, -1, 0.0),
             (2, 0.0, 5, 6, 0.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, 0.0)]
    ens = _ensemble(3, [nodes])
    c1, c2, c3, c4 = 100.0, 60.0, 25.0, 10.0
    cover = np.array([c1, c2, 40.0, 35.0, c3, c4, 15.0])
    tree, node, depth, hoff, hs = oracle.leaf_table(ens)
    k = [i for i in range(len(node)) if node[i] == 5][0]
    freq = oracle.pd_freq(ens, cover)
    want = (c2 / c1) * (1.0 - c3 / c2) * (c4 / c3)
    assert g["pattern"] == 5 and depth[k] == g["depth"]
    assert freq[hoff[k] + g["pattern"]] == pytest.approx(want, rel=1e-15)
    assert freq[hoff[k]:hoff[k] + 8].sum() == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("metric", [oracle.SHAPLEY, oracle.BANZHAF])
def test_bruteforce_equals_frequency_form(metric):
    ens, C, B = synth.make("tiny")
    cover = synth.node_covers(ens, B)
    p0, v0 = oracle.pd_values_bruteforce(ens, cover, C[:40], metric)
    p2, base = oracle.pd_values(ens, cover, C[:40], metric)
    np.testing.assert_allclose(p2, p0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v0, base, atol=1e-12)
    if metric == oracle.SHAPLEY:
        np.testing.assert_allclose(p2.sum(axis=1), oracle.predict(ens, C[:40]) - base, atol=1e-9)


def test_ragged_trees_and_zero_cover_nodes():
    w = synth.Workload("pd", 77, 30, 400, 9, 9, 12, 5, 0.5, 0.3, False)
    ens, C, B = synth.make(w)
    cover = synth.node_covers(ens, B[:50])  # few rows: some nodes are never reached
    assert (cover == 0).any()
    p0, v0 = oracle.pd_values_bruteforce(ens, cover, C)
    p2, base = oracle.pd_values(ens, cover, C)
    np.testing.assert_allclose(p2, p0, rtol=0, atol=1e-12)
