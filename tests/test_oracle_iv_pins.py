"""Pins of the oracle's interaction-value tiers (section "Beyond SHAP": Def. shap_iv_def,
Table table_shap_iv, Def. banzhaf_iv_def, Formula banzhaf_simplified_formula_interactions)
against values derived by hand, the definitions enumerated, and each other."""
import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

METRICS = [oracle.SHAPLEY, oracle.BANZHAF]


def test_two_literal_cube_by_hand():
    # v(S) = w only when both variables are in: the single difference term has weight 1
    cube = [(3.0, [(0, False), (1, False)])]
    for metric in METRICS:
        want = np.array([[0.0, 3.0], [3.0, 0.0]])
        np.testing.assert_allclose(oracle.wdnf_iv(2, cube, metric), want, atol=1e-15)
        np.testing.assert_allclose(oracle.wdnf_iv_bruteforce(2, cube, metric), want, atol=1e-15)


def test_mixed_cube_by_hand():
    # 4 (x0 and x1 and not x2 and x3): |S+| = 3, |S-| = 1, |S| = 4.
    # Shapley: same sign 4 / (2 C(3,2)) = 2/3; mixed -4 / (1 C(3,1)) = -4/(3 C(3,3)) = -4/3.
    # Banzhaf: +-4 / 2^2 = +-1.
    cube = [(4.0, [(0, False), (1, False), (2, True), (3, False)])]
    s, m = 2.0 / 3.0, -4.0 / 3.0
    shap = np.array([[0, s, m, s], [s, 0, m, s], [m, m, 0, m], [s, s, m, 0]])
    banz = np.array([[0, 1, -1, 1], [1, 0, -1, 1], [-1, -1, 0, -1], [1, 1, -1, 0]], dtype=np.float64)
    for metric, want in ((oracle.SHAPLEY, shap), (oracle.BANZHAF, banz)):
        np.testing.assert_allclose(oracle.wdnf_iv(4, cube, metric), want, atol=1e-15)
        np.testing.assert_allclose(oracle.wdnf_iv_bruteforce(4, cube, metric), want, atol=1e-15)
    # two negated literals: the both-negative cell, 4 / ((2-1) C(2,1)) = 2 for Shapley
    cube = [(4.0, [(0, True), (1, True), (2, False)])]
    assert oracle.wdnf_iv(3, cube)[0, 1] == pytest.approx(2.0)
    assert oracle.wdnf_iv_bruteforce(3, cube)[0, 1] == pytest.approx(2.0)


@pytest.mark.parametrize("metric", METRICS)
def test_closed_forms_match_the_definitions_on_random_wdnfs(metric):
    rng = np.random.default_rng(11 + metric)
    h = 7
    for _ in range(40):
        cubes = []
        for _ in range(int(rng.integers(1, 7))):
            lits = [(int(rng.integers(0, h)), bool(rng.integers(0, 2))) for _ in range(int(rng.integers(1, 6)))]
            cubes.append((float(rng.normal()), lits))  # repeats and contradictions included
        np.testing.assert_allclose(oracle.wdnf_iv(h, cubes, metric), oracle.wdnf_iv_bruteforce(h, cubes, metric),
                                   atol=1e-13)


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("wl", ["tiny", "ragged"])
def test_counts_tier_matches_the_definition_on_trees(metric, wl):
    if wl == "tiny":
        ens, C, B = synth.make("tiny")
        C, B = C[:25], B[:60]
    else:  # ragged depth-5 trees over 7 features: repeated features on paths, early leaves
        ens, C, B = synth.make(synth.Workload("ivr", 77, 25, 60, 7, 5, 12, 5, 0.5, 0.2, False))
    want = oracle.iv_bruteforce(ens, C, B, metric)
    got = oracle.iv_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C, metric)
    np.testing.assert_allclose(got, want, atol=1e-12, rtol=1e-12)
    assert np.abs(want).max() > 0.1
    np.testing.assert_allclose(got, got.transpose(0, 2, 1), atol=1e-14)  # symmetric
    assert not got[:, np.arange(ens.n_features), np.arange(ens.n_features)].any()  # no diagonal


def test_stumps_have_no_interactions():
    # a sum of one-split trees is an additive game: every pair interaction is zero
    ens, C, B = synth.make(synth.Workload("stumps", 78, 20, 50, 6, 6, 15, 1, 1.0, 0.0, True))
    got = oracle.iv_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    assert np.abs(got).max() < 1e-14
    assert np.abs(oracle.iv_bruteforce(ens, C, B)).max() < 1e-13


@pytest.mark.parametrize("metric", METRICS)
def test_path_dependent_frequency_form_matches_the_definition(metric):
    ens, C, B = synth.make(synth.Workload("ivpd", 79, 20, 400, 7, 5, 10, 5, 0.5, 0.2, False))
    cover = synth.node_covers(ens, B)
    want = oracle.pd_iv_bruteforce(ens, cover, C, metric)
    got = oracle.pd_iv(ens, cover, C, metric)
    np.testing.assert_allclose(got, want, atol=1e-12, rtol=1e-12)
    assert np.abs(want).max() > 0.01
