"""Interaction values on the GPU (wdf_explain_interactions) against the oracle's
count-based (and path-dependent) interaction tiers: Shapley (Table table_shap_iv) and
Banzhaf (Formula banzhaf_simplified_formula_interactions), several depths, the shared-
memory and the in-place accumulation paths, at the FP32-mode tolerance."""
import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-6, 1e-5
# (name, seed, n, m, F, n_gauss, T, D, leaf_std, early_leaf_p, complete)
CASES = [("d3", 81, 40, 500, 8, 8, 10, 3, 1.0, 0.0, True),
         ("d6", 82, 24, 3000, 40, 30, 25, 6, 0.1, 0.1, False),
         ("d8", 83, 12, 2000, 24, 16, 6, 8, 0.1, 0.1, False),
         ("wide", 84, 6, 1000, 300, 213, 12, 5, 0.1, 0.1, False)]  # F(F-1)/2 floats exceed the shared budget


@pytest.fixture(scope="module")
def ctx():
    import paper_2511_09376_gb300 as wdf
    return wdf.ctx_create(0)


def _check(got, want, name):
    err = np.abs(got - want)
    bound = ATOL + RTOL * np.abs(want)
    assert (err <= bound).all(), f"{name}: max |err| {err.max():.3e} (max |want| {np.abs(want).max():.3e})"


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("metric", ["shapley", "banzhaf"])
def test_background_interactions_against_oracle(ctx, case, metric):
    import torch

    import paper_2511_09376_gb300 as wdf
    name, seed, n, m, F, ng, T, D, sd, p, comp = case
    ens, C, B = synth.make(synth.Workload(name, seed, n, m, F, ng, T, D, sd, p, comp))
    om = oracle.SHAPLEY if metric == "shapley" else oracle.BANZHAF
    want = oracle.iv_hist(ens, oracle.bg_hist(ens, B), m, C, om)
    e = wdf.load_ensemble(ctx, ens)
    if metric != "shapley":
        wdf.set_metric(e, metric)
    wdf.set_background(e, torch.from_numpy(B).cuda())
    got = wdf.explain_interactions(e, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.float64)
    assert got.shape == (n, F, F)
    _check(got, want, f"{name} {metric}")
    assert np.array_equal(got, got.transpose(0, 2, 1))
    assert not got[:, np.arange(F), np.arange(F)].any()
    assert np.abs(want).max() > 1e-3
    e.close()


def test_path_dependent_interactions_against_oracle(ctx):
    import torch

    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make(synth.Workload("pdiv", 85, 24, 4000, 40, 30, 20, 6, 0.1, 0.1, False))
    cover = synth.node_covers(ens, B)
    want = oracle.pd_iv(ens, cover, C)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_covers(e, cover)
    wdf.set_path_dependent(e)
    got = wdf.explain_interactions(e, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.float64)
    _check(got, want, "path-dependent")


def test_strided_output_and_empty_input(ctx):
    import torch

    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make("tiny")
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, torch.from_numpy(B).cuda())
    F = ens.n_features
    dC = torch.from_numpy(C).cuda()
    base = wdf.explain_interactions(e, dC)
    # rows of the output padded (row stride > F * F): the same values
    big = torch.full((C.shape[0], F * F + 5), -7.0, device="cuda")
    view = big[:, :F * F].view(C.shape[0], F, F)
    wdf.explain_interactions(e, dC, out=view)
    assert torch.equal(view.cpu(), base.cpu()) or np.allclose(view.cpu().numpy(), base.cpu().numpy(), atol=1e-7)
    assert (big[:, F * F:] == -7.0).all()
    empty = wdf.explain_interactions(e, dC[:0])
    assert tuple(empty.shape) == (0, F, F)


def test_interactions_need_a_background(ctx):
    import torch

    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make("tiny")
    e = wdf.load_ensemble(ctx, ens)
    with pytest.raises(wdf.WdfError):
        wdf.explain_interactions(e, torch.from_numpy(C).cuda())
