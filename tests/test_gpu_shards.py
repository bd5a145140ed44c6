"""The background in shards (wdf_background_counts + wdf_set_background_counts): the
counts of disjoint row shards add up to the counts of all rows (Eq. bg_shap_derivation
step (d) is a sum over background rows), so finishing from summed shard counts gives
exactly what one wdf_set_background call gives."""
import numpy as np
import pytest

from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2511_09376_gb300 as wdf
    return wdf.ctx_create(0)


@pytest.mark.parametrize("name,cut", [("mid", [0, 777, 40000, 100000]), ("tiny", [0, 1, 200])])
def test_summed_shard_counts_equal_one_call(ctx, name, cut):
    import torch

    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make(name, n_consumers=3000 if name == "mid" else None)
    dB, dC = torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda()
    whole = wdf.load_ensemble(ctx, ens)
    wdf.set_background(whole, dB)
    parts = wdf.load_ensemble(ctx, ens)
    counts = None
    for a, b in zip(cut[:-1], cut[1:]):  # uneven shards, one of a single row
        counts = wdf.background_counts(parts, dB[a:b], counts)
    wdf.set_background_counts(parts, counts, B.shape[0])
    assert np.array_equal(wdf.debug_leaf_hist(parts), wdf.debug_leaf_hist(whole))
    assert torch.equal(wdf.explain(parts, dC), wdf.explain(whole, dC))
    assert wdf.expected_value(parts) == wdf.expected_value(whole)


def test_shard_validation(ctx):
    import torch

    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make("tiny")
    e = wdf.load_ensemble(ctx, ens)
    dB = torch.from_numpy(B).cuda()
    with pytest.raises(ValueError):  # counts of the wrong size
        wdf.background_counts(e, dB, torch.zeros(3, dtype=torch.int32, device="cuda"))
    counts = wdf.background_counts(e, dB)
    with pytest.raises(wdf.WdfError):
        wdf.set_background_counts(e, counts, 0)
