"""Ragged batches: one graph launch over requests against ensembles of depths 2..8 and
different feature counts gives, row for row, exactly the phi of per-ensemble explain
calls (the per-row arithmetic and its order do not depend on the batch)."""
import numpy as np
import pytest

from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

SPECS = [  # (seed, n, m, F, n_gauss, T, depth, leaf_std, early_p, complete, precision)
    (41, 0, 3000, 20, 20, 12, 2, 0.5, 0.0, True, "fp32"),
    (42, 0, 3000, 33, 20, 20, 4, 0.3, 0.1, False, "bf16x3"),
    (43, 0, 3000, 127, 90, 25, 6, 0.1, 0.1, False, "fp32"),
    (44, 0, 3000, 64, 40, 10, 6, 0.1, 0.1, False, "tf32x3"),
    (45, 0, 3000, 50, 30, 8, 7, 0.1, 0.1, False, "bf16x6"),
    (46, 0, 3000, 300, 200, 6, 8, 0.1, 0.1, False, "fp32"),
]


@pytest.fixture(scope="module")
def setup():
    import torch

    import paper_2511_09376_gb300 as wdf
    ctx = wdf.ctx_create(0)
    ens, rng = [], np.random.default_rng(7)
    for k, (seed, _, m, F, ng, T, D, sd, p, comp, prec) in enumerate(SPECS):
        e_np, _, B = synth.make(synth.Workload(f"b{k}", seed, 1, m, F, ng, T, D, sd, p, comp))
        e = wdf.load_ensemble(ctx, e_np)
        wdf.set_background(e, torch.from_numpy(B).cuda(), prec)
        ens.append(e)
    batch = wdf.batch_create(ctx, ens)
    return wdf, ctx, ens, batch, rng


def _requests(setup, sizes):
    import torch
    wdf, ctx, ens, batch, rng = setup
    reqs = []
    for k, n in sizes:
        F = wdf.ensemble_info(ens[k])["n_features"]
        C = torch.from_numpy(rng.standard_normal((n, F)).astype(np.float32)).cuda()
        reqs.append((k, C))
    return reqs


def _check(setup, reqs, outs):
    import torch
    wdf, ctx, ens, batch, rng = setup
    torch.cuda.synchronize()
    for (k, C), o in zip(reqs, outs):
        want = wdf.explain(ens[k], C)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(o.cpu().numpy(), want.cpu().numpy())


def test_batch_equals_single_calls(setup):
    wdf, ctx, ens, batch, rng = setup
    reqs = _requests(setup, [(0, 1), (1, 130), (2, 517), (3, 0), (4, 64), (5, 65), (2, 3), (0, 999)])
    outs = wdf.batch_explain(batch, reqs)
    _check(setup, reqs, outs)
    # the same graph again with other sizes, then a larger batch that grows the capacity
    reqs2 = _requests(setup, [(5, 7), (1, 2), (3, 300)])
    _check(setup, reqs2, wdf.batch_explain(batch, reqs2))
    reqs3 = _requests(setup, [(k % 6, 2000 + 37 * k) for k in range(18)])
    _check(setup, reqs3, wdf.batch_explain(batch, reqs3))


def test_batch_autotune_keeps_results(setup, tmp_path):
    wdf, ctx, ens, batch, rng = setup
    reqs = _requests(setup, [(k, 3000) for k in range(6)])
    cache = str(tmp_path / "tune.txt")
    wdf.batch_autotune(batch, reqs, reps=2, cache_path=cache)
    for D in (2, 4, 6, 7, 8):
        assert wdf.batch_tile_rows(batch, D) in (32, 64, 128)
    assert wdf.batch_tile_rows(batch, 3) == -1
    lines = open(cache).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 5
    _check(setup, reqs, wdf.batch_explain(batch, reqs))
    # a second tuning reads the cached choices
    before = {D: wdf.batch_tile_rows(batch, D) for D in (2, 4, 6, 7, 8)}
    wdf.batch_autotune(batch, reqs, reps=1, cache_path=cache)
    assert before == {D: wdf.batch_tile_rows(batch, D) for D in (2, 4, 6, 7, 8)}


def test_batch_rejects_bad_requests(setup):
    import torch
    wdf, ctx, ens, batch, rng = setup
    C = torch.zeros((4, 20), device="cuda")
    with pytest.raises(wdf.WdfError):
        wdf.batch_explain(batch, [(6, C)], outs=[torch.zeros((4, 20), device="cuda")])  # no ensemble 6
    with pytest.raises(wdf.WdfError):
        wdf.batch_explain(batch, [(2, C)], outs=[torch.zeros((4, 20), device="cuda")])  # F = 127 > 20
