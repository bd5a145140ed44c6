"""Every supported depth (2..8, complete and ragged trees) and every contraction
precision (FP32 on CUDA cores; TF32 and BF16 split-precision on tcgen05 tensor cores)
against the FP64 oracle, through the C ABI.  The bar is the FP32-mode tolerance
|gpu - oracle| <= 1e-6 + 1e-5 |oracle| for all four (background counts here stay below
2^16, where the two-part BF16 split is exact for the counts)."""
import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-6, 1e-5

CASES = {
    # name: (seed, n, m, F, n_gauss, T, depth, leaf_std, early_p, complete)
    "d2-complete": (31, 300, 5000, 10, 10, 30, 2, 0.5, 0.0, True),
    "d3-ragged": (32, 200, 6000, 12, 8, 25, 3, 0.5, 0.2, False),
    "d4-complete": (33, 200, 6000, 24, 20, 20, 4, 0.3, 0.0, True),
    "d5-ragged": (34, 200, 6000, 60, 40, 20, 5, 0.2, 0.1, False),
    # depth 6: every one of the 63 nodes real (decision bits 0-62 in record order), and
    # many early leaves (real-node counts on both sides of 32)
    "d6-complete": (37, 200, 6000, 50, 40, 20, 6, 0.2, 0.0, True),
    "d6-ragged": (38, 200, 6000, 50, 40, 40, 6, 0.2, 0.15, False),
    "d7-ragged": (35, 150, 6000, 40, 30, 15, 7, 0.1, 0.1, False),
    "d8-ragged": (36, 150, 6000, 40, 30, 15, 8, 0.1, 0.1, False),
}


@pytest.fixture(scope="module")
def ctx():
    import paper_2511_09376_gb300 as wdf
    return wdf.ctx_create(0)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    seed, n, m, F, ng, T, D, sd, p, complete = CASES[request.param]
    ens, C, B = synth.make(synth.Workload(request.param, seed, n, m, F, ng, T, D, sd, p, complete))
    want = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    return request.param, ens, C, B, want


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3", "bf16x6"])
def test_depths_and_precisions(ctx, case, precision):
    import torch

    import paper_2511_09376_gb300 as wdf
    name, ens, C, B, want = case
    e = wdf.load_ensemble(ctx, ens)
    assert wdf.ensemble_info(e)["depth"] == max(2, ens.max_depth())
    wdf.set_background(e, torch.from_numpy(B).cuda(), precision)
    phi = wdf.explain(e, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.float64)
    err = np.abs(phi - want)
    bound = ATOL + RTOL * np.abs(want)
    assert (err <= bound).all(), f"{name} {precision}: max |err| {err.max():.3e}, worst excess {(err - bound).max():.3e}"
    e.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16x6"])
def test_banzhaf_values(ctx, case, precision):
    """Banzhaf values (Formula banzhaf_simplified_formula in the pattern-pair table)
    against the oracle's Banzhaf tier."""
    import torch

    import paper_2511_09376_gb300 as wdf
    name, ens, C, B, _ = case
    want = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C, oracle.BANZHAF)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_metric(e, "banzhaf")
    wdf.set_background(e, torch.from_numpy(B).cuda(), precision)
    phi = wdf.explain(e, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.float64)
    err = np.abs(phi - want)
    bound = ATOL + RTOL * np.abs(want)
    assert (err <= bound).all(), f"{name} {precision}: max |err| {err.max():.3e}"
    # switching back to Shapley reproduces the Shapley oracle
    wdf.set_metric(e, "shapley")
    wdf.set_background(e, torch.from_numpy(B).cuda(), precision)
    phi = wdf.explain(e, torch.from_numpy(C).cuda()).cpu().numpy().astype(np.float64)
    assert (np.abs(phi - case[4]) <= ATOL + RTOL * np.abs(case[4])).all()
    e.close()
