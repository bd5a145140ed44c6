"""Oracle parity of every workload at its full size, launched as the benchmark launches it.

- mid (100,000 consumers x 100,000 background rows, 127 features, 100 depth-6 trees):
  every consumer row against the count-regrouped FP64 oracle.
- ragged batch (64 ensembles, trees 10-500, depth 2-8, features 20-300, up to 2e5
  consumers and 1e6 background rows each): one autotuned batch launch with the BF16
  hi+mid+lo contraction, 1,000 sampled rows per ensemble (every depth class, the first
  tile, tile seams and the last rows of every request) against the oracle.
- serving (4 resident ensembles of 50/200/500/1000 trees, depths 4/6/7/8, 1e6-row
  backgrounds): requests of mixed sizes through the continuous-batching server, sampled
  rows (part seams of 8,192 rows included) against the oracle.

The bar is the FP32-mode tolerance |gpu - oracle| <= 1e-6 + 1e-5 |oracle| (the batched
and served forms compute in the same stated accuracy as the plain path: Algorithm 3 and
Eq. "bg_shap_derivation" do not depend on how the rows are batched).
"""
import numpy as np
import pytest

import oracle
from conftest import assert_phi_close
from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

SPLIT = "bf16x6"  # the batched and served forms' contraction (FP32 accuracy)


@pytest.fixture(scope="module")
def wdf():
    import paper_2511_09376_gb300 as w
    return w


@pytest.fixture(scope="module")
def ctx(wdf):
    return wdf.ctx_create(0)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def test_mid_every_consumer(wdf, ctx):
    import torch
    ens, C, B = synth.make("mid")
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B))
    phi = wdf.explain(e, _dev(C)).cpu().numpy()
    torch.cuda.synchronize()
    counts = oracle.bg_hist(ens, B)
    want = oracle.values_hist(ens, counts, B.shape[0], C)
    assert_phi_close(phi, want, "mid, all 100,000 consumers")
    assert wdf.expected_value(e) == pytest.approx(oracle.base_from_hist(ens, counts, B.shape[0]), rel=1e-9)
    e.close()


def _sample_rows(n, tile, rng, k=1000):
    """k rows of [0, n): the first tile and the row after it, the seam of the last full
    tile, the last rows, then uniform draws."""
    fixed = [0, 1, tile - 1, tile, tile + 1, (n // tile) * tile - 1, (n // tile) * tile, n - 2, n - 1]
    fixed += [j * tile - 1 for j in rng.integers(1, max(2, n // tile + 1), size=16)]
    fixed = [r for r in fixed if 0 <= r < n]
    extra = rng.choice(n, size=min(n, max(0, k - len(set(fixed)))), replace=False)
    return np.unique(np.concatenate([np.array(fixed, dtype=np.int64), extra.astype(np.int64)]))[:max(k, 1)]


def test_ragged_batch_against_oracle(wdf, ctx):
    """The 64-ensemble ragged batch at full size in one autotuned graph launch; 1,000
    rows per ensemble against the FP64 oracle."""
    import torch
    specs = synth.ragged_specs()
    ens_np, ens, Cs, counts, ms = [], [], [], [], []
    for w in specs:
        e_np, C, B = synth.make(w)
        e = wdf.load_ensemble(ctx, e_np)
        wdf.set_background(e, _dev(B), SPLIT)
        counts.append(oracle.bg_hist(e_np, B))
        ms.append(B.shape[0])
        ens_np.append(e_np)
        ens.append(e)
        Cs.append(C)
        del B
    dCs = [_dev(C) for C in Cs]
    batch = wdf.batch_create(ctx, ens)
    reqs = list(enumerate(dCs))
    wdf.batch_autotune(batch, reqs, reps=1)
    outs = [torch.full((C.shape[0], e_np.n_features), float("nan"), device="cuda:0") for C, e_np in zip(Cs, ens_np)]
    wdf.batch_explain(batch, reqs, outs=outs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    depths = set()
    for k, w in enumerate(specs):
        D = wdf.ensemble_info(ens[k])["depth"]
        depths.add(D)
        n = Cs[k].shape[0]
        rows = _sample_rows(n, wdf.batch_tile_rows(batch, D), rng)
        got = outs[k][torch.from_numpy(rows).to("cuda:0")].cpu().numpy()
        assert np.isfinite(got).all(), f"ensemble {k}: rows left unwritten"
        want = oracle.values_hist(ens_np[k], counts[k], ms[k], Cs[k][rows])
        assert_phi_close(got, want, f"ragged ensemble {k} (T={w.n_trees}, D={D}, F={w.n_features}, n={n})")
    assert depths == set(range(2, 9))
    batch.close()
    for e in ens:
        e.close()


def test_served_requests_against_oracle(wdf, ctx):
    """The four resident serving ensembles on their 1e6-row backgrounds: requests of mixed
    sizes (single rows to 40,000 rows, parts of 8,192 rows cut across waves and slots) on
    every ensemble, strided inputs and outputs, sampled rows against the FP64 oracle."""
    import torch
    specs = synth.serving_specs()
    ens_np, ens, counts = [], [], []
    for w in specs:
        e_np, _, B = synth.make(w)
        e = wdf.load_ensemble(ctx, e_np)
        wdf.set_background(e, _dev(B), SPLIT)
        counts.append(oracle.bg_hist(e_np, B))
        ens_np.append(e_np)
        ens.append(e)
        del B
    torch.cuda.synchronize()
    srv = wdf.server_create(ctx, ens, device_budget_bytes=16 << 30, n_slots=3, max_wave=32)
    sizes = [1, 7, 300, 8191, 8192, 8193, 20000, 40000]
    rng = np.random.default_rng(5)
    subs = []
    for k, w in enumerate(specs):
        F = w.n_features
        C = synth.consumers(w, sum(sizes))
        off = 0
        for n in sizes:
            # rows and phi with leading dimensions larger than F
            Cw = np.full((n, F + 3), np.nan, np.float32)
            Cw[:, :F] = C[off:off + n]
            phw = np.full((n, F + 5), 7.0, np.float32)
            t, _ = wdf.server_submit(srv, k, Cw[:, :F], phi=phw[:, :F])
            subs.append((t, k, C[off:off + n], Cw, phw))
            off += n
    for t, *_ in subs:
        wdf.server_wait(srv, t, 600_000)
    st = wdf.server_stats(srv)
    assert st["completed"] == st["submitted"] == len(subs)
    assert st["queued"] == 0 and st["device_bytes_in_use"] == 0
    for t, k, C, Cw, phw in subs:
        n, F = C.shape
        assert (phw[:, F:] == 7.0).all(), "written past F in a strided phi"
        seams = [r for r in (0, 8191, 8192, 8193, 16383, 16384, n - 1) if r < n]
        rows = np.unique(np.concatenate([seams, rng.choice(n, size=min(n, 8), replace=False)])).astype(np.int64)
        want = oracle.values_hist(ens_np[k], counts[k], 1_000_000, C[rows])
        assert_phi_close(phw[rows, :F], want, f"served request of {n} rows on ensemble {k}")
        assert wdf.server_request_ms(srv, t) > 0
    srv.close()
    for e in ens:
        e.close()
