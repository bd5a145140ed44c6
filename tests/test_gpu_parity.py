"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: pattern-pair tables equal the oracle's FP64 cube values exactly; background
pattern counts are bit-exact; phi within |gpu - oracle| <= 1e-6 + 1e-5 * |oracle|
(FP32 contraction and accumulation); E_b f(b) to 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-6, 1e-5


def assert_phi_close(got, want):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - want)
    bound = ATOL + RTOL * np.abs(want)
    bad = err > bound
    assert not bad.any(), (f"{int(bad.sum())} of {bad.size} entries off; worst excess "
                           f"{(err - bound).max():.3e}, max |err| {err.max():.3e}")


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


def _run(wdf, ctx, ens, C, B, precision="fp32"):
    import torch
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B), precision)
    phi = wdf.explain(e, _dev(C))
    torch.cuda.synchronize()
    return e, phi.cpu().numpy()


def _heap_positions(ens, t):
    """Heap index (root 0, children 2h+1 / 2h+2) and depth of every node of tree t."""
    o = int(ens.tree_offset[t])
    pos = {0: (0, 0)}
    stack = [0]
    while stack:
        v = stack.pop()
        h, d = pos[v]
        if ens.feature[o + v] >= 0:
            pos[int(ens.left[o + v])] = (2 * h + 1, d + 1)
            pos[int(ens.right[o + v])] = (2 * h + 2, d + 1)
            stack += [int(ens.left[o + v]), int(ens.right[o + v])]
    return pos


# ------------------------------------------------------------------ K2 tables

@pytest.mark.parametrize("first", [
    [0, 1, 2],
    [0, 1, 2, 3, 4, 5],
    [0, 1, 0, 3, 1, 5],
    [0, 0, 0, 0],
    [0, 1, 2, 3, 4, 5, 6, 7],
    [0, 1, 1, 3, 0, 5, 6, 3],
])
@pytest.mark.parametrize("metric", ["shapley", "banzhaf"])
def test_pattern_pair_table_matches_oracle_exactly(wdf, ctx, first, metric):
    D = len(first)
    tab = wdf.debug_pair_table(ctx, first, metric)
    feats = [100 + f for f in first]  # positions sharing a first position share a feature
    K = 1 << D
    for pb in range(K):
        for pc in range(0, K, max(1, K // 64)):
            ok, vals = oracle.path_cube(feats, pc, pb, 100 + D, oracle.SHAPLEY if metric == "shapley" else oracle.BANZHAF)
            got = tab[pb, [k * K + pc for k in range(D)]]
            want = np.array([vals[100 + k] if first[k] == k else 0.0 for k in range(D)])
            np.testing.assert_array_equal(got, want)


# ------------------------------------------------------------------ K1 counts

def _check_counts(wdf, e, ens, B, counts=None):
    D = wdf.ensemble_info(e)["depth"]
    NI = (1 << D) - 1
    gpu = wdf.debug_leaf_hist(e)
    if counts is None:
        counts = oracle.bg_hist(ens, B)
    tree, node, depth, hoff, _ = oracle.leaf_table(ens)
    covered = np.zeros(gpu.shape[:2], bool)
    pos = {}
    for i in range(len(tree)):
        t, v, d, h = int(tree[i]), int(node[i]), int(depth[i]), int(hoff[i])
        if t not in pos:
            pos[t] = _heap_positions(ens, t)
        hp, hd = pos[t][v]
        assert hd == d
        q = (hp + 1) * (1 << (D - d)) - 1 - NI  # leftmost leaf below, in the complete layout
        want = np.zeros(1 << D, np.uint64)
        ones = (1 << (D - d)) - 1
        for p in range(1 << d):
            want[(p << (D - d)) | ones] = counts[h + p]
        np.testing.assert_array_equal(gpu[t, q].astype(np.uint64), want)
        covered[t, q] = True
    # leaves below a pass-through node off the kept path are never reached
    assert not gpu[~covered][:, (1 << D) - 1].any()
    m = B.shape[0]
    assert (gpu[covered].sum(axis=1) == m).all()


def test_counts_bit_exact_tiny(wdf, ctx):
    ens, C, B = synth.make("tiny")
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B))
    _check_counts(wdf, e, ens, B)


def test_counts_bit_exact_mid_ragged(wdf, ctx):
    ens, C, B = synth.make("mid", n_consumers=10, n_background=20011, n_trees=40)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B))
    _check_counts(wdf, e, ens, B)


# ------------------------------------------------------------------ phi parity

def test_phi_tiny_against_all_tiers(wdf, ctx):
    ens, C, B = synth.make("tiny")
    e, phi = _run(wdf, ctx, ens, C, B)
    p0, _ = oracle.values_bruteforce(ens, C, B)
    p2 = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    assert_phi_close(phi, p0)
    assert_phi_close(phi, p2)
    fb = oracle.predict(ens, B).mean()
    assert wdf.expected_value(e) == pytest.approx(fb, rel=1e-9, abs=1e-12)
    eff = oracle.predict(ens, C) - fb
    np.testing.assert_allclose(phi.astype(np.float64).sum(axis=1), eff, atol=1e-4)


def test_phi_mid_full_background(wdf, ctx):
    ens, C, B = synth.make("mid", n_consumers=3001)  # several tiles and a ragged tail
    e, phi = _run(wdf, ctx, ens, C, B)
    counts = oracle.bg_hist(ens, B)
    want = oracle.values_hist(ens, counts, B.shape[0], C)
    assert_phi_close(phi, want)
    assert wdf.expected_value(e) == pytest.approx(oracle.base_from_hist(ens, counts, B.shape[0]), rel=1e-9)
    # a 100-consumer slice against the per-pair tier (Eq. trival_bg) directly
    p1, base = oracle.values_pairs(ens, C[:100], B[:20000])
    e2, phi2 = _run(wdf, ctx, ens, C[:100], B[:20000])
    assert_phi_close(phi2, p1)


@pytest.fixture(scope="module")
def large():
    """The large workload (3e6 consumers, 5e6 background rows, 127 features, 200 trees of
    depth 6) and the oracle's background counts of all 5e6 rows."""
    ens, C, B = synth.make("large")
    return ens, C, B, oracle.bg_hist(ens, B)


def test_phi_large_sampled_rows(wdf, ctx, large):
    """The large workload at full size, launched as the benchmark launches it; sampled
    consumers against the oracle with the full background counts."""
    import torch
    ens, C, B, counts = large
    e = wdf.load_ensemble(ctx, ens)
    dB = _dev(B)
    wdf.set_background(e, dB)
    del dB
    dC = _dev(C)
    phi = wdf.explain(e, dC)
    seams = [(1 << 20) - 1, 1 << 20, (1 << 21) - 1, 1 << 21]  # the encoded 2^20-row chunks of one call
    rows = np.unique(np.concatenate([np.linspace(0, C.shape[0] - 1, 48).astype(np.int64),
                                     [0, 63, 64, C.shape[0] - 1], seams]))
    got = phi[torch.from_numpy(rows).to(phi.device)].cpu().numpy()
    want = oracle.values_hist(ens, counts, B.shape[0], C[rows])
    assert_phi_close(got, want)
    assert wdf.expected_value(e) == pytest.approx(oracle.base_from_hist(ens, counts, B.shape[0]), rel=1e-9)
    # background counts at full size, bit-exact for every leaf
    _check_counts(wdf, e, ens, B, counts)
    del phi, dC


@pytest.fixture(scope="module")
def large_sample(large):
    """10,000 seeded consumer rows of the large workload and their oracle values."""
    ens, C, B, counts = large
    rows = np.sort(np.random.default_rng(2511).choice(C.shape[0], 10_000, replace=False))
    return C[rows], oracle.values_hist(ens, counts, B.shape[0], C[rows])


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3", "bf16x6"])
def test_large_contraction_precisions(wdf, ctx, large, large_sample, precision):
    """Every contraction precision on the full large background, error against the FP64
    oracle on a 10,000-consumer sample.  Counts here reach 4.8e6 (23 bits): FP32, TF32
    hi+lo (22 bits per operand) and BF16 hi+mid+lo (24 bits) meet the FP32-mode bound;
    BF16 hi+lo keeps 16 bits of each count and table value (relative error up to about
    2^-16 per product) and is held to a tenfold looser bound."""
    ens, C, B, counts = large
    Cs, want = large_sample
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B), precision)
    got = wdf.explain(e, _dev(Cs)).cpu().numpy().astype(np.float64)
    err = np.abs(got - want)
    scale = 10.0 if precision == "bf16x3" else 1.0
    bound = scale * (ATOL + RTOL * np.abs(want))
    assert (err <= bound).all(), f"{precision}: max |err| {err.max():.3e}, worst ratio {(err / bound).max():.3f}"
    e.close()


# ------------------------------------------------------------------ edge cases

def test_host_memory_path_equals_device_path(wdf, ctx):
    import torch
    ens, C, B = synth.make("mid", n_consumers=777, n_background=5000, n_trees=25)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, B)  # host background
    ph_host = wdf.explain(e, C)  # host consumers -> host phi
    ph_dev = wdf.explain(e, _dev(C))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ph_host, ph_dev.cpu().numpy())
    want = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    assert_phi_close(ph_host, want)


def test_rows_are_independent_of_batch(wdf, ctx):
    import torch
    ens, C, B = synth.make("mid", n_consumers=300, n_background=4000, n_trees=30)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B))
    full = wdf.explain(e, _dev(C)).cpu().numpy()
    for lo, hi in [(0, 1), (5, 6), (17, 99), (250, 300)]:
        part = wdf.explain(e, _dev(C[lo:hi])).cpu().numpy()
        np.testing.assert_array_equal(part, full[lo:hi])
    torch.cuda.synchronize()


def test_strided_inputs_and_outputs(wdf, ctx):
    import torch
    ens, C, B = synth.make("mid", n_consumers=130, n_background=3000, n_trees=12)
    F = ens.n_features
    Bw = np.zeros((B.shape[0], F + 5), np.float32); Bw[:, :F] = B
    Cw = np.zeros((C.shape[0], F + 3), np.float32); Cw[:, :F] = C
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(Bw)[:, :F])
    out = torch.full((C.shape[0], F + 7), 7.0, device="cuda:0")
    wdf.explain(e, _dev(Cw)[:, :F], out=out[:, :F])
    o = out.cpu().numpy()
    assert (o[:, F:] == 7.0).all()
    want = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    assert_phi_close(o[:, :F], want)


def _tree_ensemble(F, trees):
    offs, f, th, l, r, v = [0], [], [], [], [], []
    for nodes in trees:
        for (a, b, c, d, x) in nodes:
            f.append(a); th.append(b); l.append(c); r.append(d); v.append(x)
        offs.append(offs[-1] + len(nodes))
    return synth.Ensemble(F, np.array(offs, np.int64), np.array(f, np.int32), np.array(th, np.float32),
                          np.array(l, np.int32), np.array(r, np.int32), np.array(v, np.float32))


def test_degenerate_trees_nan_ties_and_single_rows(wdf, ctx):
    # a single-leaf tree, a stump, a chain with a repeated feature, NaN and ties
    trees = [
        [(-1, 0, -1, -1, 0.7)],
        [(2, 0.5, 1, 2, 0.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, -1.0)],
        [(0, 0.0, 1, 2, 0.0), (-1, 0, -1, -1, 2.0), (0, 1.0, 3, 4, 0.0), (-1, 0, -1, -1, -3.0),
         (1, -0.5, 5, 6, 0.0), (-1, 0, -1, -1, 0.25), (-1, 0, -1, -1, 4.0)],
    ]
    ens = _tree_ensemble(4, trees)
    rng = np.random.default_rng(5)
    B = rng.standard_normal((257, 4)).astype(np.float32)
    B[:20, 0] = 0.0; B[20:30, 2] = 0.5; B[30:35, 1] = np.nan
    C = rng.standard_normal((65, 4)).astype(np.float32)
    C[0, 0] = np.nan; C[1, 0] = 1.0; C[2, 2] = 0.5
    e, phi = _run(wdf, ctx, ens, C, B)
    want = oracle.values_hist(ens, oracle.bg_hist(ens, B), B.shape[0], C)
    p0, _ = oracle.values_bruteforce(ens, C, B)
    np.testing.assert_allclose(want, p0, atol=1e-12)
    assert_phi_close(phi, want)
    assert not phi[:, 3].any()  # null player
    one = wdf.explain(e, _dev(C[7:8])).cpu().numpy()
    np.testing.assert_array_equal(one, phi[7:8])


def test_constant_trees_and_nan_thresholds(wdf, ctx):
    # only single-leaf trees (no threshold at all), then a tree whose only split has a
    # NaN threshold (every row goes right): values zero / only the constant part
    rng = np.random.default_rng(9)
    B = rng.standard_normal((50, 3)).astype(np.float32)
    C = rng.standard_normal((20, 3)).astype(np.float32)
    const = _tree_ensemble(3, [[(-1, 0, -1, -1, 0.5)], [(-1, 0, -1, -1, -1.25)]])
    e, phi = _run(wdf, ctx, const, C, B)
    assert not phi.any()
    assert wdf.expected_value(e) == pytest.approx(-0.75)
    nanthr = _tree_ensemble(3, [[(1, float("nan"), 1, 2, 0.0), (-1, 0, -1, -1, 3.0), (-1, 0, -1, -1, -2.0)],
                                [(0, 0.0, 1, 2, 0.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, 0.5)]])
    e, phi = _run(wdf, ctx, nanthr, C, B)
    want = oracle.values_hist(nanthr, oracle.bg_hist(nanthr, B), B.shape[0], C)
    assert_phi_close(phi, want)
    assert not phi[:, 1].any() and not phi[:, 2].any()


def test_empty_and_error_paths(wdf, ctx):
    import torch
    ens, C, B = synth.make("tiny")
    e = wdf.load_ensemble(ctx, ens)
    with pytest.raises(wdf.WdfError) as ei:
        wdf.explain(e, _dev(C))  # before set_background
    assert ei.value.status == 1
    with pytest.raises(wdf.WdfError) as ei:
        wdf.set_background(e, _dev(B[:0]))
    assert ei.value.status == 4
    with pytest.raises(wdf.WdfError) as ei:
        wdf.set_background(e, _dev(B), 4)  # no such precision
    assert ei.value.status == 1
    wdf.set_background(e, _dev(B))
    out = wdf.explain(e, _dev(C[:0]))
    assert out.shape == (0, ens.n_features)
    bad = _tree_ensemble(3, [[(0, 0.0, 1, 1, 0.0), (-1, 0, -1, -1, 1.0)]])  # a node reached twice
    with pytest.raises(wdf.WdfError) as ei:
        wdf.load_ensemble(ctx, bad)
    assert ei.value.status == 1
    bad = _tree_ensemble(3, [[(5, 0.0, 1, 2, 0.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, 1.0)]])
    with pytest.raises(wdf.WdfError):
        wdf.load_ensemble(ctx, bad)  # feature out of range
    bad = _tree_ensemble(3, [[(0, 0.0, 1, 2, 0.0), (-1, 0, -1, -1, 1.0), (-1, 0, -1, -1, 1.0),
                              (-1, 0, -1, -1, 1.0)]])
    with pytest.raises(wdf.WdfError):
        wdf.load_ensemble(ctx, bad)  # unreachable node
    # a path of 9 inner nodes: inner node d at index 2d, its left leaf at 2d+1
    nodes = []
    for d in range(9):
        nodes.append((0, float(d), 2 * d + 1, 2 * d + 2, 0.0))
        nodes.append((-1, 0, -1, -1, 1.0))
    nodes.append((-1, 0, -1, -1, 2.0))
    with pytest.raises(wdf.WdfError) as ei:
        wdf.load_ensemble(ctx, _tree_ensemble(1, [nodes]))
    assert ei.value.status == 4
    torch.cuda.synchronize()


def test_global_attribution_fp64(wdf, ctx):
    import torch
    ens, C, B = synth.make("mid", n_consumers=10007, n_background=3000, n_trees=10)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, _dev(B))
    phi = wdf.explain(e, _dev(C))
    ma, mn = wdf.global_attribution(ctx, phi)
    p = phi.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(ma.cpu().numpy(), np.abs(p).mean(axis=0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mn.cpu().numpy(), p.mean(axis=0), rtol=1e-9, atol=1e-15)
    torch.cuda.synchronize()
