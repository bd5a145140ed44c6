"""Continuous-batching server: every request's phi equals the single-call result bit for
bit, alone and in a concurrent mix; admission respects the device-memory budget."""
import threading

import numpy as np
import pytest

from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

SPECS = [(51, 2000, 30, 20, 25, 4, 0.3, 0.1, False, "fp32"),
         (52, 2000, 127, 90, 40, 6, 0.1, 0.1, False, "bf16x6"),
         (53, 2000, 60, 40, 12, 7, 0.1, 0.1, False, "tf32x3")]


@pytest.fixture(scope="module")
def setup():
    import torch

    import paper_2511_09376_gb300 as wdf
    ctx = wdf.ctx_create(0)
    ens = []
    for k, (seed, m, F, ng, T, D, sd, p, comp, prec) in enumerate(SPECS):
        e_np, _, B = synth.make(synth.Workload(f"s{k}", seed, 1, m, F, ng, T, D, sd, p, comp))
        e = wdf.load_ensemble(ctx, e_np)
        wdf.set_background(e, torch.from_numpy(B).cuda(), prec)
        ens.append(e)
    return wdf, ctx, ens


def _rows(k, n, F, seed):
    return np.random.default_rng(seed).standard_normal((n, F)).astype(np.float32)


def test_same_alone_and_in_the_mix(setup):
    wdf, ctx, ens = setup
    Fs = [wdf.ensemble_info(e)["n_features"] for e in ens]
    srv = wdf.server_create(ctx, ens, device_budget_bytes=256 << 20, n_slots=3, max_wave=8)
    probe = _rows(1, 777, Fs[1], 99)
    t, alone = wdf.server_submit(srv, 1, probe)
    wdf.server_wait(srv, t)
    single = wdf.explain(ens[1], probe)  # host-memory single call
    np.testing.assert_array_equal(alone, single)
    # the same request again among concurrent submissions from several threads
    results, errors = {}, []

    def client(tid):
        try:
            rng = np.random.default_rng(tid)
            mine = []
            for j in range(12):
                k = int(rng.integers(0, 3))
                n = int(rng.choice([1, 5, 64, 65, 300, 2500]))
                C = _rows(k, n, Fs[k], 1000 * tid + j)
                t, phi = wdf.server_submit(srv, k, C)
                mine.append((t, k, C, phi))
            for t, k, C, phi in mine:
                wdf.server_wait(srv, t)
                results[(tid, t)] = (k, C, phi)
        except Exception as exc:  # surfaced below
            errors.append(exc)

    threads = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for th in threads:
        th.start()
    t2, mixed = wdf.server_submit(srv, 1, probe)
    for th in threads:
        th.join()
    wdf.server_wait(srv, t2)
    assert not errors, errors
    np.testing.assert_array_equal(mixed, alone)
    for (tid, t), (k, C, phi) in results.items():
        np.testing.assert_array_equal(phi, wdf.explain(ens[k], C))
    st = wdf.server_stats(srv)
    assert st["completed"] == st["submitted"] == 2 + 4 * 12
    assert st["queued"] == 0 and st["device_bytes_in_use"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["waves"] < st["completed"]  # some waves carried several requests
    srv.close()


def test_budget_admission_and_rejection(setup):
    wdf, ctx, ens = setup
    F = wdf.ensemble_info(ens[0])["n_features"]
    one = 2 * 1000 * F * 4
    srv = wdf.server_create(ctx, ens, device_budget_bytes=2 * one, n_slots=4, max_wave=4)
    subs = [wdf.server_submit(srv, 0, _rows(0, 1000, F, i)) for i in range(10)]
    for t, _ in subs:
        wdf.server_wait(srv, t)
    for (t, phi), i in zip(subs, range(10)):
        np.testing.assert_array_equal(phi, wdf.explain(ens[0], _rows(0, 1000, F, i)))
    with pytest.raises(wdf.WdfError) as ei:
        wdf.server_submit(srv, 0, _rows(0, 3000, F, 7))
    assert ei.value.status == 2
    assert wdf.server_stats(srv)["device_bytes_in_use"] == 0
    srv.close()


def test_multi_part_requests_strided_across_waves_and_slots(setup):
    """Requests longer than one part (8,192 rows) with row strides larger than F on both
    sides: with two slots and waves of at most two parts, the parts of one request land
    in different waves and slots; phi still equals the single call bit for bit."""
    wdf, ctx, ens = setup
    srv = wdf.server_create(ctx, ens, device_budget_bytes=1 << 30, n_slots=2, max_wave=2)
    subs = []
    for j, (k, n) in enumerate([(1, 8193), (0, 20011), (2, 16384), (1, 3)]):
        F = wdf.ensemble_info(ens[k])["n_features"]
        Cw = np.full((n, F + 4), np.nan, np.float32)
        Cw[:, :F] = _rows(k, n, F, 500 + j)
        phw = np.full((n, F + 6), -3.0, np.float32)
        t, _ = wdf.server_submit(srv, k, Cw[:, :F], phi=phw[:, :F])
        subs.append((t, k, Cw, phw, F))
    for t, *_ in subs:
        wdf.server_wait(srv, t)
    for t, k, Cw, phw, F in subs:
        np.testing.assert_array_equal(phw[:, :F], wdf.explain(ens[k], np.ascontiguousarray(Cw[:, :F])))
        assert (phw[:, F:] == -3.0).all()
    st = wdf.server_stats(srv)
    assert st["completed"] == st["submitted"] == len(subs)
    assert st["device_bytes_in_use"] == 0 and st["queued"] == 0
    assert st["waves"] >= 4  # 2 + 3 + 2 + 1 = 8 parts in waves of at most two parts
    srv.close()


def test_small_requests_use_the_express_slot(setup):
    """With four or more slots, slot 0 serves only small requests: a single-row request
    submitted behind many large parts completes before them."""
    wdf, ctx, ens = setup
    F = wdf.ensemble_info(ens[1])["n_features"]
    srv = wdf.server_create(ctx, ens, device_budget_bytes=4 << 30, n_slots=4, max_wave=1)
    big = [wdf.server_submit(srv, 1, _rows(1, 60000, F, 900 + i)) for i in range(8)]
    t_small, phi_small = wdf.server_submit(srv, 1, _rows(1, 1, F, 999))
    wdf.server_wait(srv, t_small)
    done_big = sum(wdf.server_poll(srv, t) for t, _ in big)
    assert done_big < len(big)
    for t, _ in big:
        wdf.server_wait(srv, t)
    np.testing.assert_array_equal(phi_small, wdf.explain(ens[1], _rows(1, 1, F, 999)))
    assert wdf.server_request_ms(srv, t_small) < max(wdf.server_request_ms(srv, t) for t, _ in big)
    srv.close()
