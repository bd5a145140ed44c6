"""Failure detection without a GPU fault.

- Host side: waiting on a request with a zero timeout while it is still queued or in
  flight returns WDF_ETIMEOUT; the request still completes afterwards.
- Device side: the tensor-core contraction's first bounded mbarrier wait is shortened
  by a test hook to one non-suspending poll, so it gives up while the kernel's own
  tensor-core work is in flight.  The kernel raises its error flag, still waits at the
  normal limit for that work before freeing its tensor memory, and returns; the call
  reports WDF_ETIMEOUT and leaves the background unset.  The next normal call on the
  same context succeeds and matches the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from conftest import assert_phi_close
from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu

ETIMEOUT, EINVAL = 5, 1


@pytest.fixture(scope="module")
def wdf():
    import paper_2511_09376_gb300 as w
    return w


def test_server_wait_times_out_on_host_then_completes(wdf):
    import torch
    ctx = wdf.ctx_create(0)
    ens_np, _, B = synth.make(synth.Workload("f", 61, 1, 20000, 127, 90, 400, 8, 0.1, 0.1, False))
    e = wdf.load_ensemble(ctx, ens_np)
    wdf.set_background(e, torch.from_numpy(B).cuda())
    srv = wdf.server_create(ctx, [e], device_budget_bytes=1 << 30, n_slots=1, max_wave=1)
    C = np.random.default_rng(3).standard_normal((60000, 127)).astype(np.float32)
    t, phi = wdf.server_submit(srv, 0, C)
    with pytest.raises(wdf.WdfError) as ei:
        wdf.server_wait(srv, t, 0)
    assert ei.value.status == ETIMEOUT
    wdf.server_wait(srv, t, 600_000)
    np.testing.assert_array_equal(phi[:100], wdf.explain(e, C[:100]))
    srv.close()
    e.close()
    ctx.close()


@pytest.mark.parametrize("precision", ["bf16x6", "tf32x3"])
def test_contraction_wait_expiry_reports_timeout_and_context_recovers(wdf, precision):
    import torch
    ctx = wdf.ctx_create(0)
    ens_np, C, B = synth.make(synth.Workload("g", 62, 200, 5000, 40, 30, 60, 8, 0.1, 0.1, False))
    e = wdf.load_ensemble(ctx, ens_np)
    dB, dC = torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda()
    wdf.debug_contract_wait_limit(1)
    try:
        with pytest.raises(wdf.WdfError) as ei:
            wdf.set_background(e, dB, precision)
        assert ei.value.status == ETIMEOUT
    finally:
        wdf.debug_contract_wait_limit(0)
    assert wdf.ensemble_info(e)["has_background"] == 0
    with pytest.raises(wdf.WdfError) as ei:
        wdf.explain(e, dC)
    assert ei.value.status == EINVAL
    # the same context and ensemble, normal limits: the full result
    wdf.set_background(e, dB, precision)
    phi = wdf.explain(e, dC).cpu().numpy()
    want = oracle.values_hist(ens_np, oracle.bg_hist(ens_np, B), B.shape[0], C)
    assert_phi_close(phi, want, f"after a timed-out {precision} contraction")
    e.close()
    ctx.close()
