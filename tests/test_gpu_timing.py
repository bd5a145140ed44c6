"""Consumer-kernel timing (wdf_explain_timing): one event pair per consumer-kernel
launch (one launch per 2^20 rows of a call), nothing recorded while off, the pairs
forgotten once read, and the results unchanged by the timing."""
import numpy as np
import pytest

from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu


def test_explain_timing_counts_launches_and_leaves_phi_unchanged():
    import torch
    import paper_2511_09376_gb300 as wdf
    ctx = wdf.ctx_create(0)
    ens, C, B = synth.make("mid", n_consumers=(1 << 20) + 5000, n_background=20000)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, torch.from_numpy(B).cuda())
    dC = torch.from_numpy(C).cuda()
    plain = wdf.explain(e, dC)
    torch.cuda.synchronize()

    wdf.explain_timing(True)
    timed = wdf.explain(e, dC)
    timed2 = wdf.explain(e, dC[:1000])
    ms, launches = wdf.explain_timing_read()
    assert launches == 3  # two chunks, then one
    assert ms > 0.0
    assert wdf.explain_timing_read() == (0.0, 0)  # forgotten once read
    wdf.explain_timing(False)
    wdf.explain(e, dC[:1000])
    assert wdf.explain_timing_read()[1] == 0  # nothing recorded while off
    assert torch.equal(timed, plain)
    assert torch.equal(timed2, plain[:1000])
