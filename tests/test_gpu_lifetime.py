"""Object lifetimes through the C ABI: the ensembles, batches and servers made from a
context hold it, so destroying the context first (as a garbage collector may, in any
order) leaves them usable and their later destruction safe."""
import pytest

from paper_2511_09376_gb300 import synth

pytestmark = pytest.mark.gpu


def test_context_destroyed_before_its_objects():
    import torch
    import paper_2511_09376_gb300 as wdf
    ens, C, B = synth.make("tiny")
    ctx = wdf.ctx_create(0)
    e = wdf.load_ensemble(ctx, ens)
    wdf.set_background(e, torch.from_numpy(B).cuda())
    b = wdf.batch_create(ctx, [e])
    ref = wdf.explain(e, torch.from_numpy(C).cuda())
    ctx.close()  # the caller's handle goes first
    again = wdf.explain(e, torch.from_numpy(C).cuda())
    out = wdf.batch_explain(b, [(0, torch.from_numpy(C).cuda())])[0]
    torch.cuda.synchronize()
    assert torch.equal(again, ref) and torch.equal(out, ref)
    b.close()
    e.close()
    # a fresh context and ensemble afterwards see no error left behind
    ctx2 = wdf.ctx_create(0)
    e2 = wdf.load_ensemble(ctx2, ens)
    wdf.set_background(e2, torch.from_numpy(B).cuda())
    assert torch.equal(wdf.explain(e2, torch.from_numpy(C).cuda()), ref)
