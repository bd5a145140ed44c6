"""The allocation-free global attribution entry point, called through the C ABI.

It must give the same per-feature FP64 means as wdf_global_attribution (which takes its
partial-sum buffer from the stream-ordered allocator), call after call, although every
call reuses the library's fixed device array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-12, 1e-15  # the tolerance of the global-attribution test


def _lib():
    import paper_2511_09376_gb300 as wdf
    lib = ctypes.CDLL(wdf.library_path())
    f = lib.wdf_global_attribution_noalloc
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    lib.wdf_last_error.restype = ctypes.c_char_p
    return wdf, lib


def _noalloc(lib, torch, phi, stream):
    n, F = phi.shape
    ma = torch.full((F,), float("nan"), dtype=torch.float64, device=phi.device)
    mn = torch.full((F,), float("nan"), dtype=torch.float64, device=phi.device)
    rc = lib.wdf_global_attribution_noalloc(phi.device.index or 0, phi.data_ptr(), n, phi.stride(0), F,
                                            ma.data_ptr(), mn.data_ptr(), stream.cuda_stream)
    assert rc == 0, lib.wdf_last_error()
    return ma, mn


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    wdf, lib = _lib()
    ctx = wdf.ctx_create(0)
    gen = torch.Generator(device="cuda:0").manual_seed(20251109)
    stream = torch.cuda.current_stream()
    cases = [torch.randn((300_007, 127), device="cuda:0", generator=gen),
             torch.randn((41_000, 132), device="cuda:0", generator=gen)[:, :97]]  # ldphi > F
    for phi in cases:
        ma_ref, mn_ref = wdf.global_attribution(ctx, phi)
        for _ in range(2):  # the fixed scratch keeps the previous call's contents
            ma, mn = _noalloc(lib, torch, phi, stream)
            torch.cuda.synchronize()
            np.testing.assert_allclose(ma.cpu().numpy(), ma_ref.cpu().numpy(), rtol=RTOL, atol=ATOL)
            np.testing.assert_allclose(mn.cpu().numpy(), mn_ref.cpu().numpy(), rtol=RTOL, atol=ATOL)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    wdf, lib = _lib()
    out = torch.zeros(127, dtype=torch.float64, device="cuda:0")
    # ceil(n / 4096) * 127 * 2 doubles > 262,144 once n exceeds about 4.2 million rows
    rc = lib.wdf_global_attribution_noalloc(0, out.data_ptr(), 5_000_000, 127, 127, out.data_ptr(), out.data_ptr(),
                                            None)
    assert rc == 1
    assert b"too large" in lib.wdf_last_error()
