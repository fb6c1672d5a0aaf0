"""adr_max_abs_diff_noalloc, the error reduction for callers that cannot
allocate device memory (fully committed memory budgets, host applications
that own the allocator), against the allocating adr_max_abs_diff.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes in a fresh process on its own.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the parity tolerance of the FP32-class tests; the maxima are in fact exact


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def _call(adr, name, x, ref):
    import torch
    out = (ctypes.c_double * 2)()
    fn = getattr(adr.lib(), name)
    st = fn(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
            ctypes.c_void_p(x.data_ptr()), 1 if x.dtype == torch.float64 else 0,
            ctypes.c_void_p(ref.data_ptr()), ctypes.c_int64(x.numel()), out)
    adr._abi.check(st)
    return float(out[0]), float(out[1])


def test_noalloc_matches_allocating_reduction_twice(adr):
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    # first call: FP32 field of a 1024^2 grid; second call: a smaller FP64
    # field, so the second result can only be right if the first call's
    # scratch contents are not reused
    ref1 = torch.randn(1024 * 1024, dtype=torch.float64, device="cuda", generator=g)
    x1 = (ref1 + 1e-3 * torch.randn(ref1.shape, dtype=torch.float64, device="cuda",
                                    generator=g)).float()
    ref2 = 3.0 * torch.rand(70_001, dtype=torch.float64, device="cuda", generator=g)
    x2 = ref2 + 1e-6 * torch.randn(ref2.shape, dtype=torch.float64, device="cuda", generator=g)
    for x, ref in ((x1, ref1), (x2, ref2)):
        want = _call(adr, "adr_max_abs_diff", x, ref)
        got = _call(adr, "adr_max_abs_diff_noalloc", x, ref)
        assert abs(got[0] - want[0]) <= TOL * max(want[0], 1e-300)
        assert abs(got[1] - want[1]) <= TOL * want[1]
        # and both agree with a plain torch reduction
        assert got[1] == pytest.approx(float(ref.abs().max()), rel=1e-15)


def test_noalloc_rejects_oversized_count(adr):
    import torch
    x = torch.zeros(16, device="cuda")
    ref = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 2)()
    st = adr.lib().adr_max_abs_diff_noalloc(None, ctypes.c_void_p(x.data_ptr()), 0,
                                            ctypes.c_void_p(ref.data_ptr()),
                                            ctypes.c_int64((1 << 26) + 1), out)
    assert st == adr.ADR_EINVAL
    assert b"scratch limit" in adr.lib().adr_last_error()
