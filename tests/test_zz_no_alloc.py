"""adr_max_abs_diff_noalloc, the error reduction for callers that cannot
allocate device memory (fully committed memory budgets, host applications
that own the allocator), against the allocating adr_max_abs_diff.

Both entry points return maxima of exactly representable values, so their
results must be equal, not merely close.  This file is collected last so
that a run stopping at the first failure has already run every other test;
it also passes in a fresh process on its own.
"""
import ctypes
import math

import pytest

pytestmark = pytest.mark.gpu

MAX_COUNT = 1 << 26  # the entry point's documented limit


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def _call(adr, name, x, ref, count=None):
    import torch
    out = (ctypes.c_double * 2)()
    fn = getattr(adr.lib(), name)
    st = fn(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
            ctypes.c_void_p(x.data_ptr()), 1 if x.dtype == torch.float64 else 0,
            ctypes.c_void_p(ref.data_ptr()), ctypes.c_int64(x.numel() if count is None else count),
            out)
    adr._abi.check(st)
    return float(out[0]), float(out[1])


def _same(a, b):
    return all((x == y) or (math.isnan(x) and math.isnan(y)) for x, y in zip(a, b))


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
        assert got == want
        # and both agree with a plain torch reduction
        assert got[0] == float((x.double() - ref).abs().max())
        assert got[1] == float(ref.abs().max())


@pytest.mark.parametrize("count", [0, 1, 4096, 4096 * 37, 4096 * 37 + 1, MAX_COUNT])
def test_noalloc_sizes_block_multiples_and_limit(adr, count):
    """Empty input, one element, exact multiples of the 4096-element block,
    a ragged tail, and the largest accepted count."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(count + 1)
    ref = torch.randn(max(count, 1), dtype=torch.float64, device="cuda", generator=g)
    x = (ref + 1e-4 * torch.randn(ref.shape, dtype=torch.float64, device="cuda",
                                  generator=g)).float()
    want = _call(adr, "adr_max_abs_diff", x, ref, count)
    got = _call(adr, "adr_max_abs_diff_noalloc", x, ref, count)
    assert got == want
    if count == 0:
        assert got == (0.0, 0.0)
    del x, ref
    torch.cuda.empty_cache()


@pytest.mark.parametrize("where", ["x", "ref"])
def test_noalloc_propagates_nan_like_allocating(adr, where):
    import torch
    g = torch.Generator(device="cuda").manual_seed(11)
    ref = torch.randn(4096 * 3 + 5, dtype=torch.float64, device="cuda", generator=g)
    x = ref.float().clone()
    (x if where == "x" else ref)[4096 + 17] = float("nan")
    want = _call(adr, "adr_max_abs_diff", x, ref)
    got = _call(adr, "adr_max_abs_diff_noalloc", x, ref)
    assert math.isnan(got[0]) and _same(got, want)
    # a second call on clean data is not affected by the NaN left in scratch
    x2 = ref.nan_to_num(0.0).float()
    ref2 = ref.nan_to_num(0.0)
    assert _call(adr, "adr_max_abs_diff_noalloc", x2, ref2) == _call(adr, "adr_max_abs_diff",
                                                                     x2, ref2)


def test_noalloc_rejects_oversized_count(adr):
    import torch
    x = torch.zeros(16, device="cuda")
    ref = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 2)()
    st = adr.lib().adr_max_abs_diff_noalloc(None, ctypes.c_void_p(x.data_ptr()), 0,
                                            ctypes.c_void_p(ref.data_ptr()),
                                            ctypes.c_int64(MAX_COUNT + 1), out)
    assert st == adr.ADR_EINVAL
    assert b"scratch limit" in adr.lib().adr_last_error()
