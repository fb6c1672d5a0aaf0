"""The C ABI library builds, loads, exports what include/adr.h declares, and
rejects invalid input on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def adr():
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    adr.lib()
    return adr


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(adr_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(adr):
    names = declared_functions()
    assert "adr_plan_create" in names and "adr_step" in names and "adr_solve" in names
    L = ctypes.CDLL(adr.library_path)
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    # the binding declares a signature for every exported function
    from paper_2307_10684_gb300 import _abi
    assert names <= set(_abi.SIGNATURES), names - set(_abi.SIGNATURES)


def test_struct_layout_matches_c(adr):
    """sizeof / offsetof from a C compiler agree with the ctypes mirror."""
    from paper_2307_10684_gb300 import _abi
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "adr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(adr_problem), offsetof(adr_problem, n),
         offsetof(adr_problem, tau), offsetof(adr_problem, state), sizeof(adr_stats),
         offsetof(adr_stats, ms));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    P, S = _abi.AdrProblem, _abi.AdrStats
    assert vals == [ctypes.sizeof(P), P.n.offset, P.tau.offset, P.state.offset, ctypes.sizeof(S),
                    S.ms.offset]


def test_invalid_problems_rejected_on_host(adr):
    from paper_2307_10684_gb300 import _abi
    L = adr.lib()
    good = wl.fhn_1024(n=64)
    bad = [good.replace(d=4), good.replace(n=(2, 64)), good.replace(n=(5000, 64)),
           good.replace(tau=0.0), good.replace(tau=float("nan")), good.replace(diff=(0.0, 1.0)),
           good.replace(model=7), good.replace(precision=9), good.replace(hi=(0.0, 100.0))]
    for p in bad:
        s = adr.make_problem(p)
        plan = _abi.AdrPlan()
        st = L.adr_plan_create(ctypes.byref(s), None, ctypes.byref(plan))
        assert st == adr.ADR_EINVAL, p
        assert not plan.value
        assert len(L.adr_last_error()) > 0
    # state modes: unknown -> EINVAL; compensated where it does not apply -> EUNSUPPORTED
    for p, want in ((good.replace(state=3), adr.ADR_EINVAL),
                    (good.replace(precision=wl.FP32, state=wl.STATE_COMPENSATED),
                     adr.ADR_EUNSUPPORTED),
                    (good.replace(precision=wl.BF16X3, scheme=wl.LAWSON2B,
                                  state=wl.STATE_COMPENSATED), adr.ADR_EUNSUPPORTED)):
        s = adr.make_problem(p)
        plan = _abi.AdrPlan()
        assert L.adr_plan_create(ctypes.byref(s), None, ctypes.byref(plan)) == want, p
        assert not plan.value
    s = adr.make_problem(good)
    s.reserved = 1
    assert L.adr_plan_create(ctypes.byref(s), None, ctypes.byref(_abi.AdrPlan())) == adr.ADR_EINVAL
    assert L.adr_plan_reset_state(None) == adr.ADR_EINVAL
    assert L.adr_plan_create(None, None, ctypes.byref(_abi.AdrPlan())) == adr.ADR_EINVAL
    assert L.adr_step(None, None, None, 1) == adr.ADR_EINVAL
    assert L.adr_status_str(adr.ADR_EBUSY) == b"ADR_EBUSY"


def test_plan_bytes_host_only(adr):
    sb, cb = adr.plan_bytes(wl.fhn_1024())
    assert sb == 2 * 1024 * 1024 * 4
    assert cb > sb
    sb64, _ = adr.plan_bytes(wl.schnakenberg_64())
    assert sb64 == 2 * 64 * 64 * 8
    # a compensated state adds one FP32 word per point and component
    _, c_comp = adr.plan_bytes(wl.fhn_1024(precision=wl.BF16X3).replace(state=wl.STATE_COMPENSATED))
    _, c_plain = adr.plan_bytes(wl.fhn_1024(precision=wl.BF16X3).replace(state=wl.STATE_PLAIN))
    _, c_auto = adr.plan_bytes(wl.fhn_1024(precision=wl.BF16X3))
    assert c_comp - c_plain == 2 * 1024 * 1024 * 4 and c_auto == c_plain


def test_selftest_limits_checked_on_the_host(adr):
    """The bounded-wait self-test rejects limits outside [1 ms, 2 s] before
    touching the GPU."""
    c, w = ctypes.c_int32(), ctypes.c_int64()
    L = adr.lib()
    assert L.adr_selftest_bounded_wait(None, 0, 10, ctypes.byref(c), ctypes.byref(w)) == adr.ADR_EINVAL
    assert L.adr_selftest_bounded_wait(None, 0, 3_000_000_000, ctypes.byref(c),
                                       ctypes.byref(w)) == adr.ADR_EINVAL
    assert L.adr_selftest_bounded_wait(None, 0, 20_000_000, None, ctypes.byref(w)) == adr.ADR_EINVAL
