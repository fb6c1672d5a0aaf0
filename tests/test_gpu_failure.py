"""Failure detection on the GPU without a fault: a bounded mbarrier wait that
nothing satisfies gives up after its limit, the host reads the timeout code
from the device error word, and the context stays usable."""
import pytest

import oracle
import workloads as wl
from oracle import schemes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def test_wait_that_nothing_satisfies_times_out(adr):
    limit = 20_000_000  # 20 ms
    code, waited = adr.selftest_bounded_wait(arrive=False, limit_ns=limit)
    assert code == 1                       # the timeout code the kernels record
    assert limit <= waited < 50 * limit    # gave up after its limit, not before


def test_satisfied_wait_returns_at_once(adr):
    code, waited = adr.selftest_bounded_wait(arrive=True, limit_ns=1_000_000_000)
    assert code == 0 and waited < 100_000_000


def test_context_usable_after_a_timeout(adr):
    import torch
    adr.selftest_bounded_wait(arrive=False, limit_ns=5_000_000)
    p = wl.fhn_1024(precision=wl.BF16X3, n=64, nsteps=5)
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p) as plan:
        plan.set_timing(True)
        plan.step(u, v, p.nsteps)
        st = plan.stats()
    assert st["device_error"] == 0
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    assert oracle.max_rel_err(u.double().cpu().numpy(), v.double().cpu().numpy(), Ur, Vr) <= 1e-5

