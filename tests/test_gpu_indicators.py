"""Indicators of Sec. 4 fused into the last product of every step, and the
step-count-free run (adr_run), against the oracle.

The indicators are the trapezoid-weighted spatial mean <U_n> and the time
increment ||U_{n+1} - U_n||_F (Sec. 4, before the experiments).  The GPU
accumulates them in FP64 from the single-precision states, so the means
agree with the oracle's to about the state's own accuracy, and the
increments (differences of two single-precision states) to a few times the
states' rounding relative to the increment's size.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import metrics, schemes

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


def _oracle_indicators(p, u0, v0, nsteps):
    rows = []
    prev = [u0, v0]

    def cb(n, U, V):
        mu, du = metrics.indicators(prev[0], U)
        mv, dv = metrics.indicators(prev[1], V)
        rows.append((mu, mv, du, dv))
        prev[0], prev[1] = U, V

    U, V = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, nsteps, callback=cb)
    return np.array(rows), U, V


@pytest.mark.parametrize("n,model,kernel", [((128, 96), wl.SCHNAKENBERG, 0),
                                            ((256, 256), wl.FHN, 4),
                                            ((40, 24, 56), wl.BRUSSELATOR, -1)])
def test_fused_indicators_match_oracle_every_step(adr, n, model, kernel):
    import torch
    d = len(n)
    params = {wl.SCHNAKENBERG: (200.0, 0.1, 0.9), wl.FHN: (0.05, 2.0, -0.03),
              wl.BRUSSELATOR: (1.0, 3.0)}[model]
    L = 100.0 if model == wl.FHN else 1.0
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(L,) * d, diff=(0.05, 0.3) if L == 1.0 else (1.0, 20.0),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=model,
                   params=params, tau=2e-3 if L == 1.0 else 1e-2, nsteps=50, seed=31,
                   precision=wl.BF16X3)
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    ref, Ur, Vr = _oracle_indicators(p, u0, v0, p.nsteps)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p, kernel=kernel) as plan:
        plan.set_indicators(True)
        plan.step(u, v, 20)
        plan.step(u, v, 30)  # two calls: the history continues
        got = plan.indicator_log()
    assert got.shape == (50, 4)
    scale_mean = np.abs(ref[:, :2]).max(axis=0)
    assert np.max(np.abs(got[:, :2] - ref[:, :2]) / scale_mean) <= 1e-6, (got[:3], ref[:3])
    # an increment taken between two single-precision states cannot resolve
    # less than their rounding: about ulp(max|X|) per point, sqrt(N) in the norm
    N = float(np.prod(n))
    floor = 2.0 * np.sqrt(N) * 2.0 ** -23 * np.array([np.abs(Ur).max(), np.abs(Vr).max()])
    err = np.abs(got[:, 2:] - ref[:, 2:])
    assert np.all(err <= 1e-3 * ref[:, 2:] + floor), np.max(err / (1e-3 * ref[:, 2:] + floor))


def test_indicators_leave_the_state_unchanged(adr):
    """The same steps with indicators on and off give bitwise equal states,
    for a plain and a compensated state."""
    import torch
    for state in (wl.STATE_PLAIN, wl.STATE_COMPENSATED):
        p = wl.fhn_1024(precision=wl.BF16X3, n=192, nsteps=40).replace(state=state)
        u0, v0 = wl.initial_data(p)
        outs = []
        for on in (False, True):
            u = torch.tensor(u0, dtype=torch.float32, device="cuda")
            v = torch.tensor(v0, dtype=torch.float32, device="cuda")
            with adr.Plan(p) as plan:
                if on:
                    plan.set_indicators(True)
                plan.step(u, v, p.nsteps)
            torch.cuda.synchronize()
            outs.append((u.cpu(), v.cpu()))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1]), state


def _bruss_e6(n, tau):
    # Sec. 4.6: delta = (0.01, 0.02), alpha = 0.1 in every direction,
    # g^u = a_2 - (a_1 + 1) u + u^2 v, g^v = a_1 u - u^2 v with a_1 = 1, a_2 = 2
    vel = (0.1, 0.1, 0.1)
    return wl.Problem(d=3, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3, diff=(0.01, 0.02),
                      adv=(vel, vel), model=wl.BRUSSELATOR, params=(2.0, 1.0), tau=tau,
                      nsteps=int(round(5.0 / tau)), precision=wl.BF16X3)


def test_run_to_the_brusselator_equilibrium(adr):
    """Sec. 4.6: on 64^3 with tau = 5e-2 the Brusselator run to T = 5 (100
    steps) approaches the equilibrium (a_2, a_1 / a_2) = (2, 0.5).  adr_run
    stops on the horizon; its final state and last indicators match the
    oracle's, and the increment indicator has decayed toward zero."""
    import torch
    p = _bruss_e6(64, 5e-2)
    u0, v0 = wl.brusselator_e6_initial(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    ref, Ur, Vr = _oracle_indicators(p, u0, v0, p.nsteps)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p) as plan:
        plan.set_indicators(True)
        steps, last = plan.run(u, v, t_end=5.0, tol=0.0, check_every=16)
        log = plan.indicator_log()
    assert steps == 100 and log.shape == (100, 4)
    U, V = u.double().cpu().numpy(), v.double().cpu().numpy()
    assert max(np.max(np.abs(U - Ur)) / np.max(np.abs(Ur)),
               np.max(np.abs(V - Vr)) / np.max(np.abs(Vr))) <= 1e-5
    assert np.allclose(last, log[-1])
    assert abs(log[-1, 0] - ref[-1, 0]) <= 1e-6 * abs(ref[-1, 0])
    floor = 2.0 * np.sqrt(64.0 ** 3) * 2.0 ** -23 * np.array([np.abs(Ur).max(), np.abs(Vr).max()])
    assert np.all(np.abs(log[:, 2:] - ref[:, 2:]) <= 1e-3 * ref[:, 2:] + floor)
    # the increments decay by orders of magnitude, and the means head for (2, 0.5)
    assert max(log[-1, 2:]) < 1e-2 * max(log[0, 2:])
    assert abs(log[-1, 0] - 2.0) < abs(log[0, 0] - 2.0) and abs(log[-1, 1] - 0.5) < 0.1


def test_run_stops_at_a_stationary_state(adr):
    """With tol > 0 the run ends at the first checked step whose increment
    indicator is at most tol, before the horizon."""
    import torch
    p = _bruss_e6(32, 5e-2)
    u0, v0 = wl.brusselator_e6_initial(p)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p) as plan:
        plan.set_indicators(True)
        full = plan.indicator_log()
        assert full.shape == (0, 4)
        steps, last = plan.run(u, v, t_end=50.0, tol=1e-3, check_every=8)
        log = plan.indicator_log()
    assert steps < 1000 and steps % 8 == 0
    assert max(last[2:]) <= 1e-3
    # the previous check was still above tol
    assert max(log[-9, 2:]) > 1e-3
