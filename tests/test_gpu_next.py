"""Widened rows on the GPU: the Lawson2b scheme (Eq. 7) and the paper's other
reaction models (FitzHugh-Nagumo with rho, Eq. 13-14; DIB, Eq. 15), in every
precision, against the FP64 oracle."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as wl
from oracle import schemes, tensor

pytestmark = pytest.mark.gpu

TOL = {wl.FP64: 1e-11, wl.FP32: 1e-5, wl.BF16X3: 1e-5}


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def run(adr, p, u0, v0, nsteps):
    import torch
    dt = adr.state_dtype(p.precision)
    u = torch.tensor(u0, dtype=dt, device="cuda")
    v = torch.tensor(v0, dtype=dt, device="cuda")
    with adr.Plan(p) as plan:
        plan.step(u, v, nsteps)
    torch.cuda.synchronize()
    return u.double().cpu().numpy(), v.double().cpu().numpy()


def lawson_oracle(p, u0, v0, nsteps):
    plan = schemes.make_plan(p)
    U, V = u0, v0
    for _ in range(nsteps):
        U, V = schemes.lawson2b_step(plan, U, V)
    return U, V


@pytest.mark.parametrize("precision", [wl.FP64, wl.FP32, wl.BF16X3])
def test_lawson2b_exact_at_zero_reaction(adr, precision):
    """g = 0: one Lawson2b step is e^{tau K} u exactly (Eq. 5, no splitting)."""
    n = (16, 24)
    p = wl.Problem(d=2, n=n, lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(0.3, 0.7),
                   adv=((0.4, -0.2), (0.1, 0.3)), model=wl.NO_REACTION, params=(),
                   tau=4e-3, nsteps=1, precision=precision, seed=31, scheme=wl.LAWSON2B)
    u0, v0 = wl.initial_data(p, kind="uniform", amp=0.5)
    u0, v0 = wl.round_to(u0, precision), wl.round_to(v0, precision)
    U, V = run(adr, p, u0, v0, 1)
    for c, (X, X0) in enumerate(((U, u0), (V, v0))):
        K = tensor.kron_sum_dense(oracle.direction_matrices(p, c))
        ref = (sl.expm(p.tau * K) @ X0.ravel()).reshape(X0.shape)
        assert np.max(np.abs(X - ref)) <= TOL[precision] * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", [wl.FP64, wl.FP32, wl.BF16X3])
@pytest.mark.parametrize("n", [(40, 24), (16, 24, 32)])
def test_lawson2b_with_reactions(adr, precision, n):
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=wl.BRUSSELATOR,
                   params=(1.0, 3.0), tau=2e-3, nsteps=8, precision=precision, seed=32,
                   scheme=wl.LAWSON2B)
    u0, v0 = wl.initial_data(p, kind="uniform")
    u0, v0 = wl.round_to(u0, precision), wl.round_to(v0, precision)
    Ur, Vr = lawson_oracle(p, u0, v0, p.nsteps)
    U, V = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL[precision]


@pytest.mark.parametrize("precision", [wl.FP64, wl.FP32, wl.BF16X3])
@pytest.mark.parametrize("which", ["dib", "fhn_rho2", "fhn_rho3"])
def test_paper_models(adr, precision, which):
    # the paper's step sizes (DIB: T = 2.5 in 1250 steps; FHN: T = 10 in 20000)
    if which == "dib":
        p = wl.dib_200(precision=precision, n=48, nsteps=1250).replace(nsteps=10)
    elif which == "fhn_rho2":
        p = wl.fhn_rho(2, precision=precision, n=40, nsteps=20000).replace(nsteps=10)
    else:
        p = wl.fhn_rho(3, precision=precision, n=24, nsteps=20000).replace(nsteps=10)
    u0, v0 = wl.initial_data(p, kind="uniform", amp=0.05)
    u0, v0 = wl.round_to(u0, precision), wl.round_to(v0, precision)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    assert np.all(np.isfinite(Ur)) and np.all(np.isfinite(Vr))
    U, V = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL[precision]


def test_lawson2b_batch_equals_alone(adr):
    import torch
    probs = [wl.Problem(d=2, n=n, lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(0.05, 0.3),
                        adv=((0.2, 0.1), (0.1, 0.2)), model=m, params=prm, tau=1e-3, nsteps=20,
                        precision=wl.BF16X3, seed=40 + i, scheme=wl.LAWSON2B)
             for i, (n, m, prm) in enumerate([((64, 96), wl.BRUSSELATOR, (1.0, 3.0)),
                                             ((128, 64), wl.DIB, wl.dib_parameters()),
                                             ((72, 72), wl.SCHNAKENBERG, (200.0, 0.1, 0.9))])]
    plans = [adr.Plan(p) for p in probs]
    init = [tuple(wl.round_to(x, wl.FP32) for x in wl.initial_data(p, kind="uniform"))
            for p in probs]
    us = [torch.tensor(a, dtype=torch.float32, device="cuda") for a, _ in init]
    vs = [torch.tensor(b, dtype=torch.float32, device="cuda") for _, b in init]
    with adr.Batch(plans) as batch:
        assert batch.grouped
        batch.step(us, vs, 20)
    torch.cuda.synchronize()
    for i, plan in enumerate(plans):
        u = torch.tensor(init[i][0], dtype=torch.float32, device="cuda")
        v = torch.tensor(init[i][1], dtype=torch.float32, device="cuda")
        plan.step(u, v, 20)
        torch.cuda.synchronize()
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i])
        plan.close()


@pytest.mark.parametrize("precision", [wl.FP64, wl.BF16X3])
@pytest.mark.parametrize("n", [(40, 24), (16, 24, 32)])
def test_indicators_match_oracle(adr, precision, n):
    """Sec. 4 indicators: spatial mean (trapezoid) and Frobenius increment."""
    import torch
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(2.0,) * d, diff=(0.05, 0.3),
                   adv=((0.1,) * d, (0.2,) * d), model=wl.SCHNAKENBERG, params=(200.0, 0.1, 0.9),
                   tau=1e-3, nsteps=1, precision=precision, seed=33)
    u0, v0 = wl.initial_data(p, kind="uniform", amp=0.3)
    u0, v0 = wl.round_to(u0, precision), wl.round_to(v0, precision)
    dt = adr.state_dtype(precision)
    up = torch.tensor(u0, dtype=dt, device="cuda")
    vp = torch.tensor(v0, dtype=dt, device="cuda")
    u, v = up.clone(), vp.clone()
    with adr.Plan(p) as plan:
        plan.step(u, v, 1)
        got = plan.indicators(up, vp, u, v)
    U, V = u.double().cpu().numpy(), v.double().cpu().numpy()
    mu, iu = oracle.indicators(u0, U)
    mv, iv = oracle.indicators(v0, V)
    assert got[0] == pytest.approx(mu, rel=1e-12) and got[1] == pytest.approx(mv, rel=1e-12)
    assert got[2] == pytest.approx(iu, rel=1e-10) and got[3] == pytest.approx(iv, rel=1e-10)
