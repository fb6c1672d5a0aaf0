"""Fused two-mode products (modes 1 and 2 of the Tucker operator, Eq. 5, in
one launch; the intermediate stays in TMEM) against the FP64 oracle.

With BF16x3 products the first two directions of every Tucker operator run
as one fused launch by default: the whole operator on 2D grids; on 3D grids
the fused launch works on every x3 slab and writes its pieces in the natural
layout, and the x3 product reads them as an MN-major operand.

Covered here: grids that are not multiples of the 128 x 128 tile, grids
smaller than one tile, x2 ranges wider than the kernel's 256 intermediate
columns (several groups per tile), each reaction model and both schemes, the
compensated state, every per-direction kernel for the x3 product, and
agreement with the per-direction launches (ADR_TC_FUSED=0) to rounding level,
in 2D and 3D.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import schemes

pytestmark = pytest.mark.gpu

TOL = 1e-5
PARAMS = {wl.SCHNAKENBERG: (200.0, 0.1, 0.9), wl.FHN: (0.05, 2.0, -0.03),
          wl.BRUSSELATOR: (1.0, 3.0)}


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
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p) as plan:
        plan.set_timing(True)
        plan.step(u, v, nsteps)
        st = plan.stats()
    assert st["device_error"] == 0
    return u.double().cpu().numpy(), v.double().cpu().numpy(), st


def problem(n, model, hi=1.0, diff=(0.05, 0.3), tau=2e-3, nsteps=10, scheme=wl.ETD2RKDS,
            state=wl.STATE_AUTO, seed=51):
    return wl.Problem(d=2, n=n, lo=(0.0, 0.0), hi=(hi, hi), diff=diff,
                      adv=((0.2, -0.1), (-0.2, 0.1)), model=model, params=PARAMS[model],
                      tau=tau, nsteps=nsteps, precision=wl.BF16X3, seed=seed, scheme=scheme,
                      state=state)


def inputs(p):
    u0, v0 = wl.initial_data(p, kind="uniform")
    return wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)


def oracle_run(p, u0, v0, nsteps):
    plan = schemes.make_plan(p)
    if p.scheme == wl.LAWSON2B:
        for _ in range(nsteps):
            u0, v0 = schemes.lawson2b_step(plan, u0, v0)
        return u0, v0
    return schemes.etd2rkds_solve(plan, u0, v0, nsteps)


@pytest.mark.parametrize("n,model", [((200, 136), wl.FHN), ((72, 200), wl.SCHNAKENBERG),
                                     ((128, 256), wl.BRUSSELATOR), ((8, 16), wl.FHN),
                                     ((64, 64), wl.SCHNAKENBERG), ((264, 392), wl.FHN)])
def test_fused_matches_oracle(adr, n, model):
    p = problem(n, model)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 2 * p.nsteps  # one per Tucker operator
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("n", [(136, 520), (200, 384)])
def test_fused_several_x2_groups(adr, n, monkeypatch):
    """Without the column supports every tile contracts over all of x2,
    which is wider than the 256 intermediate columns: MMA1 and MMA2 run in
    groups and D2 accumulates across them."""
    monkeypatch.setenv("ADR_KSUPPORT", "0")
    p = problem(n, wl.FHN)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V, _ = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fused_wide_supports(adr):
    """A step for which the matrix functions are nearly dense (large
    diffusion on a short domain): the supports cover all of x2 and x1."""
    p = problem((168, 320), wl.SCHNAKENBERG, diff=(1.0, 20.0), tau=1e-2)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, 4)
    U, V, _ = run(adr, p, u0, v0, 4)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fused_lawson2b(adr):
    p = problem((200, 136), wl.FHN, scheme=wl.LAWSON2B)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 2 * p.nsteps
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fused_compensated_state(adr):
    p = problem((200, 136), wl.SCHNAKENBERG, state=wl.STATE_COMPENSATED, nsteps=40)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V, _ = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("n", [(1024, 1024), (264, 392)])
def test_fused_agrees_with_per_direction_launches(adr, n, monkeypatch):
    """The fused operator and the per-direction launches compute the same
    products in different association: they agree to rounding level."""
    if n == (1024, 1024):
        p = wl.fhn_1024(precision=wl.BF16X3, nsteps=10)
        u0, v0 = wl.initial_data(p)
        u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    else:
        p = problem(n, wl.FHN)
        u0, v0 = inputs(p)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    monkeypatch.setenv("ADR_TC_FUSED", "0")
    Ud, Vd, std = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 2 * p.nsteps
    assert std["kernels"]["mode_product_tc"]["count"] == 4 * p.nsteps
    assert oracle.max_rel_err(U, V, Ud, Vd) <= 1e-6
    assert np.isfinite(U).all() and np.isfinite(V).all()


def problem3(n, model, nsteps=6, scheme=wl.ETD2RKDS, state=wl.STATE_AUTO, seed=61):
    return wl.Problem(d=3, n=n, lo=(0.0,) * 3, hi=(1.0,) * 3, diff=(0.02, 0.1),
                      adv=((0.2, -0.1, 0.3), (-0.2, 0.1, 0.05)), model=model, params=PARAMS[model],
                      tau=2e-3, nsteps=nsteps, precision=wl.BF16X3, seed=seed, scheme=scheme,
                      state=state)


@pytest.mark.parametrize("n,model", [((40, 24, 56), wl.BRUSSELATOR), ((136, 24, 40), wl.FHN),
                                     ((64, 200, 72), wl.SCHNAKENBERG), ((8, 16, 8), wl.FHN),
                                     ((128, 128, 136), wl.BRUSSELATOR)])
def test_fused_3d_matches_oracle(adr, n, model):
    """3D: the fused pass per x3 slab (pieces out, natural layout) and the x3
    product on an MN-major operand, over ragged sides (M = n1 n2 not a
    multiple of 128, x3 not a multiple of the K-block)."""
    p = problem3(n, model)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 4 * p.nsteps  # two per Tucker operator
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("kernel", [0, 1, 2, 3, 4])
def test_fused_3d_every_kernel(adr, kernel):
    """The x3 product on an MN-major operand in every per-direction kernel
    (one-CTA and CTA-pair, 64- and 128-byte swizzle of the other operand)."""
    import torch
    p = problem3((72, 40, 48), wl.FHN)
    u0, v0 = inputs(p)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p, kernel=kernel) as plan:
        plan.step(u, v, p.nsteps)
        assert plan.stats()["device_error"] == 0
    U, V = u.double().cpu().numpy(), v.double().cpu().numpy()
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fused_3d_lawson_and_compensated(adr):
    for p in (problem3((40, 24, 56), wl.FHN, scheme=wl.LAWSON2B),
              problem3((40, 24, 56), wl.SCHNAKENBERG, state=wl.STATE_COMPENSATED, nsteps=20)):
        u0, v0 = inputs(p)
        Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
        U, V, _ = run(adr, p, u0, v0, p.nsteps)
        assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fused_3d_agrees_with_per_direction_launches(adr, monkeypatch):
    p = problem3((128, 96, 64), wl.BRUSSELATOR, nsteps=8)
    u0, v0 = inputs(p)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    monkeypatch.setenv("ADR_TC_FUSED", "0")
    Ud, Vd, std = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 4 * p.nsteps
    assert std["kernels"]["mode_product_tc"]["count"] == 6 * p.nsteps
    assert oracle.max_rel_err(U, V, Ud, Vd) <= 1e-6


def test_fused_batch_of_uneven_chunk_counts(adr):
    """A grouped launch over solves whose units have different numbers of
    64-column chunks per group (x2 sides 64, 136, 256, 520): every solve gets
    the result it gets alone, bit for bit, and matches the oracle."""
    import torch
    probs = [problem(n, m, seed=70 + i, nsteps=6)
             for i, (n, m) in enumerate([((136, 64), wl.FHN), ((200, 256), wl.SCHNAKENBERG),
                                         ((72, 136), wl.BRUSSELATOR), ((128, 520), wl.FHN)])]
    inits = [inputs(p) for p in probs]
    plans = [adr.Plan(p) for p in probs]
    us = [torch.tensor(u0, dtype=torch.float32, device="cuda") for u0, _ in inits]
    vs = [torch.tensor(v0, dtype=torch.float32, device="cuda") for _, v0 in inits]
    with adr.Batch(plans) as batch:
        batch.step(us, vs, 6)
    torch.cuda.synchronize()
    for i, (p, pl, (u0, v0)) in enumerate(zip(probs, plans, inits)):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        pl.step(u, v, 6)
        torch.cuda.synchronize()
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i]), i
        Ur, Vr = oracle_run(p, u0, v0, 6)
        assert oracle.max_rel_err(u.double().cpu().numpy(), v.double().cpu().numpy(), Ur, Vr) <= TOL, i
        assert pl.stats()["device_error"] == 0
    for pl in plans:
        pl.close()
