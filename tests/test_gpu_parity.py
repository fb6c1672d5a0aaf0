"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances: FP64 runs must match the oracle to rounding (1e-11 relative in
max norm, allowing for the different summation orders over a few hundred
steps).  FP32-class runs must stay within the 1e-5 max relative error bound
(per component ||X - X_ref||_inf / ||X_ref||_inf, maximum over u and v).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import matfun, schemes

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-11


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def run_gpu(adr, p, u0, v0, nsteps, precision):
    import torch
    dt = adr.state_dtype(precision)
    u = torch.tensor(u0, dtype=dt, device="cuda").contiguous()
    v = torch.tensor(v0, dtype=dt, device="cuda").contiguous()
    with adr.Plan(p.replace(precision=precision)) as plan:
        plan.step(u, v, nsteps)
        torch.cuda.synchronize()
    return u.double().cpu().numpy(), v.double().cpu().numpy()


def oracle_run(p, u0, v0, nsteps):
    return schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, nsteps)


def inputs(p, precision, kind="auto"):
    u0, v0 = wl.initial_data(p, kind=kind)
    return wl.round_to(u0, precision), wl.round_to(v0, precision)


# ---------------------------------------------------------------- matrix functions
@pytest.mark.parametrize("n,L,delta,alpha,tau", [
    (64, 1.0, 10.0, 0.0, 5e-4),      # 64^2 Schnakenberg, v component
    (37, 1.0, 0.02, -0.5, 1e-2),     # ragged, advective
    (129, 100.0, 20.0, 0.5, 1e-2),   # FHN-like, scaling power > 0
    (256, 1.0, 0.1, -0.5, 1e-2),     # 256^3 Brusselator, v component
])
def test_matrix_functions_match_oracle(adr, n, L, delta, alpha, tau):
    p = wl.Problem(d=2, n=(n, 5), lo=(0.0, 0.0), hi=(L, 1.0), diff=(delta, delta),
                   adv=((alpha, 0.0), (alpha, 0.0)), model=wl.NO_REACTION, params=(),
                   tau=tau, nsteps=1, precision=wl.FP64)
    with adr.Plan(p) as plan:
        A = plan.matrix(0, 0, 0)
        E, P1, P2 = (plan.matrix(w, 0, 0) for w in (1, 2, 3))
    Aref = oracle.fd_matrix(n, 0.0, L, delta, alpha)
    assert np.max(np.abs(A - Aref)) <= 1e-12 * np.max(np.abs(Aref))
    Er, P1r, P2r = matfun.phi_augmented(tau * Aref)
    for got, ref in ((E, Er), (P1, P1r), (P2, P2r)):
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_matrix_functions_identities_at_max_size(adr):
    """n = 4096 (the largest direction the ABI accepts): check X phi_1 = e^X - I
    and X phi_2 = phi_1 - I on sampled columns, properties that hold at any size."""
    n = 4096
    p = wl.Problem(d=2, n=(n, 3), lo=(0.0, 0.0), hi=(100.0, 1.0), diff=(20.0, 20.0),
                   adv=((0.5, 0.0), (0.5, 0.0)), model=wl.NO_REACTION, params=(),
                   tau=1e-2, nsteps=1, precision=wl.FP64)
    with adr.Plan(p) as plan:
        A = plan.matrix(0, 0, 0)
        E, P1, P2 = (plan.matrix(w, 0, 0) for w in (1, 2, 3))
    X = 1e-2 * A
    cols = np.random.default_rng(0).choice(n, 32, replace=False)
    I = np.eye(n)[:, cols]
    assert np.max(np.abs(X @ P1[:, cols] - (E[:, cols] - I))) <= 1e-11
    assert np.max(np.abs(X @ P2[:, cols] - (P1[:, cols] - I))) <= 1e-11


# ---------------------------------------------------------------- FP64 stepping
def test_schnakenberg_64_fp64_full_run(adr):
    """2D Schnakenberg 64x64, FP64, 200 steps to T = 0.1 against the oracle."""
    p = wl.schnakenberg_64(precision=wl.FP64)
    u0, v0 = inputs(p, wl.FP64)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V = run_gpu(adr, p, u0, v0, p.nsteps, wl.FP64)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= FP64_TOL


@pytest.mark.parametrize("n,model", [((37, 53), wl.FHN), ((3, 3), wl.SCHNAKENBERG),
                                     ((130, 17), wl.BRUSSELATOR), ((13, 17, 11), wl.BRUSSELATOR),
                                     ((5, 3, 140), wl.FHN), ((3, 3, 3), wl.SCHNAKENBERG)])
def test_ragged_shapes_fp64(adr, n, model):
    d = len(n)
    params = {wl.SCHNAKENBERG: (200.0, 0.1, 0.9), wl.FHN: (0.05, 2.0, -0.03),
              wl.BRUSSELATOR: (1.0, 3.0)}[model]
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=model,
                   params=params, tau=2e-3, nsteps=7, precision=wl.FP64, seed=11)
    u0, v0 = inputs(p, wl.FP64, kind="uniform")
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V = run_gpu(adr, p, u0, v0, p.nsteps, wl.FP64)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= FP64_TOL


# ---------------------------------------------------------------- FP32 stepping
@pytest.mark.parametrize("n", [(200, 131), (129, 257), (33, 40, 21)])
def test_ragged_shapes_fp32(adr, n):
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(100.0,) * d, diff=(1.0, 20.0),
                   adv=((0.5,) * d, (0.5,) * d), model=wl.FHN, params=(0.05, 2.0, -0.03),
                   tau=1e-2, nsteps=20, precision=wl.FP32, seed=12)
    u0, v0 = inputs(p, wl.FP32)
    Ur, Vr = oracle_run(p, u0, v0, p.nsteps)
    U, V = run_gpu(adr, p, u0, v0, p.nsteps, wl.FP32)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= FP32_TOL


def test_fhn_1024_fp32_full_size_steps(adr):
    """FHN with advection at the full 1024^2 size, 3 steps, against the oracle."""
    p = wl.fhn_1024(precision=wl.FP32)
    u0, v0 = inputs(p, wl.FP32)
    Ur, Vr = oracle_run(p, u0, v0, 3)
    U, V = run_gpu(adr, p, u0, v0, 3, wl.FP32)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= FP32_TOL


def test_brusselator_256_fp32_full_size_step(adr):
    """3D advective Brusselator at the full 256^3 size, 1 step."""
    p = wl.brusselator_256(precision=wl.FP32)
    u0, v0 = inputs(p, wl.FP32)
    Ur, Vr = oracle_run(p, u0, v0, 1)
    U, V = run_gpu(adr, p, u0, v0, 1, wl.FP32)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= FP32_TOL


# ---------------------------------------------------------------- behaviour
def test_zero_steps_and_equilibrium(adr):
    import torch
    p = wl.schnakenberg_64(precision=wl.FP32).replace(n=(50, 30))
    ue, ve = wl.equilibrium(p.model, p.params)
    u = torch.full((30, 50), ue, dtype=torch.float32, device="cuda")
    v = torch.full((30, 50), ve, dtype=torch.float32, device="cuda")
    u0 = u.clone()
    with adr.Plan(p) as plan:
        plan.step(u, v, 0)
        torch.cuda.synchronize()
        assert torch.equal(u, u0)
        plan.step(u, v, 50)
        torch.cuda.synchronize()
    assert float((u - ue).abs().max()) <= 1e-5 * ue


def test_solve_host_buffers_equals_device_step(adr):
    import torch
    p = wl.fhn_1024(precision=wl.FP32, n=96)
    u0, v0 = inputs(p, wl.FP32)
    hu = torch.tensor(u0, dtype=torch.float32).pin_memory()
    hv = torch.tensor(v0, dtype=torch.float32).pin_memory()
    ou, ov = torch.empty_like(hu).pin_memory(), torch.empty_like(hv).pin_memory()
    du, dv = hu.cuda(), hv.cuda()
    with adr.Plan(p) as plan:
        plan.solve(hu, hv, ou, ov, 9)
        plan.step(du, dv, 9)
        torch.cuda.synchronize()
    assert torch.equal(ou, du.cpu()) and torch.equal(ov, dv.cpu())


def test_invalid_pointers_rejected(adr):
    import torch
    p = wl.fhn_1024(precision=wl.FP32, n=32)
    with adr.Plan(p) as plan:
        u = torch.zeros((32, 32), device="cuda")
        with pytest.raises(adr.AdrError):
            adr._abi.check(adr.lib().adr_step(plan._p, u.data_ptr(), u.data_ptr(), 1))
        with pytest.raises(adr.AdrError):
            adr._abi.check(adr.lib().adr_step(plan._p, u.data_ptr(), None, 1))
        h = torch.zeros((32, 32))
        with pytest.raises(adr.AdrError):
            adr._abi.check(adr.lib().adr_step(plan._p, h.data_ptr(), u.data_ptr(), 1))


def test_timing_stats(adr):
    import torch
    p = wl.fhn_1024(precision=wl.FP32, n=128)
    u0, v0 = inputs(p, wl.FP32)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p) as plan:
        plan.set_timing(True)
        plan.step(u, v, 4)
        st = plan.stats()
    assert st["steps"] == 4 and st["launches"] == 4 * 6
    k = st["kernels"]["mode_product_simt"]
    assert k["count"] == 16 and k["ms"] > 0 and k["flops"] == pytest.approx(16 * 4 * 128 * 128 * 128)


@pytest.mark.parametrize("precision", [wl.FP64, wl.FP32, wl.BF16X3])
def test_graph_replay_matches_direct_launches(adr, precision, monkeypatch):
    """adr_step replays captured CUDA graphs for runs of >= 32 steps; the
    result must be bitwise identical to launching every kernel directly."""
    import torch
    p = wl.fhn_1024(precision=precision, n=64, nsteps=70)
    u0, v0 = inputs(p, precision)
    dt = adr.state_dtype(precision)
    outs = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("ADR_GRAPHS", graphs)
        u = torch.tensor(u0, dtype=dt, device="cuda")
        v = torch.tensor(v0, dtype=dt, device="cuda")
        with adr.Plan(p) as plan:
            plan.step(u, v, p.nsteps)
            st = plan.stats()
        outs.append((u.cpu(), v.cpu(), st))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert outs[0][2]["launches"] == outs[1][2]["launches"]
    assert outs[0][2]["steps"] == outs[1][2]["steps"] == p.nsteps


def test_timed_graph_replay(adr):
    """With timing on, adr_step replays graph chunks that carry event-record
    nodes around every kernel: the result is bitwise that of the untimed run
    and every launch is timed."""
    import torch
    p = wl.fhn_1024(precision=wl.BF16X3, n=64, nsteps=70)
    u0, v0 = inputs(p, wl.BF16X3)
    outs = []
    for timing in (False, True):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        with adr.Plan(p) as plan:
            plan.set_timing(timing)
            plan.step(u, v, p.nsteps)
            st = plan.stats()
        outs.append((u.cpu(), v.cpu(), st))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    st = outs[1][2]
    # a 2D step: stencil, fused Tucker operator, reaction difference, fused Tucker operator
    assert st["launches"] == 4 * p.nsteps and st["device_error"] == 0
    k = st["kernels"]
    assert k["mode_product_tc"]["count"] == 2 * p.nsteps
    assert k["rhs_stencil_reaction"]["count"] == p.nsteps == k["reaction_diff"]["count"]
    assert all(k[c]["ms"] > 0 for c in ("mode_product_tc", "rhs_stencil_reaction", "reaction_diff"))
