"""Tensor-core (tcgen05, BF16x3 split precision) path vs the FP64 oracle.

Tolerance: the 1e-5 max relative error bound (per component
||X - X_ref||_inf / ||X_ref||_inf, maximum over u and v).  The BF16x3 split
carries about 24 significant bits per operand, the same class as FP32.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import schemes

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def run(adr, p, u0, v0, nsteps, precision=wl.BF16X3):
    import torch
    dt = adr.state_dtype(precision)
    u = torch.tensor(u0, dtype=dt, device="cuda")
    v = torch.tensor(v0, dtype=dt, device="cuda")
    with adr.Plan(p.replace(precision=precision)) as plan:
        plan.set_timing(True)
        plan.step(u, v, nsteps)
        st = plan.stats()
    assert st["device_error"] == 0
    return u.double().cpu().numpy(), v.double().cpu().numpy(), st


def inputs(p, kind="auto", amp=None):
    u0, v0 = wl.initial_data(p, kind=kind, amp=amp)
    return wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)


@pytest.mark.parametrize("n", [(64, 64), (200, 136), (24, 40, 56), (264, 40, 24)])
def test_linear_stage_one(adr, n):
    """g = 0: the step is U + tau (K U) x_mu phi_1 (stage 2 adds zero), which
    isolates the stencil kernel and the stage-1 tensor-core products."""
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.02, 0.05),
                   adv=((0.3,) * d, (-0.2,) * d), model=wl.NO_REACTION, params=(),
                   tau=1e-2, nsteps=1, seed=21)
    u0, v0 = inputs(p, kind="uniform", amp=0.5)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, 1)
    U, V, st = run(adr, p, u0, v0, 1)
    # 2D: one fused launch per Tucker operator; 3D: the fused first two
    # directions, then the third
    assert st["kernels"]["mode_product_tc"]["count"] == (2 if d == 2 else 4)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("n,model", [((200, 136), wl.FHN), ((128, 256), wl.SCHNAKENBERG),
                                     ((40, 24, 56), wl.BRUSSELATOR), ((8, 16, 8), wl.FHN),
                                     ((136, 24, 40), wl.BRUSSELATOR)])
def test_ragged_shapes_bf16x3(adr, n, model):
    d = len(n)
    params = {wl.SCHNAKENBERG: (200.0, 0.1, 0.9), wl.FHN: (0.05, 2.0, -0.03),
              wl.BRUSSELATOR: (1.0, 3.0)}[model]
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=model,
                   params=params, tau=2e-3, nsteps=10, seed=13)
    u0, v0 = inputs(p, kind="uniform")
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    U, V, _ = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("fuse", ["0", "1", "2"])
@pytest.mark.parametrize("n", [(72, 200), (24, 40, 56), (136, 64)])
def test_stage_one_fusion_both_ways(adr, n, fuse, monkeypatch):
    """The stage-1 combination and reaction difference done by a separate
    kernel (0), fused into the last tensor-core product with u and v of a
    tile in one CTA (1), or fused with u and v in the two CTAs of a cluster
    exchanging U2 and V2 (2) must all match the oracle."""
    monkeypatch.setenv("ADR_TC_FUSE", fuse)
    monkeypatch.setenv("ADR_TC_VARIANT", "0")
    monkeypatch.setenv("ADR_TC_FUSED", "0")  # these epilogues belong to per-direction passes
    d = len(n)
    # the fused epilogues carry a plain FP32 state (a compensated plan keeps
    # the separate kernel)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=wl.SCHNAKENBERG,
                   params=(300.0, 0.1, 0.9), tau=1e-3, nsteps=6, seed=17, state=wl.STATE_PLAIN)
    u0, v0 = inputs(p, kind="uniform")
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["reaction_diff"]["count"] == (0 if fuse != "0" else p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_fhn_1024_full_size_steps(adr):
    p = wl.fhn_1024(precision=wl.BF16X3)
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, 3)
    U, V, _ = run(adr, p, u0, v0, 3)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_brusselator_256_full_size_step(adr):
    p = wl.brusselator_256(precision=wl.BF16X3)
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, 1)
    U, V, _ = run(adr, p, u0, v0, 1)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_unsupported_grid_rejected(adr):
    p = wl.fhn_1024(precision=wl.BF16X3, n=100)  # 100 % 8 != 0
    with pytest.raises(adr.AdrError) as ei:
        adr.Plan(p)
    assert ei.value.status == adr.ADR_EUNSUPPORTED


def test_bf16x3_not_less_accurate_than_fp32(adr):
    """On a 256^2 FHN run of 100 steps the split-precision tensor-core result
    is at least as close to FP64 as the plain FP32 result (within 2x)."""
    p = wl.fhn_1024(n=256, nsteps=100)
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    Ub, Vb, _ = run(adr, p, u0, v0, p.nsteps, wl.BF16X3)
    Uf, Vf, _ = run(adr, p, u0, v0, p.nsteps, wl.FP32)
    eb = oracle.max_rel_err(Ub, Vb, Ur, Vr)
    ef = oracle.max_rel_err(Uf, Vf, Ur, Vr)
    assert eb <= TOL and ef <= TOL
    assert eb <= 2.0 * ef, (eb, ef)


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4"])
@pytest.mark.parametrize("n", [(200, 136), (40, 24, 56), (256, 384)])
def test_kernel_variants(adr, n, variant, monkeypatch):
    """Every mode-product kernel variant (one-CTA tiles of 128 x 128 or
    128 x 64 with 64- or 128-byte swizzle; CTA-pair tiles of 256 x 128)
    matches the oracle, including grids whose sizes are not multiples of the
    tile sizes."""
    monkeypatch.setenv("ADR_TC_VARIANT", variant)
    monkeypatch.setenv("ADR_TC_FUSED", "0")  # 2D grids too: one launch per direction
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=wl.FHN,
                   params=(0.05, 2.0, -0.03), tau=2e-3, nsteps=5, seed=19)
    u0, v0 = inputs(p, kind="uniform")
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps)
    assert st["kernels"]["mode_product_tc"]["count"] == 2 * d * p.nsteps
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_largest_direction_bf16x3(adr):
    """The largest direction the tensor path takes, n = 4096 (with 512 in the
    other direction), two steps against the oracle.  The oracle's matrix
    functions come from its eigen route (exact for these symmetric operators,
    no advection), because Pade on the 3n x 3n augmented matrix takes minutes
    at this size."""
    from oracle import fd, matfun
    p = wl.Problem(d=2, n=(4096, 512), lo=(0.0, 0.0), hi=(100.0, 100.0), diff=(1.0, 20.0),
                   adv=((0.0, 0.0), (0.0, 0.0)), model=wl.FHN, params=(0.05, 2.0, -0.03),
                   tau=1e-2, nsteps=2, precision=wl.BF16X3, seed=23)
    A = [fd.direction_matrices(p, 0), fd.direction_matrices(p, 1)]
    fns = [[matfun.phi_eigen(p.tau * Am) for Am in A[c]] for c in range(2)]
    plan = schemes.Plan(d=2, tau=p.tau, model=p.model, params=tuple(p.params), A=A,
                        E=[[f[0] for f in fc] for fc in fns],
                        phi1=[[f[1] for f in fc] for fc in fns],
                        phi2=[[f[2] for f in fc] for fc in fns])
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(plan, u0, v0, p.nsteps)
    U, V, _ = run(adr, p, u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


@pytest.mark.parametrize("n,model", [((200, 136), wl.FHN), ((40, 24, 56), wl.BRUSSELATOR),
                                     ((128, 256), wl.SCHNAKENBERG)])
def test_tf32x3_ragged_shapes(adr, n, model):
    """TF32 hi + lo tensor-core products (kind::tf32, three MMAs) on grids
    that are not multiples of the tile sizes, against the oracle."""
    d = len(n)
    params = {wl.SCHNAKENBERG: (200.0, 0.1, 0.9), wl.FHN: (0.05, 2.0, -0.03),
              wl.BRUSSELATOR: (1.0, 3.0)}[model]
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=model,
                   params=params, tau=2e-3, nsteps=10, seed=13)
    u0, v0 = inputs(p, kind="uniform")
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    U, V, st = run(adr, p, u0, v0, p.nsteps, wl.TF32X3)
    assert st["kernels"]["mode_product_tc"]["count"] == 2 * d * p.nsteps
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_tf32x3_fhn_1024_full_size_steps(adr):
    p = wl.fhn_1024(precision=wl.TF32X3)
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, 3)
    U, V, _ = run(adr, p, u0, v0, 3, wl.TF32X3)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL


def test_split_precisions_ordered_by_accuracy(adr):
    """On a 256^2 FHN run of 100 steps: BF16x3 (about 24 bits per operand)
    is at least as accurate as TF32x3 (about 22 bits), and both stay within
    a small factor of plain FP32."""
    p = wl.fhn_1024(n=256, nsteps=100)
    u0, v0 = inputs(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)
    errs = {}
    for prec in (wl.BF16X3, wl.TF32X3, wl.FP32):
        U, V, _ = run(adr, p, u0, v0, p.nsteps, prec)
        errs[prec] = oracle.max_rel_err(U, V, Ur, Vr)
    assert errs[wl.BF16X3] <= 1.5 * errs[wl.TF32X3], errs
    assert errs[wl.TF32X3] <= 20.0 * errs[wl.FP32], errs


@pytest.mark.parametrize("n", [(256, 384), (40, 24, 56)])
def test_every_kernel_choice_gives_the_same_result(adr, n):
    """Plans created with each tensor-core kernel (adr_plan_create_tuned)
    accumulate every output's products in the same K order, so their results
    are bitwise identical."""
    import torch
    d = len(n)
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.05, 0.3),
                   adv=((0.2, -0.1, 0.3)[:d], (-0.2, 0.1, 0.05)[:d]), model=wl.FHN,
                   params=(0.05, 2.0, -0.03), tau=2e-3, nsteps=5, precision=wl.BF16X3, seed=29)
    u0, v0 = inputs(p, kind="uniform")
    outs = []
    for k in range(5):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        with adr.Plan(p, kernel=k) as plan:
            plan.step(u, v, p.nsteps)
        torch.cuda.synchronize()
        outs.append((u.cpu(), v.cpu()))
    for k in range(1, 5):
        assert torch.equal(outs[k][0], outs[0][0]) and torch.equal(outs[k][1], outs[0][1]), k


def test_autotune_times_every_candidate(adr):
    """adr_autotune times each tensor-core kernel on the problem's grid and
    returns the fastest; FP32 problems have nothing to tune."""
    p = wl.fhn_1024(precision=wl.BF16X3, n=512)
    best, ms = adr.autotune(p, nsteps=8, cache=False)
    assert set(ms) == {0, 1, 2, 3, 4} and all(t > 0 for t in ms.values())
    assert best == min(ms, key=ms.get)
    bt, mt = adr.autotune(p.replace(precision=wl.TF32X3), nsteps=8, cache=False)
    assert bt == 1 and set(mt) == {1}
    assert adr.autotune(p.replace(precision=wl.FP32), nsteps=8, cache=False) == (-1, {})


@pytest.mark.gpu
def test_set_kernel_keeps_the_plan_and_its_results(adr):
    """adr_plan_set_kernel swaps the tensor-core kernel of a live plan; its
    steps stay bitwise equal to a plan created with that kernel."""
    import torch
    p = wl.fhn_1024(precision=wl.BF16X3, n=256, nsteps=20)
    u0, v0 = wl.initial_data(p)

    def run(plan):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        plan.step(u, v, p.nsteps)
        torch.cuda.synchronize()
        return u.cpu(), v.cpu()

    with adr.Plan(p, kernel=4) as ref_plan:
        ref = run(ref_plan)
    with adr.Plan(p, kernel=0) as plan:
        run(plan)
        for k in (4, 2, 3):
            plan.set_kernel(k)
            got = run(plan)
            assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), k


@pytest.mark.gpu
def test_autotune_batch_times_the_whole_batch(adr):
    """autotune_batch times every kernel on the batch itself and leaves its
    plans on the fastest one, which then steps like any batch."""
    import torch
    probs = [wl.fhn_1024(precision=wl.BF16X3, n=n, nsteps=6) for n in (64, 128, 96, 64)]
    plans = [adr.Plan(p) for p in probs]
    best, ms = adr.autotune_batch(plans, nsteps=2)
    assert set(ms) == {0, 1, 2, 3, 4} and best == min(ms, key=ms.get)
    us, vs = [], []
    for p in probs:
        u0, v0 = wl.initial_data(p)
        us.append(torch.tensor(u0, dtype=torch.float32, device="cuda"))
        vs.append(torch.tensor(v0, dtype=torch.float32, device="cuda"))
    with adr.Batch(plans) as b:
        b.step(us, vs, 6)
    torch.cuda.synchronize()
    for p, u, v in zip(probs, us, vs):
        with adr.Plan(p, kernel=best) as one:
            u0, v0 = wl.initial_data(p)
            u1 = torch.tensor(u0, dtype=torch.float32, device="cuda")
            v1 = torch.tensor(v0, dtype=torch.float32, device="cuda")
            one.step(u1, v1, 6)
        torch.cuda.synchronize()
        assert torch.equal(u1, u) and torch.equal(v1, v)
    for pl in plans:
        pl.close()
