"""Batched solves (many independent grids of uneven sizes advanced by grouped
launches): every result must equal the same solve run alone, and match the
FP64 oracle within the 1e-5 max relative error bound."""
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


def mixed_problems(d=2, count=6, precision=wl.BF16X3):
    sides = (64, 96, 128, 72, 136, 192) if d == 2 else (24, 40, 16, 32, 48, 56)
    out = []
    for i in range(count):
        n = (sides[i % len(sides)], sides[(i + 2) % len(sides)])
        if d == 3:
            n = n + (sides[(i + 4) % len(sides)],)
        if i % 2 == 0:
            p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(1.0, 5.0 + 3 * i),
                           adv=((0.0,) * d, (0.0,) * d), model=wl.SCHNAKENBERG,
                           params=(100.0 + 150 * i, 0.1, 0.9), tau=2e-4, nsteps=20,
                           precision=precision, seed=1000 + i)
        else:
            p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(100.0,) * d, diff=(1.0, 5.0 + 3 * i),
                           adv=((0.5,) * d, (0.5,) * d), model=wl.FHN, params=(0.05, 2.0, -0.03),
                           tau=1e-2, nsteps=20, precision=precision, seed=1000 + i)
        out.append(p)
    return out


def states(adr, probs):
    import torch
    us, vs, inits = [], [], []
    for p in probs:
        u0, v0 = wl.initial_data(p)
        u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
        inits.append((u0, v0))
        us.append(torch.tensor(u0, dtype=torch.float32, device="cuda"))
        vs.append(torch.tensor(v0, dtype=torch.float32, device="cuda"))
    return us, vs, inits


@pytest.mark.parametrize("d", [2, 3])
def test_batch_equals_alone_and_oracle(adr, d):
    import torch
    probs = mixed_problems(d)
    nsteps = 20
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    with adr.Batch(plans) as batch:
        assert batch.grouped
        batch.step(us, vs, nsteps)
        st = batch.stats()
    torch.cuda.synchronize()
    assert st["device_error"] == 0
    for i, (p, plan) in enumerate(zip(probs, plans)):
        u = torch.tensor(inits[i][0], dtype=torch.float32, device="cuda")
        v = torch.tensor(inits[i][1], dtype=torch.float32, device="cuda")
        plan.step(u, v, nsteps)
        torch.cuda.synchronize()
        # alone vs in the mix: the same kernels on the same tiles, bit for bit
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i]), i
        Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), *inits[i], nsteps)
        err = oracle.max_rel_err(us[i].double().cpu().numpy(), vs[i].double().cpu().numpy(),
                                 Ur, Vr)
        assert err <= TOL, (i, err)
    for plan in plans:
        plan.close()


def test_batch_graph_replay_matches_direct(adr, monkeypatch):
    import torch
    probs = mixed_problems(2, count=4)
    outs = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("ADR_GRAPHS", graphs)
        plans = [adr.Plan(p) for p in probs]
        us, vs, _ = states(adr, probs)
        with adr.Batch(plans) as batch:
            batch.step(us, vs, 35)
            st = batch.stats()
        torch.cuda.synchronize()
        outs.append(([u.cpu() for u in us], [v.cpu() for v in vs], st))
        for plan in plans:
            plan.close()
    for a, b in zip(outs[0][0] + outs[0][1], outs[1][0] + outs[1][1]):
        assert torch.equal(a, b)
    # a 2D step: stencil, fused Tucker operator, reaction difference, fused Tucker operator
    assert outs[0][2]["launches"] == outs[1][2]["launches"] == 35 * 4
    assert outs[0][2]["steps"] == 35


def test_batch_of_fp32_plans_steps_each(adr):
    import torch
    probs = mixed_problems(2, count=3, precision=wl.FP32)
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    with adr.Batch(plans) as batch:
        assert not batch.grouped
        batch.step(us, vs, 5)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), *inits[i], 5)
        assert oracle.max_rel_err(us[i].double().cpu().numpy(), vs[i].double().cpu().numpy(),
                                  Ur, Vr) <= TOL
    for plan in plans:
        plan.close()


def test_batch_churn_without_synchronisation(adr):
    """Batches created, stepped and destroyed back to back on one stream with
    no synchronisation in between (descriptor uploads through the page-locked
    ring, stream-ordered batch memory, deferred teardown): every solve equals
    the same solve stepped alone.  The loop uploads more descriptor bytes than
    the ring's first capacity, so the ring wraps and waits for its events.
    The compensated state is carried across calls (ADR_STATE_COMPENSATED),
    so 40 one-step calls in changing batches equal one call of 40 steps."""
    import torch
    probs = [p.replace(state=wl.STATE_COMPENSATED) for p in mixed_problems(d=2, count=6)]
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    ref = []
    for p, pl, (u0, v0) in zip(probs, plans, inits):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        pl.step(u, v, 40)
        ref.append((u, v))
    steps_done = [0] * len(probs)
    rounds = 0
    for r in range(120):  # about 120 x 5 x (4 passes x 768 B + ...) > 1 MB of uploads
        members = [i for i in range(len(probs)) if (i + r) % 6 != 0]
        members = [i for i in members if steps_done[i] < 40]
        if len(members) < 2:
            break
        b = adr.Batch([plans[i] for i in members])
        b.step([us[i] for i in members], [vs[i] for i in members], 1)
        for i in members:
            steps_done[i] += 1
        b.close()
        rounds += 1
    for i, pl in enumerate(plans):
        if steps_done[i] < 40:
            pl.step(us[i], vs[i], 40 - steps_done[i])
    torch.cuda.synchronize()
    assert rounds > 30
    for i in range(len(probs)):
        assert torch.equal(us[i], ref[i][0]) and torch.equal(vs[i], ref[i][1]), i
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("d", [2, 3])
def test_batch_with_cluster_exchange_equals_alone(adr, d, monkeypatch):
    """Grouped batches whose stage-1 reaction difference is fused through the
    two-CTA cluster exchange give every solve the result it gets alone."""
    import torch
    monkeypatch.setenv("ADR_TC_FUSE", "2")
    monkeypatch.setenv("ADR_TC_FUSED", "0")  # the exchange belongs to per-direction passes
    probs = mixed_problems(d=d, count=5)
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    b = adr.Batch(plans)
    assert b.grouped
    b.step(us, vs, 20)
    torch.cuda.synchronize()
    for i, (p, pl, (u0, v0)) in enumerate(zip(probs, plans, inits)):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        pl.step(u, v, 20)
        torch.cuda.synchronize()
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i]), i
    b.close()
    for pl in plans:
        pl.close()


def test_batch_mixing_kernels_is_split_and_equals_alone(adr):
    """A batch whose plans run different mode-product kernels (a 1024 x 1024
    grid takes the CTA-pair kernel, smaller grids the one-CTA kernel) runs
    one grouped launch sequence per kernel; every solve equals its solve
    alone."""
    import torch
    probs = mixed_problems(d=2, count=3) + [wl.fhn_1024(precision=wl.BF16X3, nsteps=20)]
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    b = adr.Batch(plans)
    assert b.grouped
    b.step(us, vs, 20)
    st = b.stats()
    assert st["device_error"] == 0
    torch.cuda.synchronize()
    for i, (pl, (u0, v0)) in enumerate(zip(plans, inits)):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        pl.step(u, v, 20)
        torch.cuda.synchronize()
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i]), i
    b.close()
    for pl in plans:
        pl.close()


def test_plans_of_a_live_batch_are_protected(adr):
    """While a batch uses a plan, destroying the plan or changing its kernel
    is refused (ADR_EBUSY) and leaves both usable; after the batch is
    destroyed both succeed."""
    import torch
    probs = mixed_problems(d=2, count=2)
    plans = [adr.Plan(p) for p in probs]
    us, vs, _ = states(adr, probs)
    b = adr.Batch(plans)
    b2 = adr.Batch(plans[:1])  # a second batch over the first plan
    for pl in plans:
        with pytest.raises(adr.AdrError) as ei:
            pl.close()
        assert ei.value.status == adr.ADR_EBUSY
        with pytest.raises(adr.AdrError) as ei:
            pl.set_kernel(2)
        assert ei.value.status == adr.ADR_EBUSY
    b.step(us, vs, 3)  # still steps: nothing was freed or changed
    b.close()
    with pytest.raises(adr.AdrError):
        plans[0].close()  # b2 still holds it
    plans[1].set_kernel(2)
    plans[1].close()
    b2.close()
    plans[0].set_kernel(2)
    plans[0].close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("d", [2, 3])
def test_mixed_horizons_in_one_call_equal_alone(adr, d):
    """adr_batch_step with a horizon per solve (0, 3, 17, 40, ...): solves
    that finish drop out of the grouped work of the rest; each result equals
    the same solve stepped alone for its own horizon (bitwise), and a solve
    with horizon 0 is untouched."""
    import torch
    probs = mixed_problems(d=d, count=6)
    horizons = [40, 3, 17, 0, 40, 33]
    plans = [adr.Plan(p) for p in probs]
    us, vs, inits = states(adr, probs)
    with adr.Batch(plans) as b:
        assert b.grouped
        b.step(us, vs, horizons)
    torch.cuda.synchronize()
    for i, (p, (u0, v0)) in enumerate(zip(probs, inits)):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        with adr.Plan(p) as one:
            one.step(u, v, horizons[i])
        torch.cuda.synchronize()
        assert torch.equal(u, us[i]) and torch.equal(v, vs[i]), i
    assert torch.equal(us[3], torch.tensor(inits[3][0], dtype=torch.float32, device="cuda"))
    for pl in plans:
        pl.close()


def test_equal_operators_share_one_matrix_set(adr):
    """Plans whose directional operators and step coincide take the FP64
    matrix functions (and their split pieces) from the library's cache
    instead of computing them again; the shared plan still steps exactly like
    the first."""
    import torch
    # a step no other test uses, so that no live plan holds these sets
    p = wl.fhn_1024(precision=wl.BF16X3, n=192, nsteps=10).replace(tau=0.0123456789)
    a = adr.Plan(p)
    # FHN on a square grid: each component's operator is the same in both
    # directions, so a plan holds two distinct sets (u's, v's)
    assert a.stats()["shared_matrices"] == 0
    b = adr.Plan(p)
    assert b.stats()["shared_matrices"] == 2  # both found in the cache
    for w in range(4):
        for c in range(2):
            for mu in range(2):
                assert np.array_equal(a.matrix(w, c, mu), b.matrix(w, c, mu))
    u0, v0 = wl.initial_data(p)
    outs = []
    for pl in (a, b):
        u = torch.tensor(u0, dtype=torch.float32, device="cuda")
        v = torch.tensor(v0, dtype=torch.float32, device="cuda")
        pl.step(u, v, p.nsteps)
        torch.cuda.synchronize()
        outs.append((u.cpu(), v.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    a.close()
    # the set outlives the first plan while the second holds it
    c = adr.Plan(p)
    assert c.stats()["shared_matrices"] == 2
    b.close()
    c.close()
    # a different step is another operator function: nothing shared
    d = adr.Plan(p.replace(tau=p.tau * 0.5))
    assert d.stats()["shared_matrices"] == 0
    d.close()
