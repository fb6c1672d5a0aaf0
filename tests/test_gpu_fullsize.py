"""The full-length workloads on the GPU against the FP64 oracle's own solve
(not against an FP64 GPU solve): FitzHugh-Nagumo 1024^2 for 500 steps,
Brusselator 256^3 for 100 steps, and a deterministic sample of the batch of
512 solves at 100 steps.  Bound: max relative error <= 1e-5 (per component
||X - X_ref||_inf / ||X_ref||_inf, maximum over u and v).

The oracle's solves take tens of seconds to a few minutes on the host cores;
they run in a spawned worker process while the GPU side runs.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _oracle_solve(p):
    from oracle import schemes
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    return schemes.etd2rkds_solve(schemes.make_plan(p), u0, v0, p.nsteps)


BATCH_SAMPLE = list(range(0, 512, 32))  # 16 of the 512 solves


@pytest.fixture(scope="module")
def refs():
    """Oracle solves of every full-length case, computed in a spawned worker."""
    jobs = {"fhn1024": wl.fhn_1024(precision=wl.FP64),
            "bruss256": wl.brusselator_256(precision=wl.FP64)}
    probs = wl.batched_512(precision=wl.FP64)
    for i in BATCH_SAMPLE:
        jobs[f"batch{i}"] = probs[i]
    ex = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
    futs = {k: ex.submit(_oracle_solve, p) for k, p in jobs.items()}
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def _run(adr, p, precision):
    import torch
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    dt = adr.state_dtype(precision)
    u = torch.tensor(u0, dtype=dt, device="cuda")
    v = torch.tensor(v0, dtype=dt, device="cuda")
    with adr.Plan(p.replace(precision=precision)) as plan:
        plan.step(u, v, p.nsteps)
        st = plan.stats()
    assert st["device_error"] == 0
    return u.double().cpu().numpy(), v.double().cpu().numpy()


def test_fhn_1024_500_steps_against_oracle(adr, refs):
    """The headline workload: BF16x3 split products (the plain and the
    compensated state) and the plain FP32 SIMT form, all against the oracle
    over the 500 steps; the split form is at least as accurate as plain FP32
    (within 1.5x)."""
    p = wl.fhn_1024()
    Uc, Vc = _run(adr, p.replace(state=wl.STATE_COMPENSATED), wl.BF16X3)
    Ub, Vb = _run(adr, p, wl.BF16X3)
    Uf, Vf = _run(adr, p, wl.FP32)
    Ur, Vr = refs["fhn1024"].result()
    eb = oracle.max_rel_err(Ub, Vb, Ur, Vr)
    ec = oracle.max_rel_err(Uc, Vc, Ur, Vr)
    ef = oracle.max_rel_err(Uf, Vf, Ur, Vr)
    print(f"fhn1024 500 steps: bf16x3 {eb:.3e}, bf16x3 compensated {ec:.3e}, fp32 {ef:.3e}")
    assert eb <= TOL and ec <= TOL, (eb, ec, ef)
    assert eb <= 1.5 * ef, (eb, ef)


def test_brusselator_256_100_steps_against_oracle(adr, refs):
    p = wl.brusselator_256()
    Ub, Vb = _run(adr, p, wl.BF16X3)
    Uc, Vc = _run(adr, p.replace(state=wl.STATE_COMPENSATED), wl.BF16X3)
    Ur, Vr = refs["bruss256"].result()
    eb = oracle.max_rel_err(Ub, Vb, Ur, Vr)
    ec = oracle.max_rel_err(Uc, Vc, Ur, Vr)
    print(f"bruss256 100 steps: bf16x3 {eb:.3e}, bf16x3 compensated {ec:.3e}")
    assert eb <= TOL and ec <= TOL, (eb, ec)


def test_batch_512_sample_against_oracle(adr, refs):
    """The whole batch of 512 solves stepped together (grouped launches),
    every 32nd solve compared with the oracle."""
    import torch
    probs = wl.batched_512(precision=wl.BF16X3)
    plans = [adr.Plan(p) for p in probs]
    us, vs = [], []
    for p in probs:
        u0, v0 = wl.initial_data(p)
        us.append(torch.tensor(wl.round_to(u0, wl.FP32), dtype=torch.float32, device="cuda"))
        vs.append(torch.tensor(wl.round_to(v0, wl.FP32), dtype=torch.float32, device="cuda"))
    with adr.Batch(plans) as b:
        assert b.grouped
        b.step(us, vs, probs[0].nsteps)
    torch.cuda.synchronize()
    errs = {}
    for i in BATCH_SAMPLE:
        Ur, Vr = refs[f"batch{i}"].result()
        errs[i] = oracle.max_rel_err(us[i].double().cpu().numpy(), vs[i].double().cpu().numpy(),
                                     Ur, Vr)
    for pl in plans:
        pl.close()
    print("batch sample errors:", {k: f"{e:.2e}" for k, e in errs.items()})
    assert max(errs.values()) <= TOL, errs
