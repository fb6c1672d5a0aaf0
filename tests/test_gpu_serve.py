"""Continuous-batching server: requests of mixed 2D/3D grids, models and
horizons arriving over time; each result must equal the same request solved
alone (bit for bit: the same kernels on the same tiles), with admission
limited by a device-memory budget, and match the FP64 oracle within 1e-5."""
import numpy as np
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


def small_requests(count=10, seed=9):
    from paper_2307_10684_gb300.serve import Request
    r = wl.uniform01(seed, 8 * count)
    reqs = []
    t = 0.0
    for i in range(count):
        q = r[8 * i: 8 * i + 8]
        t += -np.log(1.0 - q[0]) / 400.0
        three = q[1] < 0.4
        s = (16, 24, 32)[int(q[2] * 3)] if three else (64, 96, 128)[int(q[2] * 3)]
        n = (s, s, s) if three else (s, (64, 128)[int(q[3] * 2)])
        d = len(n)
        model = int(q[4] * 3)
        if model == wl.SCHNAKENBERG:
            p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(1.0, 8.0),
                           adv=((0.0,) * d, (0.0,) * d), model=model,
                           params=(300.0 + 400 * q[5], 0.1, 0.9), tau=2e-4, nsteps=0,
                           precision=wl.BF16X3, seed=500 + i)
        elif model == wl.FHN:
            p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(100.0,) * d, diff=(1.0, 10.0),
                           adv=((0.5,) * d, (0.5,) * d), model=model, params=(0.05, 2.0, -0.03),
                           tau=1e-2, nsteps=0, precision=wl.BF16X3, seed=500 + i)
        else:
            p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.02, 0.1),
                           adv=((-0.5,) * d, (-0.5,) * d), model=model, params=(1.0, 3.0),
                           tau=1e-2, nsteps=0, precision=wl.BF16X3, seed=500 + i)
        steps = 18 + int(q[6] * 40)
        p = p.replace(nsteps=steps)

        def init(p=p):
            u0, v0 = wl.initial_data(p)
            return wl.round_to(u0, wl.FP32).astype(np.float32), wl.round_to(v0, wl.FP32).astype(np.float32)

        reqs.append(Request(i, t, p, init, steps))
    return reqs


@pytest.mark.parametrize("budget_mb", [100000, 8])
def test_served_results_equal_alone(adr, budget_mb):
    import torch
    from paper_2307_10684_gb300.serve import Server, served_problem
    reqs = small_requests()
    srv = Server(budget_bytes=budget_mb * 2**20, chunk=16, keep_results=True)
    res = srv.run(reqs)
    assert len(res) == len(reqs) and all(r.nsteps > 0 for r in res)
    assert srv.stats["ticks"] > 0 and srv.used == 0
    if budget_mb < 100:
        assert srv.stats["admission_deferred"] > 0
    for req, out in zip(reqs, res):
        u0, v0 = req.init()
        u = torch.tensor(u0, device="cuda")
        v = torch.tensor(v0, device="cuda")
        # alone: the same problem as the server plans it (compensated state
        # carried across its ticks), stepped in one call
        assert served_problem(req.problem).state == wl.STATE_COMPENSATED
        with adr.Plan(served_problem(req.problem)) as plan:
            plan.step(u, v, req.nsteps)
        torch.cuda.synchronize()
        assert torch.equal(u.cpu(), out.u) and torch.equal(v.cpu(), out.v), req.rid
        assert out.latency > 0 and out.finished >= out.admitted >= out.arrival


def test_served_results_match_oracle(adr):
    from paper_2307_10684_gb300.serve import Server
    reqs = small_requests(count=4, seed=3)
    res = Server(budget_bytes=2**34, keep_results=True).run(reqs)
    for req, out in zip(reqs, res):
        u0, v0 = req.init()
        Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(req.problem), u0.astype(np.float64),
                                        v0.astype(np.float64), req.nsteps)
        err = oracle.max_rel_err(out.u.double().numpy(), out.v.double().numpy(), Ur, Vr)
        assert err <= 1e-5, (req.rid, err)
