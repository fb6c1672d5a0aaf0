"""General plans (adr_plan_create_general): m = 1..4 components, dense
directional matrices, polynomial reactions, against the general oracle
(oracle/general.py), whose own pins are in test_oracle_general_pins.py.

Tolerances: FP64 products 1e-11 (rounding of the dense products over a few
steps), FP32 products 1e-5 (the single-precision bound of the other paths).
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import general, schemes

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


def _rand_dense(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return scale * (-(B @ B.T / n + np.eye(n)) + 0.3 * (B - B.T) / math.sqrt(n))


THREE = [(0, (0, 1, 1), 1.0), (0, (1, 0, 0), -1.0), (1, (1, 0, 0), 0.7), (1, (0, 2, 0), -0.5),
         (2, (0, 0, 0), 0.3), (2, (1, 1, 0), 0.4), (2, (0, 0, 1), -1.2)]


def _gpu(adr, A, terms, tau, Us, nsteps, precision):
    import torch
    dt = torch.float64 if precision == wl.FP64 else torch.float32
    xs = [torch.tensor(U, dtype=dt, device="cuda") for U in Us]
    with adr.GeneralPlan(A, terms, tau, precision=precision) as gp:
        gp.step(xs, nsteps)
        torch.cuda.synchronize()
        mats = gp.matrix(2, 0, 0), gp.matrix(3, len(Us) - 1, len(A[0]) - 1)
    return [x.double().cpu().numpy() for x in xs], mats


def _max_rel(Xs, Rs):
    return max(np.max(np.abs(X - R)) / np.max(np.abs(R)) for X, R in zip(Xs, Rs))


@pytest.mark.parametrize("n", [(24, 40), (16, 24, 8), (130, 72)])
@pytest.mark.parametrize("precision,tol", [(wl.FP64, 1e-11), (wl.FP32, 1e-5)])
def test_three_components_dense_matrices_match_oracle(adr, n, precision, tol):
    d = len(n)
    A = [[_rand_dense(n[mu], 10 * c + mu, scale=3.0) for mu in range(d)] for c in range(3)]
    tau, nsteps = 1e-2, 6
    shape = tuple(reversed(n))
    rng = np.random.default_rng(4)
    Us = [1.0 + 0.2 * rng.standard_normal(shape) for _ in range(3)]
    if precision == wl.FP32:
        Us = [U.astype(np.float32).astype(np.float64) for U in Us]
    gp = general.make_general_plan(A, tau, THREE)
    ref = general.etd2rkds_solve_general(gp, Us, nsteps)
    got, (p1, p2) = _gpu(adr, A, THREE, tau, Us, nsteps, precision)
    assert _max_rel(got, ref) <= tol, _max_rel(got, ref)
    # the plan's FP64 matrix functions of dense matrices match the oracle's
    assert np.max(np.abs(p1 - gp.phi1[0][0])) <= 1e-12 * np.max(np.abs(gp.phi1[0][0]))
    assert np.max(np.abs(p2 - gp.phi2[2][d - 1])) <= 1e-12 * np.max(np.abs(gp.phi2[2][d - 1]))


def test_two_components_through_the_general_path_equal_the_fd_plan(adr):
    """The FD Brusselator as a general plan (A_mu from the oracle's FD
    matrices, the reaction as monomials) agrees with the oracle and with the
    finite-difference FP64 plan to rounding."""
    import torch
    from oracle import fd
    p = wl.Problem(d=2, n=(48, 40), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(0.02, 0.1),
                   adv=((-0.3, 0.2), (0.1, -0.2)), model=wl.BRUSSELATOR, params=(1.0, 3.0),
                   tau=1e-2, nsteps=10, seed=9, precision=wl.FP64)
    A = [fd.direction_matrices(p, 0), fd.direction_matrices(p, 1)]
    U0, V0 = wl.initial_data(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), U0, V0, p.nsteps)
    got, _ = _gpu(adr, A, general.brusselator_terms(1.0, 3.0), p.tau, [U0, V0], p.nsteps, wl.FP64)
    assert _max_rel(got, [Ur, Vr]) <= 1e-11
    u = torch.tensor(U0, dtype=torch.float64, device="cuda")
    v = torch.tensor(V0, dtype=torch.float64, device="cuda")
    with adr.Plan(p) as plan:
        plan.step(u, v, p.nsteps)
    torch.cuda.synchronize()
    assert _max_rel(got, [u.cpu().numpy(), v.cpu().numpy()]) <= 1e-11


@pytest.mark.parametrize("m", [1, 4])
def test_one_and_four_components(adr, m):
    """m = 1 (a Fisher-KPP-type logistic reaction u - u^2) and m = 4 (a
    cyclic coupling with one quadratic term per component), 3D."""
    n = (16, 8, 24)
    d = 3
    A = [[_rand_dense(n[mu], 5 * c + mu, scale=2.0) for mu in range(d)] for c in range(m)]
    if m == 1:
        terms = [(0, (1,), 1.0), (0, (2,), -1.0)]
    else:
        terms = []
        for c in range(4):
            e = [0, 0, 0, 0]
            e[(c + 1) % 4] = 1
            terms.append((c, tuple(e), 0.5))
            e2 = [0, 0, 0, 0]
            e2[c] = 2
            terms.append((c, tuple(e2), -0.3))
    tau, nsteps = 2e-2, 5
    rng = np.random.default_rng(m)
    Us = [0.5 + 0.1 * rng.standard_normal(tuple(reversed(n))) for _ in range(m)]
    gp = general.make_general_plan(A, tau, terms)
    ref = general.etd2rkds_solve_general(gp, Us, nsteps)
    got, _ = _gpu(adr, A, terms, tau, Us, nsteps, wl.FP64)
    assert _max_rel(got, ref) <= 1e-11


def test_general_plans_reject_bad_input_and_the_fd_entry_points(adr):
    import ctypes
    import torch
    A = [[_rand_dense(8, 1), _rand_dense(8, 2)]]
    with pytest.raises(adr.AdrError):
        adr.GeneralPlan(A, [(1, (1,), 1.0)], 1e-2)   # term of a component that does not exist
    with pytest.raises(adr.AdrError):
        adr.GeneralPlan(A, [], 1e-2, precision=wl.BF16X3)  # FP64 / FP32 only
    with adr.GeneralPlan(A, [(0, (1,), -1.0)], 1e-2) as gp:
        u = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
        v = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
        st = adr.lib().adr_step(gp._p, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), 1)
        assert st == adr.ADR_EINVAL
