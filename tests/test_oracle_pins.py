"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, a library routine for a special case, an independent route, brute
force on tiny inputs, invariants, or numbers printed in the paper.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as wl
from oracle import fd, matfun, metrics, models, schemes, tensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ FD matrices
@pytest.mark.parametrize("n,delta,alpha", [(5, 1.0, 0.0), (17, 0.02, -0.5), (64, 20.0, 0.5)])
def test_fd_rows_sum_to_zero(n, delta, alpha):
    """Neumann rows: constants are in the kernel (K const = 0)."""
    A = fd.fd_matrix(n, 0.0, 1.0 if n < 60 else 100.0, delta, alpha)
    assert np.max(np.abs(A.sum(axis=1))) <= 1e-9 * np.max(np.abs(A))


def test_fd_mass_conservation_without_advection():
    """For alpha = 0, w^T A = 0 with trapezoid weights (discrete mass)."""
    A = fd.fd_matrix(33, 0.0, 2.0, 0.7, 0.0)
    w = metrics.trapezoid_weights(33)
    assert np.max(np.abs(w @ A)) <= 1e-12 * np.max(np.abs(A))


def test_fd_tridiagonal_stencil_values():
    """Interior row = centred second and first differences (Sec. 4 text)."""
    n, L, delta, alpha = 11, 2.0, 0.3, 0.4
    h = L / (n - 1)
    A = fd.fd_matrix(n, 0.0, L, delta, alpha)
    i = 5
    assert A[i, i - 1] == pytest.approx(delta / h**2 + alpha / (2 * h), rel=1e-15)
    assert A[i, i] == pytest.approx(-2 * delta / h**2, rel=1e-15)
    assert A[i, i + 1] == pytest.approx(delta / h**2 - alpha / (2 * h), rel=1e-15)
    assert np.count_nonzero(np.triu(A, 2)) == 0 and np.count_nonzero(np.tril(A, -2)) == 0


def test_fd_second_order_consistency():
    """(A f)(x_i) -> delta f'' - alpha f' with O(h^2) error for a function with
    zero normal derivative at both ends (the Neumann condition)."""
    L, delta, alpha = 3.0, 0.8, 0.6
    errs = []
    for n in (41, 81, 161):
        x = fd.grid(n, 0.0, L)
        f = np.cos(math.pi * x / L)
        exact = -delta * (math.pi / L) ** 2 * f + alpha * (math.pi / L) * np.sin(math.pi * x / L)
        A = fd.fd_matrix(n, 0.0, L, delta, alpha)
        errs.append(np.max(np.abs(A @ f - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


# ------------------------------------------------------------------ Pade / matrix functions
def test_pade13_matches_taylor_to_order_26():
    """The [13/13] approximant p(x)/p(-x) agrees with e^x through x^26 (the
    defining property of the diagonal Pade approximant), in exact arithmetic."""
    b = matfun.pade13_coefficients()
    assert b[13] == 1
    q = [c * (-1) ** j for j, c in enumerate(b)]
    # Taylor coefficients of p/q by power-series division
    N = 27
    p_ext = b + [Fraction(0)] * (N - len(b))
    q_ext = q + [Fraction(0)] * (N - len(q))
    r = []
    for k in range(N):
        s = p_ext[k] - sum(q_ext[j] * r[k - j] for j in range(1, k + 1))
        r.append(s / q_ext[0])
    for k in range(N):
        assert r[k] == Fraction(1, math.factorial(k)), k
    # and not through x^27 (order exactly 2m)
    s = Fraction(0) - sum(q_ext[j] * r[27 - j] for j in range(1, 14) if 27 - j < N)
    assert s / q_ext[0] != Fraction(1, math.factorial(27))


@pytest.mark.parametrize("scale", [0.1, 3.0, 40.0, 900.0])
def test_expm_matches_scipy(scale):
    """Library routine on random matrices, with and without squaring."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((24, 24)) * scale / 24**0.5
    if scale > 100:
        X = -X @ X.T / scale  # keep e^X finite: negative semidefinite
    E = matfun.expm_pade13(X)
    R = sl.expm(X)
    assert np.max(np.abs(E - R)) <= 1e-12 * max(1.0, np.max(np.abs(R)))


@pytest.mark.parametrize("x", [-800.0, -50.0, -3.0, -1e-3, 0.0, 1e-6, 0.5, 2.0])
def test_phi_scalar_closed_forms(x):
    """n = 1: e^x, (e^x - 1)/x, (e^x - 1 - x)/x^2 (Eq. 9 integrated)."""
    E, P1, P2 = matfun.phi_augmented(np.array([[x]]))
    if x == 0.0:
        e0, e1, e2 = 1.0, 1.0, 0.5
    else:
        e0 = math.exp(x)
        e1 = math.expm1(x) / x
        # series where the closed form cancels
        e2 = (math.expm1(x) - x) / x**2 if abs(x) > 0.1 else sum(x**k / math.factorial(k + 2) for k in range(20))
    assert E[0, 0] == pytest.approx(e0, rel=1e-13, abs=1e-300)
    assert P1[0, 0] == pytest.approx(e1, rel=1e-13)
    assert P2[0, 0] == pytest.approx(e2, rel=1e-13)


def test_phi_at_zero_matrix():
    E, P1, P2 = matfun.phi_augmented(np.zeros((6, 6)))
    I = np.eye(6)
    for M, ref in ((E, I), (P1, I), (P2, 0.5 * I)):
        assert np.max(np.abs(M - ref)) <= 4e-16


@pytest.mark.parametrize("n,L,delta,alpha,tau", [(40, 1.0, 1.0, 0.0, 5e-4),
                                                 (48, 100.0, 20.0, 0.5, 1e-2),
                                                 (32, 1.0, 0.02, -0.1, 1e-2)])
def test_phi_identities_and_eigen_route(n, L, delta, alpha, tau):
    """X phi_1 = e^X - I, X phi_2 = phi_1 - I, and agreement with the
    independent symmetrise-and-diagonalise route."""
    X = tau * fd.fd_matrix(n, 0.0, L, delta, alpha)
    E, P1, P2 = matfun.phi_augmented(X)
    I = np.eye(n)
    assert np.max(np.abs(X @ P1 - (E - I))) <= 1e-13
    assert np.max(np.abs(X @ P2 - (P1 - I))) <= 1e-13
    E2, Q1, Q2 = matfun.phi_eigen(X)
    for a, b in ((E, E2), (P1, Q1), (P2, Q2)):
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


def test_phi_against_quadrature_of_definition():
    """Eq. (9) integrated by 40-point Gauss-Legendre with e^{(1-theta)X} from
    a library expm."""
    X = 0.01 * fd.fd_matrix(20, 0.0, 1.0, 1.0, 0.3) * 0.2
    th, wq = np.polynomial.legendre.leggauss(40)
    th = 0.5 * (th + 1.0)
    wq = 0.5 * wq
    Q1 = sum(w * sl.expm((1 - t) * X) for t, w in zip(th, wq))
    Q2 = sum(w * t * sl.expm((1 - t) * X) for t, w in zip(th, wq))
    _, P1, P2 = matfun.phi_augmented(X)
    assert np.max(np.abs(P1 - Q1)) <= 1e-13
    assert np.max(np.abs(P2 - Q2)) <= 1e-13


def test_phi_row_sums_follow_kernel():
    """w^T A = 0 implies w^T phi_ell(tau A) = w^T / ell! (series form)."""
    A = fd.fd_matrix(30, 0.0, 1.0, 1.0, 0.0)
    w = metrics.trapezoid_weights(30)
    E, P1, P2 = matfun.phi_augmented(1e-3 * A)
    assert np.max(np.abs(w @ E - w)) < 1e-13
    assert np.max(np.abs(w @ P1 - w)) < 1e-13
    assert np.max(np.abs(w @ P2 - 0.5 * w)) < 1e-13


# ------------------------------------------------------------------ tensor operations
def _brute_mode_product(W, M, mu):
    d = W.ndim
    axis = d - mu
    out = np.zeros(W.shape[:axis] + (M.shape[0],) + W.shape[axis + 1:])
    for idx in np.ndindex(*out.shape):
        i = idx[axis]
        s = 0.0
        for j in range(W.shape[axis]):
            src = idx[:axis] + (j,) + idx[axis + 1:]
            s += M[i, j] * W[src]
        out[idx] = s
    return out


@pytest.mark.parametrize("shape", [(3, 4), (5, 3, 4)])
def test_mode_product_brute_force(shape):
    rng = np.random.default_rng(3)
    W = rng.standard_normal(shape)
    d = len(shape)
    for mu in range(1, d + 1):
        n = shape[d - mu]
        M = rng.standard_normal((n + 1, n))  # rectangular: catches transposes
        assert np.allclose(tensor.mode_product(W, M, mu), _brute_mode_product(W, M, mu),
                           rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("shape", [(5, 7), (3, 4, 5)])
def test_tucker_equals_kronecker(shape):
    """Eq. (5): vec(W x_1 M_1 ... x_d M_d) = (M_d kron ... kron M_1) vec(W)."""
    rng = np.random.default_rng(5)
    W = rng.standard_normal(shape)
    d = len(shape)
    Ms = [rng.standard_normal((shape[d - 1 - m], shape[d - 1 - m])) for m in range(d)]
    lhs = tensor.tucker(W, Ms).ravel()
    rhs = tensor.kron_dense(Ms) @ W.ravel()
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("shape", [(6, 9), (4, 5, 6)])
def test_tucker_of_exponentials_is_exp_of_kron_sum(shape):
    """e^{tau K} w = vec(W x_mu e^{tau A_mu}) exactly (Eq. 5), against a
    library expm of the assembled N x N Kronecker sum (Eq. 3)."""
    rng = np.random.default_rng(9)
    d = len(shape)
    As = [fd.fd_matrix(shape[d - 1 - m], 0.0, 1.0, 0.5 + 0.1 * m, 0.3) for m in range(d)]
    tau = 2e-3
    W = rng.standard_normal(shape)
    Es = [matfun.phi_augmented(tau * A)[0] for A in As]
    K = tensor.kron_sum_dense(As)
    ref = sl.expm(tau * K) @ W.ravel()
    got = tensor.tucker(W, Es).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # and the Kronecker-sum action matches K vec(W)
    assert np.allclose(tensor.kron_sum_action(W, As).ravel(), K @ W.ravel(), rtol=1e-13, atol=1e-9)


# ------------------------------------------------------------------ ETD2RKds
def _tiny(model, shape=(5, 6), d=2, adv=0.2, seed=1):
    n = tuple(reversed(shape))
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.3, 1.1),
                   adv=((adv,) * d, (-adv,) * d), model=model,
                   params={0: (50.0, 0.1, 0.9), 1: (0.05, 2.0, -0.03), 2: (1.0, 3.0),
                           3: ()}[model],
                   tau=3e-3, nsteps=1, seed=seed)
    return p


@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(5, 6), (3, 4, 5)])
def test_step_equals_dense_kronecker_form(model, shape):
    """Eq. (11) with the Tucker operators replaced by explicit Kronecker
    products and K by the assembled Kronecker sum."""
    p = _tiny(model, shape, d=len(shape))
    plan = schemes.make_plan(p)
    U, V = wl.initial_data(p, kind="uniform", amp=0.1)
    a = schemes.etd2rkds_step(plan, U, V)
    b = schemes.etd2rkds_step_dense_form(plan, U, V)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-13 * np.max(np.abs(y))


def test_step_reduces_to_exponential_in_one_direction():
    """With n_2 = 1 (A_2 = [0]) and g = 0 the split step is exact:
    U + tau phi_1(tau A_1) A_1 U = e^{tau A_1} U."""
    A1 = fd.fd_matrix(12, 0.0, 1.0, 1.0, 0.4)
    Z = np.zeros((1, 1))
    plan = schemes.make_plan_from_matrices([A1, Z], [A1, Z], 0.01, models.NO_REACTION, ())
    rng = np.random.default_rng(2)
    U = rng.standard_normal((1, 12))
    Un, _ = schemes.etd2rkds_step(plan, U, U)
    ref = sl.expm(0.01 * A1) @ U[0]
    assert np.max(np.abs(Un[0] - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_one_step_splitting_error_is_third_order():
    """At g = 0 the split step differs from e^{tau K} by O(tau^3) per step
    (Eq. 10a embedded in a first-stage update)."""
    shape = (7, 8)
    As = [fd.fd_matrix(8, 0.0, 1.0, 1.0, 0.3), fd.fd_matrix(7, 0.0, 1.0, 0.6, -0.2)]
    K = tensor.kron_sum_dense(As)
    rng = np.random.default_rng(4)
    U = rng.standard_normal(shape)
    diffs = []
    for tau in (1e-3, 5e-4, 2.5e-4):
        plan = schemes.make_plan_from_matrices(As, As, tau, models.NO_REACTION, ())
        Un, _ = schemes.etd2rkds_step(plan, U, U)
        diffs.append(np.linalg.norm(Un.ravel() - sl.expm(tau * K) @ U.ravel()))
    s1 = math.log2(diffs[0] / diffs[1])
    s2 = math.log2(diffs[1] / diffs[2])
    assert 2.8 < s1 < 3.2 and 2.8 < s2 < 3.2


def test_dib_derived_parameter_gives_the_equilibrium():
    """Sec. 4.4: a4v is chosen so that (0, a4u) is an equilibrium of Eq. 15."""
    prm = wl.dib_parameters()
    gu, gv = models.reaction(models.DIB, prm, np.array([0.0]), np.array([prm[4]]))
    assert abs(gu[0]) < 1e-13 and abs(gv[0]) < 1e-12
    # and the other terms do not vanish there on their own
    assert abs(prm[5] * (1 - prm[4]) * (1 - prm[7] * (1 - prm[4]))) > 1.0


def test_fhn_rho_is_the_fhn_family():
    """Eq. 13 with rho = 1 is the FHN variant with eps = a1, a1' = a2, a0 = 0."""
    rng = np.random.default_rng(8)
    U, V = rng.standard_normal(50), rng.standard_normal(50)
    a = models.reaction(models.FHN_RHO, (1.0, 11.0, 0.1), U, V)
    b = models.reaction(models.FHN, (11.0, 0.1, 0.0), U, V)
    assert np.allclose(a[0], b[0], rtol=1e-15) and np.allclose(a[1], b[1], rtol=1e-15)
    c = models.reaction(models.FHN_RHO, (65.731, 11.0, 0.1), U, V)
    assert np.allclose(c[0], 65.731 * a[0], rtol=1e-14)


@pytest.mark.parametrize("model,params", [(0, (1000.0, 0.1, 0.9)), (1, (0.05, 2.0, -0.03)),
                                          (2, (1.0, 3.0)), (4, (65.731, 11.0, 0.1)),
                                          (5, wl.dib_parameters())])
def test_equilibria_preserved(model, params):
    """Spatially constant steady states stay put over 100 steps."""
    p = wl.Problem(d=2, n=(16, 12), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, 10.0),
                   adv=((0.3, 0.1), (0.2, -0.4)), model=model, params=params,
                   tau=1e-3, nsteps=100)
    ue, ve = wl.equilibrium(model, params)
    # the equilibrium really is one
    gu, gv = models.reaction(model, params, np.array(ue), np.array(ve))
    assert abs(gu) < 1e-13 and abs(gv) < 1e-13
    plan = schemes.make_plan(p)
    U = np.full(p.shape, ue)
    V = np.full(p.shape, ve)
    U, V = schemes.etd2rkds_solve(plan, U, V, 100)
    # rounding only: K const is a sum of O(delta/h^2) terms cancelling to zero
    assert np.max(np.abs(U - ue)) <= 1e-12 * max(1.0, abs(ue))
    assert np.max(np.abs(V - ve)) <= 1e-12 * max(1.0, abs(ve))


@pytest.mark.parametrize("d", [2, 3])
def test_mass_conserved_without_advection_or_reaction(d):
    """alpha = 0, g = 0: the trapezoid-weighted sum is invariant, since
    w^T A_mu = 0 gives (w kron .. kron w)^T K = 0."""
    n = (9, 7, 5)[:d]
    p = wl.Problem(d=d, n=n, lo=(0.0,) * d, hi=(1.0,) * d, diff=(0.7, 2.0),
                   adv=((0.0,) * d, (0.0,) * d), model=models.NO_REACTION, params=(),
                   tau=5e-3, nsteps=1, seed=3)
    plan = schemes.make_plan(p)
    U, V = wl.initial_data(p, kind="uniform", amp=0.5)
    m0 = metrics.spatial_mean(U)
    U1, _ = schemes.etd2rkds_solve(plan, U, V, 20)
    assert abs(metrics.spatial_mean(U1) - m0) <= 1e-14


def _brusselator_e6(n, nsteps):
    v = (0.1, 0.1, 0.1)
    # Sec. 4.6: delta^u = 0.01, delta^v = 0.02, alpha = 0.1, a_1 = 1, a_2 = 2,
    # so g^u = a_2 - (a_1 + 1) u + u^2 v, g^v = a_1 u - u^2 v  (a = 2, b = 1)
    return wl.Problem(d=3, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3, diff=(0.01, 0.02),
                      adv=(v, v), model=wl.BRUSSELATOR, params=(2.0, 1.0),
                      tau=1.0 / nsteps, nsteps=nsteps)


def test_order_two_on_brusselator():
    """Observed order in [1.9, 2.2] under step halving against a 16x finer
    run (paper: 2.05-2.13, Sec. 4.6)."""
    n = 12
    ref_steps = 16 * 200
    p = _brusselator_e6(n, ref_steps)
    U0, V0 = wl.brusselator_e6_initial(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p, tau=1.0 / ref_steps), U0, V0, ref_steps)
    errs = []
    for m in (50, 100, 200):
        U, V = schemes.etd2rkds_solve(schemes.make_plan(p, tau=1.0 / m), U0, V0, m)
        errs.append(metrics.paper_rel_err(U, V, Ur, Vr))
    o1, o2 = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert 1.9 <= o1 <= 2.2 and 1.9 <= o2 <= 2.2, (errs, o1, o2)


def _lawson_orders(step):
    n = 12
    ref_steps = 16 * 200
    p = _brusselator_e6(n, ref_steps)
    U0, V0 = wl.brusselator_e6_initial(p)

    def solve(m):
        plan = schemes.make_plan(p, tau=1.0 / m)
        U, V = U0, V0
        for _ in range(m):
            U, V = step(plan, U, V)
        return U, V

    Ur, Vr = solve(ref_steps)
    errs = [metrics.paper_rel_err(*solve(m), Ur, Vr) for m in (50, 100, 200)]
    return errs, math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])


def test_lawson2b_order_two_on_brusselator():
    """Lawson2b (Eq. 7) converges with order 2 under step halving against a
    16x finer Lawson2b run on the Sec. 4.6 Brusselator."""
    errs, o1, o2 = _lawson_orders(schemes.lawson2b_step)
    assert 1.8 <= o1 <= 2.3 and 1.8 <= o2 <= 2.3, (errs, o1, o2)


def test_lawson2b_without_final_reaction_is_first_order():
    """Planted mistake: dropping the last stage's tau/2 G(U2, V2) term of
    Eq. 7 makes the scheme inconsistent at order 2 (observed order about 1),
    so the order pin above would catch it."""
    from oracle.models import reaction
    from oracle.tensor import tucker

    def broken(plan, U, V):
        tau = plan.tau
        GU, GV = reaction(plan.model, plan.params, U, V)
        return (tucker(U + 0.5 * tau * GU, plan.E[0]), tucker(V + 0.5 * tau * GV, plan.E[1]))

    errs, o1, o2 = _lawson_orders(broken)
    assert o1 < 1.5 and o2 < 1.5, (errs, o1, o2)


def test_split_and_unsplit_etd2rk_errors_comparable():
    """On a tiny grid the split scheme's global error is within a small
    factor of unsplit ETD2RK's (Eq. 8 with dense phi(tau K)); the paper's
    tables show ratios near 1 (Sec. 4.1, 4.6)."""
    p = wl.Problem(d=2, n=(10, 9), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(0.05, 0.1),
                   adv=((0.2, 0.1), (0.2, 0.1)), model=wl.BRUSSELATOR, params=(1.0, 2.0),
                   tau=0.05, nsteps=20, seed=4)
    U0, V0 = wl.initial_data(p, kind="uniform", amp=0.3)
    fine = schemes.make_plan(p, tau=1.0 / 640)
    dfine = schemes.make_dense_plan(fine, p.shape)
    Ur, Vr = U0, V0
    for _ in range(640):
        Ur, Vr = schemes.etd2rk_dense_step(dfine, Ur, Vr)
    plan = schemes.make_plan(p)
    dplan = schemes.make_dense_plan(plan, p.shape)
    Us, Vs = schemes.etd2rkds_solve(plan, U0, V0, 20)
    Ud, Vd = U0, V0
    for _ in range(20):
        Ud, Vd = schemes.etd2rk_dense_step(dplan, Ud, Vd)
    es = metrics.paper_rel_err(Us, Vs, Ur, Vr)
    ed = metrics.paper_rel_err(Ud, Vd, Ur, Vr)
    assert es < 5e-3 and ed < 5e-3
    assert 0.2 < es / ed < 5.0, (es, ed)


def test_wrong_stage_two_factor_breaks_order(monkeypatch):
    """Planting factor 1 instead of 2^(d-1) in the oracle must break order 2,
    so the order pin above really checks that factor."""
    orig = schemes.etd2rkds_step

    def planted(plan, U, V):
        tau = plan.tau
        GU, GV = models.reaction(plan.model, plan.params, U, V)
        WU = tensor.kron_sum_action(U, plan.A[0]) + GU
        WV = tensor.kron_sum_action(V, plan.A[1]) + GV
        U2 = U + tau * tensor.tucker(WU, plan.phi1[0])
        V2 = V + tau * tensor.tucker(WV, plan.phi1[1])
        GU2, GV2 = models.reaction(plan.model, plan.params, U2, V2)
        return (U2 + tau * tensor.tucker(GU2 - GU, plan.phi2[0]),
                V2 + tau * tensor.tucker(GV2 - GV, plan.phi2[1]))

    monkeypatch.setattr(schemes, "etd2rkds_step", planted)
    with pytest.raises(AssertionError):
        test_order_two_on_brusselator()
    monkeypatch.setattr(schemes, "etd2rkds_step", orig)


def test_paper_brusselator_error_magnitudes():
    """Pin against Table 'bruss' (Sec. 4.6): ETD2RKds errors at 50..200 steps
    against a 1600-step run.  The errors are time-discretisation errors and
    depend only weakly on the grid, so a 24^3 grid reproduces the paper's
    64^3 numbers to within a few percent; 15% is allowed for the unstated
    reference step count and grid."""
    rows = np.loadtxt(os.path.join(GOLDEN, "brusselator_e6_table.txt"))
    n = 24
    ref_steps = 1600
    p = _brusselator_e6(n, ref_steps)
    U0, V0 = wl.brusselator_e6_initial(p)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p, tau=1.0 / ref_steps), U0, V0, ref_steps)
    for steps, err_paper, _ in rows:
        m = int(steps)
        U, V = schemes.etd2rkds_solve(schemes.make_plan(p, tau=1.0 / m), U0, V0, m)
        e = metrics.paper_rel_err(U, V, Ur, Vr)
        assert abs(e / err_paper - 1.0) < 0.15, (m, e, err_paper)


# ------------------------------------------------------------------ metrics / inputs
def test_metrics_definitions():
    R = np.array([[1.0, -2.0], [0.5, 4.0]])
    X = R + np.array([[0.0, 0.1], [0.0, 0.0]])
    assert metrics.max_rel_err(X, R, R, R) == pytest.approx(0.1 / 4.0)
    assert metrics.paper_rel_err(X, R, R, R) == pytest.approx(0.1 / np.linalg.norm(R))
    # trapezoid mean of a linear function = its midpoint value
    x = fd.grid(11, 0.0, 1.0)
    assert metrics.spatial_mean(np.add.outer(x, 2 * x)) == pytest.approx(1.5, rel=1e-14)


def test_splitmix64_published_vector():
    """First outputs of SplitMix64 from seed 0 (Vigna's reference code)."""
    z = wl.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = wl.uniform01(7, 100000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    g = wl.normal(7, 100000)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02
