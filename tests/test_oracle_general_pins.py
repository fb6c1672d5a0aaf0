"""Pins of the general oracle (m components, dense A_mu, polynomial
reactions: oracle/general.py) against mathematics it does not share code
with: the two-component oracle where the settings coincide, explicit
Kronecker algebra, exact linear dynamics, the one-direction reduction to
e^(tau A), and the scheme's order 2.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import workloads as wl
from oracle import general, schemes


def _rand_dense(n, seed, zero_rows=False, scale=1.0):
    """A dense directional matrix with a negative spectrum: -(B B^T/n + I)
    plus a skew part; with zero_rows a dense generator instead (non-negative
    off-diagonal entries, rows summing to 0, spectrum in the closed left
    half plane by Gershgorin)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    if zero_rows:
        B = np.abs(B) / n
        np.fill_diagonal(B, 0.0)
        return scale * (B - np.diag(B.sum(axis=1)))
    A = -(B @ B.T / n + np.eye(n)) + 0.3 * (B - B.T) / math.sqrt(n)
    return scale * A


def test_two_components_equal_the_two_component_oracle():
    """m = 2 with the Brusselator written as monomials equals the pinned
    two-component ETD2RKds oracle (Eq. 11, Eq. 17) on FD matrices."""
    p = wl.Problem(d=2, n=(9, 7), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(0.05, 0.2),
                   adv=((0.3, -0.1), (0.2, 0.1)), model=wl.BRUSSELATOR, params=(1.0, 3.0),
                   tau=5e-3, nsteps=4, seed=2)
    plan2 = schemes.make_plan(p)
    U0, V0 = wl.initial_data(p, kind="uniform", amp=0.2)
    Ur, Vr = schemes.etd2rkds_solve(plan2, U0, V0, 4)
    gp = general.make_general_plan([plan2.A[0], plan2.A[1]], p.tau,
                                   general.brusselator_terms(1.0, 3.0))
    U, V = general.etd2rkds_solve_general(gp, [U0, V0], 4)
    assert np.max(np.abs(U - Ur)) <= 1e-13 * np.max(np.abs(Ur))
    assert np.max(np.abs(V - Vr)) <= 1e-13 * np.max(np.abs(Vr))


THREE = [(0, (0, 1, 1), 1.0), (0, (1, 0, 0), -1.0), (1, (1, 0, 0), 0.7), (1, (0, 2, 0), -0.5),
         (2, (0, 0, 0), 0.3), (2, (1, 1, 0), 0.4), (2, (0, 0, 1), -1.2)]


@pytest.mark.parametrize("shape", [(4, 5), (3, 4, 2)])
def test_three_components_equal_dense_kronecker_form(shape):
    """m = 3, random dense A_mu per component and direction: the Tucker form
    equals explicit Kronecker products (Eq. 5) and the assembled sum K."""
    d = len(shape)
    n = tuple(reversed(shape))
    A = [[_rand_dense(n[mu], 10 * c + mu, scale=4.0) for mu in range(d)] for c in range(3)]
    gp = general.make_general_plan(A, 2e-2, THREE)
    rng = np.random.default_rng(5)
    Us = [1.0 + 0.2 * rng.standard_normal(shape) for _ in range(3)]
    a = general.etd2rkds_step_general(gp, Us)
    b = general.etd2rkds_step_general_dense_form(gp, Us)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-13 * np.max(np.abs(y))


def test_linear_reaction_uniform_mode_is_heun_exactly():
    """Rows of every A_mu sum to zero, so a spatially constant state sees
    K U = 0 and one step is Heun's method on the reaction ODE; with a linear
    reaction g = M u + f (three components, written as monomials) the
    deviation from the equilibrium u* = -M^-1 f follows R(tau M)^n exactly,
    R(Z) = I + Z + Z^2 / 2."""
    M = np.array([[-1.0, 0.5, 0.2], [0.3, -2.0, 0.4], [0.1, -0.6, -0.7]])
    f = np.array([0.4, -0.2, 0.9])
    terms = [(c, (0, 0, 0), f[c]) for c in range(3)]
    for c in range(3):
        for j in range(3):
            e = [0, 0, 0]
            e[j] = 1
            terms.append((c, tuple(e), M[c, j]))
    A = [[_rand_dense(6, 3 * c + mu, zero_rows=True, scale=5.0) for mu in range(2)]
         for c in range(3)]
    tau, nsteps = 0.05, 40
    gp = general.make_general_plan(A, tau, terms)
    ue = -np.linalg.solve(M, f)
    d0 = np.array([1e-3, -2e-3, 1.5e-3])
    Us = [np.full((6, 6), ue[c] + d0[c]) for c in range(3)]
    Us = general.etd2rkds_solve_general(gp, Us, nsteps)
    dn = np.array([U.mean() - ue[c] for c, U in enumerate(Us)])
    R = np.eye(3) + tau * M + (tau * M) @ (tau * M) / 2.0
    pred = np.linalg.matrix_power(R, nsteps) @ d0
    assert max(np.ptp(U) for U in Us) <= 1e-12
    assert np.linalg.norm(dn - pred) <= 1e-11 * np.linalg.norm(pred)


def test_one_direction_reduces_to_the_exponential():
    """n_2 = 1 (A_2 = [0]) and no reaction: U+ = e^(tau A_1) U for every
    component, with dense non-normal A_1."""
    A = [[_rand_dense(9, 40 + c, scale=3.0), np.zeros((1, 1))] for c in range(3)]
    tau = 0.03
    gp = general.make_general_plan(A, tau, [])
    rng = np.random.default_rng(8)
    Us = [rng.standard_normal((1, 9)) for _ in range(3)]
    out = general.etd2rkds_step_general(gp, Us)
    for c in range(3):
        ref = sl.expm(tau * A[c][0]) @ Us[c][0]
        assert np.max(np.abs(out[c][0] - ref)) <= 1e-13 * np.max(np.abs(ref))


def _order_errors(step):
    A = [[_rand_dense(8, 7 * c + mu, scale=2.0) for mu in range(2)] for c in range(3)]
    rng = np.random.default_rng(3)
    U0 = [1.0 + 0.3 * rng.standard_normal((8, 8)) for _ in range(3)]
    T = 1.0

    def solve(m):
        gp = general.make_general_plan(A, T / m, THREE)
        Us = U0
        for _ in range(m):
            Us = step(gp, Us)
        return Us

    ref = solve(16 * 64)
    errs = []
    for m in (16, 32, 64):
        Us = solve(m)
        errs.append(max(np.linalg.norm(U - R) / np.linalg.norm(R) for U, R in zip(Us, ref)))
    return errs, math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])


def test_three_component_order_two():
    errs, o1, o2 = _order_errors(general.etd2rkds_step_general)
    assert 1.8 <= o1 <= 2.3 and 1.8 <= o2 <= 2.3, (errs, o1, o2)


def test_wrong_stage_two_factor_breaks_the_order_pin():
    """Planted mistake: factor 1 instead of 2^(d-1) in stage 2."""
    from oracle.tensor import kron_sum_action, tucker

    def planted(gp, Us):
        G = general.poly_reaction(gp.terms, Us)
        U2 = [U + gp.tau * tucker(kron_sum_action(U, gp.A[c]) + G[c], gp.phi1[c])
              for c, U in enumerate(Us)]
        G2 = general.poly_reaction(gp.terms, U2)
        return [U2[c] + gp.tau * tucker(G2[c] - G[c], gp.phi2[c]) for c in range(gp.m)]

    errs, o1, o2 = _order_errors(planted)
    assert not (1.8 <= o1 <= 2.3 and 1.8 <= o2 <= 2.3), (errs, o1, o2)


def test_planted_wrong_term_component_breaks_the_linear_pin(monkeypatch):
    """A reaction evaluator that adds each term to the wrong component fails
    the exact linear-dynamics pin above."""
    orig = general.poly_reaction

    def planted(terms, Us):
        return orig([((c + 1) % len(Us), e, k) for c, e, k in terms], Us)

    monkeypatch.setattr(general, "poly_reaction", planted)
    with pytest.raises(AssertionError):
        test_linear_reaction_uniform_mode_is_heun_exactly()
