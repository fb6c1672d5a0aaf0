"""Time steppers for the tensor ODE system of Sec. 2, Eq. (6).

* ``etd2rkds_step`` - ETD2RKds, Sec. 3, Eq. (11): the directional split
  ETD2RK.  Stage 1 applies the Tucker operator of phi_1(tau A_mu) to
  tau (K U + G(U, V)); stage 2 applies the Tucker operator of phi_2(tau A_mu)
  to 2^(d-1) tau (G(U2, V2) - G(U, V)).  The factor 2^(d-1) is (ell!)^(d-1)
  of the splitting formula Eq. (10a) at ell = 2.
* ``lawson2b_step`` - Lawson2b in tensor form, Eq. (7).
* ``etd2rk_dense_step`` - unsplit ETD2RK, Eq. (8), with phi_ell(tau K) of the
  assembled N x N Kronecker sum (tiny grids only).

A Plan holds, per component c in {u, v} and direction mu, the directional
matrix A_mu^c and phi_1(tau A_mu^c), phi_2(tau A_mu^c) (and e^(tau A_mu^c)
for Lawson2b), computed once for the constant step tau as the paper does
(Sec. 4, opening text).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from .fd import direction_matrices
from .matfun import phi_augmented
from .models import reaction
from .tensor import kron_dense, kron_sum_action, kron_sum_dense, tucker


@dataclasses.dataclass
class Plan:
    d: int
    tau: float
    model: int
    params: tuple
    A: List[List[np.ndarray]]        # A[c][mu]
    E: List[List[np.ndarray]]        # e^(tau A[c][mu])
    phi1: List[List[np.ndarray]]     # phi_1(tau A[c][mu])
    phi2: List[List[np.ndarray]]     # phi_2(tau A[c][mu])


def make_plan_from_matrices(A_u: Sequence[np.ndarray], A_v: Sequence[np.ndarray],
                            tau: float, model: int, params) -> Plan:
    """Plan from arbitrary dense directional matrices (the method does not
    need the A_mu to be tridiagonal, Sec. 1)."""
    A = [list(A_u), list(A_v)]
    E, P1, P2 = [], [], []
    for c in range(2):
        trip = [phi_augmented(tau * Am) for Am in A[c]]
        E.append([t[0] for t in trip])
        P1.append([t[1] for t in trip])
        P2.append([t[2] for t in trip])
    return Plan(d=len(A_u), tau=tau, model=model, params=tuple(params),
                A=A, E=E, phi1=P1, phi2=P2)


def make_plan(problem, tau: Optional[float] = None) -> Plan:
    """Plan for a workloads.Problem (finite-difference A_mu of oracle.fd)."""
    t = problem.tau if tau is None else tau
    return make_plan_from_matrices(direction_matrices(problem, 0),
                                   direction_matrices(problem, 1),
                                   t, problem.model, problem.params)


def etd2rkds_step(plan: Plan, U: np.ndarray, V: np.ndarray):
    """One ETD2RKds step, Eq. (11):
        U2 = U + tau (sum_mu U x_mu A_mu^u + G^u(U,V)) x_{mu=1..d} phi_1(tau A_mu^u)
        V2 = V + tau (sum_mu V x_mu A_mu^v + G^v(U,V)) x_{mu=1..d} phi_1(tau A_mu^v)
        U+ = U2 + 2^(d-1) tau (G^u(U2,V2) - G^u(U,V)) x_{mu=1..d} phi_2(tau A_mu^u)
        V+ = V2 + 2^(d-1) tau (G^v(U2,V2) - G^v(U,V)) x_{mu=1..d} phi_2(tau A_mu^v)
    Both stage values U2, V2 are formed before either stage-2 reaction."""
    tau, d = plan.tau, plan.d
    GU, GV = reaction(plan.model, plan.params, U, V)
    WU = kron_sum_action(U, plan.A[0]) + GU
    WV = kron_sum_action(V, plan.A[1]) + GV
    U2 = U + tau * tucker(WU, plan.phi1[0])
    V2 = V + tau * tucker(WV, plan.phi1[1])
    GU2, GV2 = reaction(plan.model, plan.params, U2, V2)
    c2 = 2.0 ** (d - 1) * tau
    Un = U2 + c2 * tucker(GU2 - GU, plan.phi2[0])
    Vn = V2 + c2 * tucker(GV2 - GV, plan.phi2[1])
    return Un, Vn


def etd2rkds_solve(plan: Plan, U0: np.ndarray, V0: np.ndarray, nsteps: int, callback=None):
    """nsteps ETD2RKds steps from (U0, V0); callback(n, U, V) after each."""
    U, V = np.array(U0, dtype=np.float64), np.array(V0, dtype=np.float64)
    for n in range(nsteps):
        U, V = etd2rkds_step(plan, U, V)
        if callback is not None:
            callback(n + 1, U, V)
    return U, V


def lawson2b_step(plan: Plan, U: np.ndarray, V: np.ndarray):
    """One Lawson2b step in tensor form, Eq. (7)."""
    tau = plan.tau
    GU, GV = reaction(plan.model, plan.params, U, V)
    U2 = tucker(U + tau * GU, plan.E[0])
    V2 = tucker(V + tau * GV, plan.E[1])
    GU2, GV2 = reaction(plan.model, plan.params, U2, V2)
    Un = tucker(U + 0.5 * tau * GU, plan.E[0]) + 0.5 * tau * GU2
    Vn = tucker(V + 0.5 * tau * GV, plan.E[1]) + 0.5 * tau * GV2
    return Un, Vn


@dataclasses.dataclass
class DensePlan:
    """phi_ell(tau K^c) of the assembled Kronecker sums, for Eq. (8)."""
    tau: float
    model: int
    params: tuple
    shape: tuple
    K: List[np.ndarray]
    phi1: List[np.ndarray]
    phi2: List[np.ndarray]


def make_dense_plan(plan: Plan, shape) -> DensePlan:
    K = [kron_sum_dense(plan.A[c]) for c in range(2)]
    P1, P2 = [], []
    for c in range(2):
        _, p1, p2 = phi_augmented(plan.tau * K[c])
        P1.append(p1)
        P2.append(p2)
    return DensePlan(tau=plan.tau, model=plan.model, params=plan.params,
                     shape=tuple(shape), K=K, phi1=P1, phi2=P2)


def etd2rk_dense_step(dp: DensePlan, U: np.ndarray, V: np.ndarray):
    """One unsplit ETD2RK step, Eq. (8), on vec(U), vec(V)."""
    tau = dp.tau
    u, v = U.ravel(), V.ravel()
    gu, gv = reaction(dp.model, dp.params, u, v)
    u2 = u + tau * dp.phi1[0] @ (dp.K[0] @ u + gu)
    v2 = v + tau * dp.phi1[1] @ (dp.K[1] @ v + gv)
    gu2, gv2 = reaction(dp.model, dp.params, u2, v2)
    un = u2 + tau * dp.phi2[0] @ (gu2 - gu)
    vn = v2 + tau * dp.phi2[1] @ (gv2 - gv)
    return un.reshape(dp.shape), vn.reshape(dp.shape)


def etd2rkds_step_dense_form(plan: Plan, U: np.ndarray, V: np.ndarray):
    """Eq. (11) written with the Tucker operators as explicit Kronecker
    products (Eq. 5, Eq. 10b) and K as the assembled Kronecker sum (Eq. 3).
    Independent of mode_product; tiny grids only."""
    tau, d = plan.tau, plan.d
    u, v = U.ravel(), V.ravel()
    K = [kron_sum_dense(plan.A[c]) for c in range(2)]
    P1 = [kron_dense(plan.phi1[c]) for c in range(2)]
    P2 = [kron_dense(plan.phi2[c]) for c in range(2)]
    gu, gv = reaction(plan.model, plan.params, u, v)
    u2 = u + tau * P1[0] @ (K[0] @ u + gu)
    v2 = v + tau * P1[1] @ (K[1] @ v + gv)
    gu2, gv2 = reaction(plan.model, plan.params, u2, v2)
    c2 = 2.0 ** (d - 1) * tau
    un = u2 + c2 * P2[0] @ (gu2 - gu)
    vn = v2 + c2 * P2[1] @ (gv2 - gv)
    return un.reshape(U.shape), vn.reshape(V.shape)
