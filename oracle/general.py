"""ETD2RKds for m >= 1 components with arbitrary dense directional matrices
and polynomial reactions: the general setting of the method (Sec. 1,
Eq. 3-4: any A_mu in the Kronecker sum; Sec. 3, closing remark: the scheme
extends to more than two components).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy FP64.

Reaction: a list of monomial terms (c, exps, coef), each adding
coef * prod_j U_j^exps[j] to g^c.  The step is Eq. 11 component by
component:
    W_c  = sum_mu U_c x_mu A_mu^c + G_c(U)
    U2_c = U_c + tau W_c x_1 phi_1(tau A_1^c) ... x_d phi_1(tau A_d^c)
    U+_c = U2_c + 2^(d-1) tau (G_c(U2) - G_c(U)) x_mu phi_2(tau A_mu^c)
with every stage value U2 formed before any stage-2 reaction.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

from .matfun import phi_augmented
from .tensor import kron_dense, kron_sum_action, kron_sum_dense, tucker

Term = Tuple[int, Tuple[int, ...], float]


def poly_reaction(terms: Sequence[Term], Us: Sequence[np.ndarray]) -> List[np.ndarray]:
    """g^c(U) = sum over the terms of component c of coef * prod_j U_j^e_j."""
    G = [np.zeros_like(Us[0]) for _ in Us]
    for c, exps, coef in terms:
        t = np.full_like(Us[0], float(coef))
        for j, e in enumerate(exps):
            for _ in range(int(e)):
                t = t * Us[j]
        G[c] = G[c] + t
    return G


@dataclasses.dataclass
class GeneralPlan:
    d: int
    m: int
    tau: float
    terms: List[Term]
    A: List[List[np.ndarray]]     # A[c][mu]
    phi1: List[List[np.ndarray]]
    phi2: List[List[np.ndarray]]


def make_general_plan(A: Sequence[Sequence[np.ndarray]], tau: float,
                      terms: Sequence[Term]) -> GeneralPlan:
    """phi_1, phi_2 of tau A_mu^c for every component and direction (Eq. 9
    through the augmented-matrix exponential)."""
    A = [list(Ac) for Ac in A]
    P1, P2 = [], []
    for Ac in A:
        fns = [phi_augmented(tau * Am) for Am in Ac]
        P1.append([f[1] for f in fns])
        P2.append([f[2] for f in fns])
    return GeneralPlan(d=len(A[0]), m=len(A), tau=tau, terms=list(terms), A=A, phi1=P1, phi2=P2)


def etd2rkds_step_general(plan: GeneralPlan, Us: Sequence[np.ndarray]) -> List[np.ndarray]:
    tau, d = plan.tau, plan.d
    G = poly_reaction(plan.terms, Us)
    U2 = [U + tau * tucker(kron_sum_action(U, plan.A[c]) + G[c], plan.phi1[c])
          for c, U in enumerate(Us)]
    G2 = poly_reaction(plan.terms, U2)
    c2 = 2.0 ** (d - 1) * tau
    return [U2[c] + c2 * tucker(G2[c] - G[c], plan.phi2[c]) for c in range(plan.m)]


def etd2rkds_solve_general(plan: GeneralPlan, Us: Sequence[np.ndarray], nsteps: int):
    Us = [np.array(U, dtype=np.float64) for U in Us]
    for _ in range(nsteps):
        Us = etd2rkds_step_general(plan, Us)
    return Us


def etd2rkds_step_general_dense_form(plan: GeneralPlan, Us: Sequence[np.ndarray]):
    """The same step with the Tucker operators as explicit Kronecker
    products (Eq. 5) and K as the assembled Kronecker sum (Eq. 3); tiny grids
    only, independent of the mode product."""
    tau, d = plan.tau, plan.d
    shape = Us[0].shape
    us = [U.ravel() for U in Us]
    K = [kron_sum_dense(plan.A[c]) for c in range(plan.m)]
    P1 = [kron_dense(plan.phi1[c]) for c in range(plan.m)]
    P2 = [kron_dense(plan.phi2[c]) for c in range(plan.m)]
    g = poly_reaction(plan.terms, us)
    u2 = [us[c] + tau * P1[c] @ (K[c] @ us[c] + g[c]) for c in range(plan.m)]
    g2 = poly_reaction(plan.terms, u2)
    c2 = 2.0 ** (d - 1) * tau
    return [(u2[c] + c2 * P2[c] @ (g2[c] - g[c])).reshape(shape) for c in range(plan.m)]


def brusselator_terms(a: float, b: float) -> List[Term]:
    """The Brusselator of Eq. 17 as monomials: g^u = a - (b+1) u + u^2 v,
    g^v = b u - u^2 v."""
    return [(0, (0, 0), a), (0, (1, 0), -(b + 1.0)), (0, (2, 1), 1.0),
            (1, (1, 0), b), (1, (2, 1), -1.0)]
