"""Reaction terms g^u(u, v), g^v(u, v), evaluated pointwise.

* Schnakenberg (Sec. 4.1, Eq. 12), params (gamma, a, b):
      g^u = gamma (a - u + u^2 v),   g^v = gamma (b - u^2 v)
* FitzHugh-Nagumo variant with linear recovery, params (eps, a1, a0):
      g^u = u - u^3 - v,             g^v = eps (u - a1 v - a0)
  (the paper's own FHN form, Sec. 4.2, Eq. 13, with rho = 1 is this one with
  eps = a_1^v, a1 = a_2^v and a0 = 0)
* Advective Brusselator (Sec. 4.6, Eq. 17, with a_2 -> a, a_1 -> b),
  params (a, b):
      g^u = a - (b + 1) u + u^2 v,   g^v = b u - u^2 v
* No reaction, g^u = g^v = 0: the linear advection-diffusion case used by
  the g = 0 checks of the splitting.
"""
from __future__ import annotations

import numpy as np

SCHNAKENBERG = 0
FHN = 1
BRUSSELATOR = 2
NO_REACTION = 3


def reaction(model: int, params, U: np.ndarray, V: np.ndarray):
    """(G^u, G^v) at every grid point."""
    if model == SCHNAKENBERG:
        gamma, a, b = params[:3]
        u2v = U * U * V
        return gamma * (a - U + u2v), gamma * (b - u2v)
    if model == FHN:
        eps, a1, a0 = params[:3]
        return U - U * U * U - V, eps * (U - a1 * V - a0)
    if model == BRUSSELATOR:
        a, b = params[:2]
        u2v = U * U * V
        return a - (b + 1.0) * U + u2v, b * U - u2v
    if model == NO_REACTION:
        return np.zeros_like(U), np.zeros_like(V)
    raise ValueError(f"unknown model {model}")
