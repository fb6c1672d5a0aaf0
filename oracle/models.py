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
* FitzHugh-Nagumo in the paper's form (Sec. 4.2, Eq. 13; Sec. 4.3, Eq. 14),
  params (rho, a1, a2):
      g^u = rho (-u (u^2 - 1) - v),  g^v = rho a1 (u - a2 v)
* Morpho-chemical DIB model (Sec. 4.4, Eq. 15), params
  (rho, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v):
      g^u = rho (a1u (1 - v) u - a2u u^3 - a3u (v - a4u))
      g^v = rho (a1v (1 + a2v u)(1 - v)(1 - a3v (1 - v))
                 - a4v v (1 + a5v u)(1 + a3v v))
"""
from __future__ import annotations

import numpy as np

SCHNAKENBERG = 0
FHN = 1
BRUSSELATOR = 2
NO_REACTION = 3
FHN_RHO = 4
DIB = 5


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
    if model == FHN_RHO:
        rho, a1, a2 = params[:3]
        return rho * (-U * (U * U - 1.0) - V), rho * a1 * (U - a2 * V)
    if model == DIB:
        rho, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v = params[:10]
        gu = rho * (a1u * (1.0 - V) * U - a2u * U ** 3 - a3u * (V - a4u))
        gv = rho * (a1v * (1.0 + a2v * U) * (1.0 - V) * (1.0 - a3v * (1.0 - V))
                    - a4v * V * (1.0 + a5v * U) * (1.0 + a3v * V))
        return gu, gv
    raise ValueError(f"unknown model {model}")
