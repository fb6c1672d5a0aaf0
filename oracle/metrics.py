"""Error measures and dynamics indicators (Sec. 4).

* ``paper_rel_err``: the paper measures "the 2-norm of the relative Frobenius
  norm of the solutions U and V at final time".  Reading taken:
  sqrt(e_U^2 + e_V^2) with e_X = ||X - X_ref||_F / ||X_ref||_F.
* ``max_rel_err``: per component ||X - X_ref||_inf / ||X_ref||_inf, maximum
  over the two components.  This is the "max rel err vs FP64" measure of the
  GPU results (fields that pass through zero make a pointwise relative error
  ill-defined, so the norm-wise form is used).
* ``indicators``: spatial mean <U_n> (trapezoid weights over the vertex grid,
  normalised by the domain measure) and the increment ||U_{n+1} - U_n||_F.
"""
from __future__ import annotations

import numpy as np


def _relF(X, R):
    return float(np.linalg.norm((X - R).ravel()) / np.linalg.norm(R.ravel()))


def paper_rel_err(U, V, Uref, Vref) -> float:
    return float(np.hypot(_relF(U, Uref), _relF(V, Vref)))


def max_rel_err(U, V, Uref, Vref) -> float:
    eu = np.max(np.abs(U - Uref)) / np.max(np.abs(Uref))
    ev = np.max(np.abs(V - Vref)) / np.max(np.abs(Vref))
    return float(max(eu, ev))


def trapezoid_weights(n: int) -> np.ndarray:
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    return w


def spatial_mean(U: np.ndarray) -> float:
    """<U> = (1/|Omega|) int u dx by the trapezoid rule on the vertex grid
    (grid spacing cancels against |Omega|)."""
    W = np.ones(())
    for n in U.shape:
        W = np.multiply.outer(W, trapezoid_weights(n))
    return float(np.sum(W * U) / np.sum(W))


def indicators(U_prev: np.ndarray, U_next: np.ndarray):
    """(<U_next>, ||U_next - U_prev||_F)."""
    return spatial_mean(U_next), float(np.linalg.norm((U_next - U_prev).ravel()))
