"""Tensor operations of Sec. 2.

A state tensor W of order d is stored as a numpy array of shape
(n_d, ..., n_1): x_1 is the last (fastest) axis, so W.ravel() is the
column-major vec(W) of Sec. 2, and direction mu lives on axis d - mu.
"""
from __future__ import annotations

from functools import reduce
from typing import Sequence

import numpy as np


def mode_product(W: np.ndarray, M: np.ndarray, mu: int) -> np.ndarray:
    """mu-mode product W x_mu M (Sec. 2, text around Eq. 5): M multiplies the
    mu-fibres of W,  (W x_mu M)[.., i_mu, ..] = sum_j M[i_mu, j] W[.., j, ..].
    mu is 1-based."""
    d = W.ndim
    axis = d - mu
    Y = np.tensordot(M, W, axes=([1], [axis]))   # new axis 0 = i_mu
    return np.moveaxis(Y, 0, axis)


def tucker(W: np.ndarray, Ms: Sequence[np.ndarray]) -> np.ndarray:
    """Tucker operator W x_1 M_1 x_2 ... x_d M_d (Eq. 5)."""
    for mu, M in enumerate(Ms, start=1):
        W = mode_product(W, M, mu)
    return W


def kron_sum_action(W: np.ndarray, As: Sequence[np.ndarray]) -> np.ndarray:
    """K vec(W) in tensor form: sum_mu W x_mu A_mu (Sec. 2, Eq. 6 and the
    identity after it)."""
    return sum(mode_product(W, A, mu) for mu, A in enumerate(As, start=1))


def kron_dense(Ms: Sequence[np.ndarray]) -> np.ndarray:
    """M_d kron ... kron M_1 as one dense matrix (Eq. 5's right-hand side in
    matrix form); only for tiny grids."""
    return reduce(np.kron, list(reversed(list(Ms))))


def kron_sum_dense(As: Sequence[np.ndarray]) -> np.ndarray:
    """K = A_d (+) ... (+) A_1 = sum_mu I_d x .. x A_mu x .. x I_1 (Eq. 3)."""
    ns = [A.shape[0] for A in As]
    K = 0
    for mu, A in enumerate(As):
        factors = [np.eye(n) for n in ns]
        factors[mu] = A
        K = K + kron_dense(factors)
    return K
