"""Matrix functions of small dense matrices: e^X, phi_1(X), phi_2(X).

phi_ell is defined in Sec. 2, Eq. (9):
    phi_ell(X) = int_0^1 theta^(ell-1)/(ell-1)! e^((1-theta) X) dtheta,
equivalently phi_ell(X) = sum_k X^k / (k + ell)!.

The paper computes them by quadrature plus a modified scaling and squaring
(Sec. 4, opening text).  This oracle instead evaluates them, as the build's
method statement fixes, through the exponential of the augmented matrix

    Ahat = [[X, I, 0],
            [0, 0, I],
            [0, 0, 0]]      exp(Ahat) = [[e^X, phi_1(X), phi_2(X)], [0, I, I], [0, 0, I]]

(Higham, "Functions of Matrices", SIAM 2008, Sec. 10.7.4; Saad 1992), with
exp taken by the Pade [13/13] scaling-and-squaring method of Higham,
"The scaling and squaring method for the matrix exponential revisited",
SIMAX 26 (2005).  The Pade coefficients are generated from their closed form.

``phi_eigen`` is a second, independent route (diagonal symmetrisation of a
tridiagonal matrix and an eigendecomposition) used only to pin the first.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import List, Tuple

import numpy as np

# Largest scaled 1-norm for which the [13/13] Pade approximant meets double
# precision backward error (Higham 2005, Table 2.3).
THETA13 = 5.371920351148152


def pade13_coefficients() -> List[Fraction]:
    """b_j, j = 0..13, of the numerator p_13(x) = sum_j b_j x^j of the
    diagonal [13/13] Pade approximant of e^x:
        b_j = (2m - j)! m! / ((2m)! j! (m - j)!),   m = 13.
    The denominator is q_13(x) = p_13(-x).  Returned as exact fractions,
    scaled so that b_13 = 1 (a common factor cancels in q^{-1} p)."""
    m = 13
    b = [Fraction(math.factorial(2 * m - j) * math.factorial(m),
                  math.factorial(2 * m) * math.factorial(j) * math.factorial(m - j))
         for j in range(m + 1)]
    return [x / b[m] for x in b]


def _norm1(X: np.ndarray) -> float:
    return float(np.max(np.sum(np.abs(X), axis=0))) if X.size else 0.0


def scaling_power(X: np.ndarray) -> int:
    """s = max(0, ceil(log2(||X||_1 / theta_13)))."""
    nrm = _norm1(X)
    if nrm <= THETA13:
        return 0
    return max(0, int(math.ceil(math.log2(nrm / THETA13))))


def expm_pade13(X: np.ndarray) -> np.ndarray:
    """e^X by Pade [13/13] with scaling and squaring (Higham 2005).

    Scale X by 2^-s, evaluate p_13 and q_13 with the even/odd split
    p = V + U, q = V - U, U = X (odd part in X^2), V = even part, using X^2,
    X^4, X^6; solve q R = p; square R s times."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    b = [float(c) for c in pade13_coefficients()]
    s = scaling_power(X)
    Xs = X / (2.0 ** s)
    I = np.eye(n)
    X2 = Xs @ Xs
    X4 = X2 @ X2
    X6 = X2 @ X4
    U = Xs @ (X6 @ (b[13] * X6 + b[11] * X4 + b[9] * X2)
              + b[7] * X6 + b[5] * X4 + b[3] * X2 + b[1] * I)
    V = (X6 @ (b[12] * X6 + b[10] * X4 + b[8] * X2)
         + b[6] * X6 + b[4] * X4 + b[2] * X2 + b[0] * I)
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def phi_augmented(X: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(e^X, phi_1(X), phi_2(X)) from the first block row of exp(Ahat)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    Ah = np.zeros((3 * n, 3 * n))
    Ah[:n, :n] = X
    Ah[:n, n:2 * n] = np.eye(n)
    Ah[n:2 * n, 2 * n:] = np.eye(n)
    E = expm_pade13(Ah)
    return E[:n, :n].copy(), E[:n, n:2 * n].copy(), E[:n, 2 * n:].copy()


def phi_scalar(x: np.ndarray, ell: int) -> np.ndarray:
    """Scalar phi_ell(x), ell in {0, 1, 2}: closed forms e^x, (e^x-1)/x,
    (e^x-1-x)/x^2, with the series sum_k x^k/(k+ell)! near 0."""
    x = np.asarray(x, dtype=np.float64)
    if ell == 0:
        return np.exp(x)
    small = np.abs(x) < 0.5
    out = np.empty_like(x)
    xs = x[small]
    ser = np.zeros_like(xs)
    for k in range(24, -1, -1):
        ser = ser * xs + 1.0 / math.factorial(k + ell)
    out[small] = ser
    xl = x[~small]
    if ell == 1:
        out[~small] = np.expm1(xl) / xl
    elif ell == 2:
        out[~small] = (np.expm1(xl) - xl) / xl ** 2
    else:
        raise ValueError(ell)
    return out


def phi_eigen(X: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(e^X, phi_1(X), phi_2(X)) for a tridiagonal X whose off-diagonal
    products X[i,i+1] X[i+1,i] are positive: D X D^-1 is symmetric for
    d_{i+1} = d_i sqrt(X[i,i+1]/X[i+1,i]); with D X D^-1 = Q diag(l) Q^T,
    f(X) = D^-1 Q f(diag(l)) Q^T D.  Well conditioned only while the d_i stay
    within a few orders of magnitude (small grids or no advection)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    d = np.ones(n)
    for i in range(n - 1):
        if X[i, i + 1] * X[i + 1, i] <= 0.0:
            raise ValueError("not diagonally symmetrisable")
        d[i + 1] = d[i] * math.sqrt(X[i, i + 1] / X[i + 1, i])
    B = (d[:, None] * X) / d[None, :]
    B = 0.5 * (B + B.T)
    lam, Q = np.linalg.eigh(B)
    left = Q / d[:, None]          # D^-1 Q
    right = Q.T * d[None, :]       # Q^T D
    return tuple(left @ (phi_scalar(lam, ell)[:, None] * right) for ell in (0, 1, 2))
