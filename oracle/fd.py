"""Space discretisation (Sec. 4, opening text; Eq. 2-4 for the Kronecker-sum
structure).

The paper discretises diffusion and advection with second-order centred
finite differences on equispaced points and embeds homogeneous Neumann
conditions into the matrices, which are tridiagonal.  It does not say whether
the grid is vertex- or cell-centred nor how the Neumann rows are formed.
Reading taken here: vertex-centred grid x_i = lo + i h, h = (hi - lo)/(n - 1),
and a ghost value mirrored across each boundary (u_{-1} = u_1,
u_n = u_{n-2}).  For the operator  delta * d2/dx2 - alpha * d/dx  this gives

    interior row i:   A[i,i-1] = delta/h^2 + alpha/(2h)
                      A[i,i]   = -2 delta/h^2
                      A[i,i+1] = delta/h^2 - alpha/(2h)
    row 0:            A[0,0] = -2 delta/h^2,   A[0,1] = 2 delta/h^2
    row n-1:          A[n-1,n-1] = -2 delta/h^2, A[n-1,n-2] = 2 delta/h^2

(the centred advection difference vanishes under the mirror).
"""
from __future__ import annotations

import numpy as np


def grid(n: int, lo: float, hi: float) -> np.ndarray:
    """Vertex-centred equispaced points x_0 = lo, ..., x_{n-1} = hi."""
    return lo + (hi - lo) * np.arange(n, dtype=np.float64) / (n - 1)


def fd_matrix(n: int, lo: float, hi: float, delta: float, alpha: float) -> np.ndarray:
    """Dense n x n matrix of delta d2/dx2 - alpha d/dx with Neumann rows."""
    if n < 3:
        raise ValueError("need n >= 3 grid points")
    h = (hi - lo) / (n - 1)
    A = np.zeros((n, n), dtype=np.float64)
    lower = delta / h ** 2 + alpha / (2.0 * h)
    diag = -2.0 * delta / h ** 2
    upper = delta / h ** 2 - alpha / (2.0 * h)
    for i in range(1, n - 1):
        A[i, i - 1] = lower
        A[i, i] = diag
        A[i, i + 1] = upper
    A[0, 0] = diag
    A[0, 1] = 2.0 * delta / h ** 2
    A[n - 1, n - 1] = diag
    A[n - 1, n - 2] = 2.0 * delta / h ** 2
    return A


def direction_matrices(problem, component: int):
    """[A_1, ..., A_d] for component c (0 = u, 1 = v) of a workloads.Problem."""
    return [fd_matrix(problem.n[m], problem.lo[m], problem.hi[m],
                      problem.diff[component], problem.adv[component][m])
            for m in range(problem.d)]
