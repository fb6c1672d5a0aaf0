"""FP64 CPU oracle of the ETD2RKds time stepper (Caliari & Cassini,
arXiv:2307.10684).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may call it.  It shares no code with the CUDA
path; the only common module is ``workloads`` (seeded inputs, no method
arithmetic).

Everything here is plain numpy in float64, written from the paper:

* ``fd``       - grid and the second-order centred finite-difference matrices
                 A_mu with homogeneous Neumann rows (Sec. 4, opening text).
* ``matfun``   - e^X, phi_1(X), phi_2(X) of small dense matrices (Eq. 9,
                 the phi_ell definition) by Pade [13/13] scaling and squaring
                 of the 3n x 3n augmented matrix.
* ``tensor``   - mu-mode product, Tucker operator (Eq. 5) and the
                 Kronecker-sum action K U (Eq. 6).
* ``models``   - reaction terms g^u, g^v (Eq. 12, Eq. 17 and a FitzHugh-Nagumo
                 variant with advection).
* ``schemes``  - ETD2RKds (Sec. 3, Eq. 11), plus Lawson2b (Eq. 7) and unsplit
                 dense ETD2RK (Eq. 8) used as references on tiny grids.
* ``metrics``  - relative error measures and the dynamics indicators (Sec. 4).

Parity status: every function is pinned by a ``-m "not gpu"`` test except
where its docstring says "parity unpinned".
"""
from .fd import grid, fd_matrix, direction_matrices  # noqa: F401
from .matfun import pade13_coefficients, expm_pade13, phi_augmented, phi_eigen  # noqa: F401
from .tensor import mode_product, tucker, kron_sum_action  # noqa: F401
from .models import reaction  # noqa: F401
from .schemes import Plan, make_plan, etd2rkds_step, etd2rkds_solve  # noqa: F401
from .metrics import max_rel_err, paper_rel_err, indicators  # noqa: F401
