"""Column supports of the tensor-core mode products.

The matrices phi_l(tau A_mu) of Eq. 11 are dense, but their entries decay
quickly away from the diagonal: on the FHN 1024^2 grid every row holds all
but 2^-40 of its absolute sum within about 50 columns of the diagonal.  The
tensor-core path therefore contracts each 128-row group of a matrix only over
the column range that holds that mass (widened to multiples of 64 columns).

These tests check
- the multiply-add count the library reports against a numpy restatement of
  the support rule on the oracle's matrices,
- that results with and without supports (ADR_KSUPPORT=0) agree to rounding
  level, and both with the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import schemes

pytestmark = pytest.mark.gpu

TOL = 1e-5
DROP = 2.0 ** -40
# kernel choice -> (rows per tile of phi, K values per block)
KERNELS = {0: (128, 32), 1: (128, 64), 2: (64, 32), 3: (128, 32), 4: (128, 64)}


@pytest.fixture(scope="module")
def adr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2307_10684_gb300 import build
    build.build()
    import paper_2307_10684_gb300 as adr
    return adr


def group_supports(M, group=128):
    """Per 128-row group: the union of the rows' narrowest column ranges that
    leave out at most DROP of the row's absolute sum (half on each side),
    widened to multiples of 64 columns."""
    n = M.shape[0]
    A = np.abs(M)
    tot = A.sum(axis=1)
    t = 0.5 * DROP * tot
    before = np.cumsum(A, axis=1) - A                     # sum_{j < l}, nondecreasing in l
    from_h = np.cumsum(A[:, ::-1], axis=1)[:, ::-1]       # sum_{j >= h}, nonincreasing in h
    lo = (before <= t[:, None]).sum(axis=1) - 1           # the last l with sum_{j < l} <= t
    hi = (from_h > t[:, None]).sum(axis=1)                # one past the last h with sum > t
    zero = tot == 0.0
    lo[zero] = np.arange(n)[zero]
    hi[zero] = lo[zero] + 1
    out = []
    for g0 in range(0, n, group):
        lo_g, hi_g = int(lo[g0:g0 + group].min()), int(hi[g0:g0 + group].max())
        out.append((lo_g // 64 * 64, min(n, -(-hi_g // 64) * 64)))
    return out


_PLANS = {}


def oracle_plan(p):
    key = (p.d, tuple(p.n), p.seed, p.model)
    if key not in _PLANS:
        _PLANS[key] = schemes.make_plan(p)
    return _PLANS[key]


def expected_macs(p, kernel, fused):
    """(dense, computed) multiply-adds of one ETD2RKds step.  fused: the first
    two directions of each Tucker operator are one two-mode launch per x3
    slab (MMA1 over the union of the Phi_b tiles' x2 supports of a unit, in
    groups of up to 256 padded to 64 -- one unit holds every x2 tile when
    n2 <= 256; MMA2 per tile over its chunks), and a 3D operator's x3 product
    is a launch of its own; otherwise one launch per direction."""
    bn, bk = KERNELS[kernel]
    op = oracle_plan(p)
    N = int(np.prod(p.n))
    dense = computed = 0.0
    for mats in (op.phi1, op.phi2):
        for c in range(2):
            if fused:
                n1, n2 = p.n[0], p.n[1]
                slabs = N // (n1 * n2)
                dense += slabs * (n1 * n1 * n2 + n2 * n2 * n1)
                sa, sb = group_supports(mats[c][0]), group_supports(mats[c][1])
                tn = -(-n2 // 128)
                bunit = tn if n2 <= 256 else 1  # tiles sharing one intermediate
                for a0 in range(0, n1, 128):
                    lo, hi = sa[a0 // 128]
                    kb0, kb1 = lo // 32, min(-(-n1 // 32), -(-hi // 32))
                    rows = min(128, n1 - a0)
                    kin = min(kb1 * 32, n1) - kb0 * 32
                    for b0 in range(0, tn, bunit):
                        tiles = range(b0, b0 + bunit)
                        lo2 = min(sb[b][0] for b in tiles)
                        hi2 = max(sb[b][1] for b in tiles)
                        for g2 in range(lo2, hi2, 256):
                            nch = -(-min(256, hi2 - g2) // 64)
                            computed += slabs * rows * 64 * nch * kin
                            for b in tiles:
                                c0 = max(0, (sb[b][0] - g2) // 64)
                                c1 = min(nch, -(-(sb[b][1] - g2) // 64))
                                if c1 > c0:
                                    computed += slabs * rows * min(128, n2 - 128 * b) * 64 * (c1 - c0)
                if p.d == 2:
                    continue
            for mu in range(2 if fused else 0, p.d):
                K = p.n[mu]
                M = N // K
                sup = group_supports(mats[c][mu])
                dense += M * K * K
                for n0 in range(0, K, bn):
                    lo, hi = sup[n0 // 128]
                    nk = -(-K // bk)
                    kb0, kb1 = lo // bk, min(nk, -(-hi // bk))
                    rows = min(bn, K - n0)
                    computed += M * rows * (min(kb1 * bk, K) - kb0 * bk)
    return dense, computed


def solve(adr, p, u0, v0, nsteps, kernel=-1):
    import torch
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    v = torch.tensor(v0, dtype=torch.float32, device="cuda")
    with adr.Plan(p, kernel=kernel) as plan:
        macs = plan.mode_product_macs()
        plan.step(u, v, nsteps)
        assert plan.stats()["device_error"] == 0
    torch.cuda.synchronize()
    return u.double().cpu().numpy(), v.double().cpu().numpy(), macs


CASES = {
    "fhn1024": lambda: wl.fhn_1024(precision=wl.BF16X3, nsteps=10),
    "fhn_rect": lambda: wl.Problem(d=2, n=(384, 200), lo=(0.0, 0.0), hi=(40.0, 20.0),
                                   diff=(1.0, 20.0), adv=((0.5, 0.5), (0.5, 0.5)), model=wl.FHN,
                                   params=(0.05, 2.0, -0.03), tau=1e-2, nsteps=10,
                                   precision=wl.BF16X3, seed=41),
    "bruss3d": lambda: wl.Problem(d=3, n=(128, 64, 96), lo=(0.0,) * 3, hi=(1.0,) * 3,
                                  diff=(0.02, 0.1), adv=((-0.5,) * 3, (-0.5,) * 3),
                                  model=wl.BRUSSELATOR, params=(1.0, 3.0), tau=1e-2, nsteps=5,
                                  precision=wl.BF16X3, seed=43),
}


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("kernel", [0, 2, 4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_reported_work_matches_the_support_rule(adr, case, kernel, fused, monkeypatch):
    p = CASES[case]()
    if not fused:
        monkeypatch.setenv("ADR_TC_FUSED", "0")
    with adr.Plan(p, kernel=kernel) as plan:
        dense, computed = plan.mode_product_macs()
    e_dense, e_comp = expected_macs(p, kernel, fused)
    assert dense == e_dense == 4 * np.prod(p.n) * sum(p.n)
    # a row whose prefix sum sits on the threshold could round either way in
    # the two FP64 summation orders and move one range end by 64 columns
    assert computed == pytest.approx(e_comp, rel=0.02), (computed, e_comp)


@pytest.mark.parametrize("fused", [True, False])
def test_fhn1024_contracts_a_fraction_of_k(adr, fused, monkeypatch):
    """The headline grid: the supports cut the tensor-core work to under 40%
    of the dense products (fused: MMA1 runs over up to 256 x2 values for 128
    output rows, so its share is higher than the per-direction passes')."""
    if not fused:
        monkeypatch.setenv("ADR_TC_FUSED", "0")
    p = CASES["fhn1024"]()
    with adr.Plan(p, kernel=4) as plan:
        dense, computed = plan.mode_product_macs()
    assert computed / dense < (0.4 if fused else 0.25)


@pytest.mark.parametrize("case", sorted(CASES))
def test_supports_off_agrees(adr, case, monkeypatch):
    p = CASES[case]()
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, wl.FP32), wl.round_to(v0, wl.FP32)
    U, V, (dense, computed) = solve(adr, p, u0, v0, p.nsteps)
    monkeypatch.setenv("ADR_KSUPPORT", "0")
    Uf, Vf, (dense_f, computed_f) = solve(adr, p, u0, v0, p.nsteps)
    assert dense_f == dense and computed_f >= computed
    # the left-out mass is 2^-40 of each row; what differs is rounding
    assert oracle.max_rel_err(U, V, Uf, Vf) <= 1e-6
    Ur, Vr = schemes.etd2rkds_solve(oracle_plan(p), u0, v0, p.nsteps)
    assert oracle.max_rel_err(U, V, Ur, Vr) <= TOL
    assert oracle.max_rel_err(Uf, Vf, Ur, Vr) <= TOL


def test_every_kernel_runs_the_same_supports(adr, monkeypatch):
    """The supports do not depend on the kernel choice: all five
    per-direction kernels give bitwise the same state."""
    monkeypatch.setenv("ADR_TC_FUSED", "0")
    p = CASES["fhn_rect"]()
    u0, v0 = wl.initial_data(p)
    outs = [solve(adr, p, u0, v0, 5, kernel=k)[:2] for k in range(5)]
    for k in range(1, 5):
        assert np.array_equal(outs[k][0], outs[0][0]) and np.array_equal(outs[k][1], outs[0][1]), k
