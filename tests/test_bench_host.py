"""bench.py's host-side logic (no GPU): the roofline arithmetic, the use of
the committed ncu captures, and the oracle baseline's scheme dispatch."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as wl  # noqa: E402
from oracle import schemes  # noqa: E402


def test_tensor_roofline_arithmetic():
    peaks = {"bf16_tflops": 2000.0, "hbm_gbs": 8000.0}
    # 10 launches of 1 GFLOP (algorithmic) and 1 MB in 1 ms in all
    kd = {"ms": 1.0, "count": 10, "flops": 10e9, "bytes": 10e6}
    r = bench.tc_roofline(kd, wl.BF16X3, peaks, "test", None)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(6 * 1e9 / 1e-4 / 1e12)  # six MMAs per product
    assert r["frac"] == pytest.approx(r["achieved"] / 2000.0)
    r32 = bench.tc_roofline(kd, wl.TF32X3, peaks, "test", None)
    assert r32["peak"] == pytest.approx(1000.0)  # tf32 at half the bf16 rate, 3 MMAs
    assert r32["achieved"] == pytest.approx(3 * 1e9 / 1e-4 / 1e12)


def test_hbm_roofline_arithmetic():
    peaks = {"bf16_tflops": 2000.0, "hbm_gbs": 8000.0}
    kd = {"ms": 1.0, "count": 10, "flops": 10e6, "bytes": 10e9}
    r = bench.tc_roofline(kd, wl.BF16X3, peaks, "test", 123)
    assert r["bound"] == "hbm" and r["traffic"] == 123
    assert r["achieved"] == pytest.approx(1e9 / 1e-4 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 8000.0)


def test_traffic_only_for_the_captured_source_and_kernel(tmp_path):
    """A capture summary is used only when its source hash is the current
    tc.cu's and its kernel is the one timed."""
    import hashlib
    src = os.path.join(ROOT, "paper_2307_10684_gb300", "csrc", "tc.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    (tmp_path / "tc_mode_fhn1024.md").write_text(
        f"source_sha256(tc.cu): {sha}\ncaptured_kernel: 4\ndram_bytes_per_launch: 25000000\n")
    (tmp_path / "tc_mode_old.md").write_text(
        "source_sha256(tc.cu): 0123456789abcdef\ncaptured_kernel: 4\n"
        "dram_bytes_per_launch: 25000000\n")
    assert bench.profiled_traffic("fhn1024", 4, str(tmp_path)) == 25000000
    assert bench.profiled_traffic("fhn1024", 0, str(tmp_path)) is None
    assert bench.profiled_traffic("old", 4, str(tmp_path)) is None
    assert bench.profiled_traffic("no_such_workload", 4, str(tmp_path)) is None
    # the fused two-mode kernel has its own summary
    (tmp_path / "tc_fused_fhn1024.md").write_text(
        f"source_sha256(tc.cu): {sha}\ncaptured_kernel: fused\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic("fhn1024", "fused", str(tmp_path)) == 123
    (tmp_path / "tc_fused_bruss256.md").write_text(
        f"source_sha256(tc.cu): {sha}\ncaptured_kernel: fused+0\ndram_bytes_per_launch: 456\n")
    assert bench.profiled_traffic("bruss256", "fused+0", str(tmp_path)) == 456
    assert bench.profiled_traffic("bruss256", "fused+4", str(tmp_path)) is None


def test_in_step_roofline_arithmetic():
    """Algorithmic work per mode-product launch: 4 n N flops per product and
    16 + 8/P bytes per point (P launches per Tucker operator); frac is the
    slower bound's share of the duration."""
    peaks = {"bf16_tflops": 2000.0, "hbm_gbs": 8000.0}
    p = wl.fhn_1024(precision=wl.BF16X3)  # 1024^2, d = 2
    N = 1024 * 1024
    r = bench.mode_product_roofline(p, wl.BF16X3, 0.02, 4, peaks, "test", None)
    assert r["algorithmic_flops_per_launch"] == pytest.approx(4 * 1024 * N)
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(20 * N + 8 * 1024 * 1024)
    t_tc = 4 * 1024 * N / 2e15
    t_hbm = (20 * N + 8 * 1024 * 1024) / 8e12
    assert r["bound"] == ("tensor" if t_tc >= t_hbm else "hbm")
    assert r["frac"] == pytest.approx(max(t_tc, t_hbm) / 2e-5)
    assert r["issued_tensor_frac"] == pytest.approx(6 * t_tc / 2e-5)
    # fused 2D operators: two launches per step, each two mode products
    # reading and writing the field once (24 B per point with the base)
    rf = bench.mode_product_roofline(p, wl.BF16X3, 0.02, 2, peaks, "test", None, 0.5)
    assert rf["mode_products_per_launch"] == 2
    assert rf["algorithmic_flops_per_launch"] == pytest.approx(8 * 1024 * N)
    assert rf["algorithmic_bytes_per_launch"] == pytest.approx(24 * N + 16 * 1024 * 1024)
    assert rf["issued_tensor_frac"] == pytest.approx(0.5 * 6 * (8 * 1024 * N / 2e15) / 2e-5)
    q = wl.brusselator_256(precision=wl.BF16X3)  # 256^3, d = 3: HBM-bound
    # fused 3D operators: a fused launch (two products) and an x3 launch per
    # operator, 4 per step: 1.5 products and 16 + 8/2 B per point per launch
    M3 = 256 ** 3
    r3f = bench.mode_product_roofline(q, wl.BF16X3, 0.1, 4, peaks, "test", None)
    assert r3f["mode_products_per_launch"] == pytest.approx(1.5)
    assert r3f["algorithmic_flops_per_launch"] == pytest.approx(1.5 * 4 * 256 * M3)
    assert r3f["algorithmic_bytes_per_launch"] == pytest.approx(20 * M3 + 1.5 * 8 * 256 * 256)
    r3 = bench.mode_product_roofline(q, wl.BF16X3, 0.1, 6, peaks, "test", None)
    assert r3["bound"] == "hbm" and r3["unit"] == "GB/s"
    assert r3["achieved"] == pytest.approx(((16 + 8 / 3) * 256 ** 3 + 8 * 256 * 256) / 1e-4 / 1e9)


@pytest.mark.parametrize("scheme", [wl.ETD2RKDS, wl.LAWSON2B])
def test_oracle_solve_follows_the_scheme(scheme):
    p = wl.fhn_1024(precision=wl.FP64, n=16, nsteps=3).replace(scheme=scheme)
    u0, v0 = wl.initial_data(p)
    plan = schemes.make_plan(p)
    U, V = bench.oracle_solve(plan, p, u0, v0, 3)
    if scheme == wl.LAWSON2B:
        Ur, Vr = u0, v0
        for _ in range(3):
            Ur, Vr = schemes.lawson2b_step(plan, Ur, Vr)
    else:
        Ur, Vr = schemes.etd2rkds_solve(plan, u0, v0, 3)
    assert np.array_equal(U, Ur) and np.array_equal(V, Vr)
