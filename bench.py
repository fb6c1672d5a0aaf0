"""Benchmark of the ETD2RKds hot path on GB300.

Workload (default): the 2D FitzHugh-Nagumo system with advection on a
1024 x 1024 grid, [0,100]^2, D = (1, 20), velocity (0.5, 0.5), eps = 0.05,
a1 = 2, a0 = -0.03, tau = 1e-2, seeded N(0, 0.05^2) data.  One benchmark
step is one whole solve of 500 ETD2RKds time steps from the seeded initial
data, with the state resident in HBM; the metric is point-steps/s (grid
points x time steps, both components advanced) over the timed solves.  L2 is
flushed (256 MB write) between timed solves.

Printed JSON line (rank 0): metric, value, unit, e2e (same metric through
adr_solve with pinned host buffers, copies inside the timed region),
roofline of the dominant kernel, the FP64 oracle timed on the host cores,
the clocks sampled during the timed region and the max relative error of the
timed precision against an FP64 GPU solve of the same data.

Under torchrun each rank runs its own replica of the workload (independent
solves, no collective on the data path): "scaling": "weak".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

PREC = {"fp64": wl.FP64, "fp32": wl.FP32, "tf32x3": wl.TF32X3, "bf16x3": wl.BF16X3}
PREC_NAME = {v: k for k, v in PREC.items()}
DTYPE_NAME = {wl.FP64: "f64", wl.FP32: "f32", wl.TF32X3: "f32 (tf32x3 tensor-core products)",
              wl.BF16X3: "f32 (bf16x3 tensor-core products)"}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def measured_gemm_peak(dtype) -> float:
    """Flop/s of a dense 4096^3 GEMM in `dtype` (torch.matmul, best of 5,
    CUDA events); the roofline denominator of the FP32 / FP64 mode products."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 4096
        a = torch.randn(n, n, dtype=dtype, device="cuda")
        b = torch.randn(n, n, dtype=dtype, device="cuda")
        c = a @ b
        best = float("inf")
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        del a, b, c
        return 2.0 * n ** 3 / best
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def profiled_traffic(workload_name: str, kernel, profiles: str = None):
    """DRAM bytes per launch of the tensor-core mode-product kernel from the
    committed ncu summary, or None when the kernel source has changed since
    that capture or the capture is of another kernel than `kernel` (a
    variant number of the per-direction kernel; "fused" for the fused
    two-mode kernel of 2D grids, or "fused+<variant>" for the two launches
    of a 3D operator, summarised in tc_fused_<workload>.md)."""
    import hashlib
    import re
    stem = "tc_fused" if str(kernel).startswith("fused") else "tc_mode"
    prof = os.path.join(profiles or os.path.join(ROOT, "profiles"), f"{stem}_{workload_name}.md")
    src = os.path.join(ROOT, "paper_2307_10684_gb300", "csrc", "tc.cu")
    try:
        txt = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m_sha = re.search(r"source_sha256\([^)]*\): ([0-9a-f]+)", txt)
        m_b = re.search(r"dram_bytes_per_launch: (\d+)", txt)
        m_k = re.search(r"captured_kernel: (\S+)", txt)
        if m_sha and m_b and m_k and m_sha.group(1) == sha and m_k.group(1) == str(kernel):
            return int(m_b.group(1))
    except OSError:
        pass
    return None


# workload name -> the key of its committed capture summary (profiles/tc_mode_<key>.md)
PROFILE_KEY = {"fhn2d_adv_1024": "fhn1024", "brusselator3d_adv_256": "bruss256"}


def workload(name: str, precision: int):
    if name == "fhn1024":
        return wl.fhn_1024(precision=precision)
    if name == "bruss256":
        return wl.brusselator_256(precision=precision)
    if name == "schnak64":
        return wl.schnakenberg_64(precision=precision)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


SCHEMES = {"etd2rkds": wl.ETD2RKDS, "lawson2b": wl.LAWSON2B}
SCHEME_NAMES = {wl.ETD2RKDS: "ETD2RKds", wl.LAWSON2B: "Lawson2b"}


def oracle_solve(plan, p, u0, v0, nsteps: int):
    """nsteps steps of the oracle in the problem's scheme."""
    from oracle import schemes
    if p.scheme == wl.LAWSON2B:
        for _ in range(nsteps):
            u0, v0 = schemes.lawson2b_step(plan, u0, v0)
        return u0, v0
    return schemes.etd2rkds_solve(plan, u0, v0, nsteps)


def cpu_baseline(p, sample_steps: int):
    """The FP64 oracle (as it stands) timed on the host cores on a bounded
    sample: `sample_steps` steps of the same workload."""
    from oracle import schemes
    cores = len(os.sched_getaffinity(0))
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, p.precision), wl.round_to(v0, p.precision)
    t0 = time.perf_counter()
    plan = schemes.make_plan(p)
    plan_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle_solve(plan, p, u0, v0, sample_steps)
    dt = time.perf_counter() - t0
    return {"value": p.npoints * sample_steps / dt, "unit": "point-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{sample_steps} {SCHEME_NAMES[p.scheme]} steps of the same {p.name} grid, "
                      f"FP64 numpy (plan time {plan_s:.1f} s excluded)"}


class Replicas:
    """The ranks of a torchrun launch, each running its own replica of the
    workload (independent solves, nothing exchanged on the data path).  The
    timed region is bracketed by barriers, its length is the max over ranks
    (the job ends with its slowest replica) and the work is summed over
    ranks.  One process: every reduction returns its argument."""

    def __init__(self, backend: str = "nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if backend == "nccl":
                self.device = torch.device("cuda", self.local)
                dist.init_process_group(backend, device_id=self.device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def sum(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)

    def gather(self, items: list) -> list:
        """Every rank's list, concatenated in rank order."""
        if not self.dist:
            return list(items)
        out = [None] * self.world
        self.dist.all_gather_object(out, list(items))
        return [x for part in out for x in part]

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(units_per_replica: float, world: int, seconds: float) -> float:
    """Units all replicas processed per second of the slowest replica."""
    return world * units_per_replica / seconds


def percentile(sorted_vals: list, q: float) -> float:
    i = min(len(sorted_vals) - 1, max(0, int(round(q * (len(sorted_vals) - 1)))))
    return sorted_vals[i]


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle on this workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = workload(args.workload, PREC[args.precision]).replace(scheme=SCHEMES[args.scheme])
    sample = args.ref_sample
    from oracle import schemes
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, p.precision), wl.round_to(v0, p.precision)
    plan = schemes.make_plan(p)
    for _ in range(args.warmup):
        oracle_solve(plan, p, u0, v0, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(plan, p, u0, v0, sample)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = p.npoints * sample * args.steps / tot
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": "point-steps/s", "value": value,
            "unit": "point-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": p.name, "grid": list(p.n[: p.d]), "tau": p.tau,
                       "scheme": SCHEME_NAMES[p.scheme], "time_steps_per_bench_step": sample},
            "cpu_baseline": {"value": value, "unit": "point-steps/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each bench step = {sample} {SCHEME_NAMES[p.scheme]} "
                                       f"steps of {p.name}"},
            "e2e": {"value": value, "unit": "point-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tc_roofline(kd, prec, peaks, peak_src, traffic):
    """Roofline of the tensor-core mode-product kernel class: the slower of
    (issued MMA flops at the measured dense BF16 peak) and (algorithmic bytes
    at the measured HBM bandwidth)."""
    issue = 3.0 if prec == wl.TF32X3 else 6.0   # MMAs per algorithmic product
    ratio = 0.5 if prec == wl.TF32X3 else 1.0   # tf32 dense rate = 1/2 of bf16
    avg_s = kd["ms"] / kd["count"] / 1e3
    flops = kd["flops"] / kd["count"]
    nbytes = kd["bytes"] / kd["count"]
    tc_peak = peaks["bf16_tflops"] * 1e12 * ratio
    bw = peaks["hbm_gbs"] * 1e9
    t_tensor = issue * flops / tc_peak
    t_hbm = nbytes / bw
    if t_tensor >= t_hbm:
        return {"bound": "tensor", "achieved": issue * flops / avg_s / 1e12,
                "peak": tc_peak / 1e12, "unit": "TFLOP/s", "frac": t_tensor / avg_s,
                "traffic": traffic, "kernel": "mode_product_tc",
                "algorithmic_flops_per_launch": flops, "issued_flops_per_launch": issue * flops,
                "algorithmic_bytes_per_launch": nbytes,
                "frac_algorithmic_flops": flops / avg_s / tc_peak,
                "hbm_frac": t_hbm / avg_s,
                "peak_source": f"{peak_src} dense bf16 (x{ratio}); achieved counts the "
                               f"{int(issue)} split-piece MMAs per product"}
    return {"bound": "hbm", "achieved": nbytes / avg_s / 1e9, "peak": bw / 1e9, "unit": "GB/s",
            "frac": t_hbm / avg_s, "traffic": traffic, "kernel": "mode_product_tc",
            "algorithmic_bytes_per_launch": nbytes, "algorithmic_flops_per_launch": flops,
            "tensor_frac": t_tensor / avg_s,
            "peak_source": f"{peak_src} HBM copy bandwidth"}


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_final(p, nsteps: int):
    """Worker (spawned process): the oracle's final state of the workload
    from the same rounded initial data the GPU solve starts from."""
    from oracle import schemes
    u0, v0 = wl.initial_data(p)
    u0, v0 = wl.round_to(u0, p.precision), wl.round_to(v0, p.precision)
    plan = schemes.make_plan(p)
    t0 = time.perf_counter()
    U, V = oracle_solve(plan, p, u0, v0, nsteps)
    return U, V, time.perf_counter() - t0


class OracleJobs:
    """Whole-horizon oracle solves in one spawned worker process, started
    before any GPU call, with `threads` BLAS threads (the rest of the host
    cores stay with the GPU process)."""

    def __init__(self, jobs, threads: int):
        import concurrent.futures as cf
        import multiprocessing as mp
        saved = {k: os.environ.get(k) for k in THREAD_VARS}
        for k in THREAD_VARS:
            os.environ[k] = str(threads)
        try:
            self.ex = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
            self.futs = [self.ex.submit(_oracle_final, p, n) for p, n in jobs]
            # the worker is spawned now, with the thread counts above
            self.ex.submit(int, 0).result()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.threads = threads

    def result(self, i: int):
        return self.futs[i].result()

    def close(self):
        self.ex.shutdown(wait=True)


def mode_product_roofline(p, prec, ms_launch: float, per_step: int, peaks, peak_src, traffic,
                          computed_share: float = 1.0):
    """Roofline of the tensor-core mode-product launch, timed as it runs
    inside a step (adr_plan_time_mode_products), on the algorithmic work of
    the method per launch.  A step holds two Tucker operators (Eq. 11 or
    Eq. 7); with `per_step` launches each operator takes P = per_step / 2
    launches, so one launch computes d / P mode products (2D grids fuse both
    directions of an operator into one launch):
      flops: 2 flops x n_mu per output x 2 components per product
             = (d / P) x 4 n_mu N (n_mu averaged over the directions)
      bytes: FP32 operand in + out for both components = 16 B per point per
             launch, plus the base (U or U2) the operator's last launch reads:
             16 + 8 / P B per point on average (ETD2RKds).
    The bound is the slower of the two at the measured peaks (dense BF16
    burst, HBM copy); `frac` is the algorithmic fraction.  The split-precision
    form issues 6 (BF16x3) or 3 TF32 (= 6 BF16-rate) MMAs per product it
    computes, and computes `computed_share` of the dense products (tiles
    contract over the column supports of their rows of phi; a fused launch
    recomputes part of its intermediate, adr_plan_mode_product_macs):
    `issued_tensor_frac` counts the MMAs actually issued."""
    d = p.d
    N = float(p.npoints)
    nmu = float(sum(p.n[:d])) / d
    passes = max(1.0, per_step / 2.0)
    products = d / passes
    flops = products * 4.0 * nmu * N
    per_pt = 16.0 + (8.0 / passes if p.scheme == wl.ETD2RKDS else 0.0)
    nbytes = per_pt * N + products * 2.0 * 4.0 * nmu * nmu
    issue = 3.0 if prec == wl.TF32X3 else 6.0
    ratio = 0.5 if prec == wl.TF32X3 else 1.0
    tc_peak = peaks["bf16_tflops"] * 1e12 * ratio
    bw = peaks["hbm_gbs"] * 1e9
    avg_s = ms_launch / 1e3
    t_tc, t_hbm = flops / tc_peak, nbytes / bw
    common = {"kernel": "mode_product_tc", "traffic": traffic,
              "duration_us": 1e6 * avg_s,
              "duration_source": "adr_plan_time_mode_products: the mode-product launches of 64 "
                                 "steps replayed back to back in one CUDA graph (programmatic "
                                 "dependent launch, no timing node between launches)",
              "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
              "mode_products_per_launch": products,
              "tensor_frac_algorithmic": t_tc / avg_s, "hbm_frac_algorithmic": t_hbm / avg_s,
              "issued_tensor_frac": issue * computed_share * t_tc / avg_s,
              "issued_mmas_per_product": int(issue),
              "computed_share_of_dense_products": computed_share,
              "launches_per_time_step": per_step}
    if t_tc >= t_hbm:
        return dict(common, bound="tensor", achieved=flops / avg_s / 1e12, peak=tc_peak / 1e12,
                    unit="TFLOP/s", frac=t_tc / avg_s,
                    peak_source=f"{peak_src} dense bf16 burst (x{ratio})")
    return dict(common, bound="hbm", achieved=nbytes / avg_s / 1e9, peak=bw / 1e9, unit="GB/s",
                frac=t_hbm / avg_s, peak_source=f"{peak_src} HBM copy bandwidth")


def run_single(args, p, nts: int, R, with_compare: bool, oracle):
    """One single-solve workload: timed solves from resident data, e2e
    through adr_solve, roofline, accuracy; returns the JSON fields (rank 0)."""
    import torch
    import paper_2307_10684_gb300 as adr

    world, rank, local = R.world, R.rank, R.local
    prec = p.precision
    dt = adr.state_dtype(prec)
    u0n, v0n = wl.initial_data(p)
    u0 = torch.tensor(wl.round_to(u0n, prec), dtype=dt, device="cuda")
    v0 = torch.tensor(wl.round_to(v0n, prec), dtype=dt, device="cuda")
    u = torch.empty_like(u0)
    v = torch.empty_like(v0)
    stream = torch.cuda.current_stream()

    # kernel choice by the library's autotuner (times each tensor-core kernel
    # on this grid), then the plan
    t0 = time.perf_counter()
    if args.kernel == -2 and prec in (wl.BF16X3, wl.TF32X3):
        kernel, tune_ms = adr.autotune(p)
    else:
        kernel, tune_ms = max(args.kernel, -1), {}
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    plan = adr.Plan(p, kernel=kernel)
    plan_ms = 1e3 * (time.perf_counter() - t0)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def one_solve():
        u.copy_(u0)
        v.copy_(v0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.step(u, v, nts)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    plan.set_timing(False)  # resets the counters; steps replay captured CUDA graphs
    R.barrier()
    torch.cuda.synchronize()
    evs = [one_solve() for _ in range(args.steps)]
    torch.cuda.synchronize()
    R.barrier()
    launches = plan.stats()["launches"]
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = R.max(sum(ms))
    npts = p.npoints
    value = whole_job_rate(npts * nts * args.steps, world, tot_ms / 1e3)
    # the timed state after one solve, for the accuracy fields below
    one_solve()
    torch.cuda.synchronize()
    uf, vf = u.clone(), v.clone()

    # per-kernel shares: the same solves again with each launch bracketed by
    # CUDA events (graph chunks replayed with event-record nodes: no host
    # launch gap is timed, but the kernels are serialised)
    plan.set_timing(True)
    for _ in range(args.steps):
        one_solve()
    torch.cuda.synchronize()
    stats = plan.stats()
    plan.set_timing(False)
    kern = {k: d for k, d in stats["kernels"].items() if d["count"] > 0}
    total_kernel_ms = sum(d["ms"] for d in kern.values())

    # end to end through adr_solve with pinned host buffers
    hu0 = u0.cpu().pin_memory()
    hv0 = v0.cpu().pin_memory()
    huT = torch.empty_like(hu0).pin_memory()
    hvT = torch.empty_like(hv0).pin_memory()
    plan.solve(hu0, hv0, huT, hvT, nts)  # warm
    torch.cuda.synchronize()
    R.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.solve(hu0, hv0, huT, hvT, nts)
    e2e_s = R.max(time.perf_counter() - t0)
    e2e = {"value": whole_job_rate(npts * nts * args.steps, world, e2e_s), "unit": "point-steps/s",
           "h2d_bytes_per_step": int(2 * hu0.numel() * hu0.element_size()),
           "d2h_bytes_per_step": int(2 * huT.numel() * huT.element_size())}

    # roofline of the dominant kernel class
    peaks, peak_src = load_peaks()
    dom = max(kern, key=lambda k: kern[k]["ms"])
    kd = kern[dom]
    in_step = None
    if dom == "mode_product_tc":
        used = kernel if kernel >= 0 else (4 if npts >= 1000000 else 0)  # the plan default
        if prec == wl.BF16X3 and os.environ.get("ADR_TC_FUSED", "1") != "0":
            # 2D operators run as one fused two-mode launch; 3D operators as a
            # fused launch and an x3 launch of kernel `used` (the summary then
            # gives the mean DRAM bytes of the two per launch)
            used = "fused" if p.d == 2 else f"fused+{used}"
        traffic = (profiled_traffic(PROFILE_KEY.get(p.name, p.name), used)
                   if p.scheme == wl.ETD2RKDS and int(getattr(p, "state", 0)) != wl.STATE_COMPENSATED
                   else None)
        ms_launch, per_step = plan.time_mode_products(u, v, reps=64)
        dense_macs, computed_macs = plan.mode_product_macs()
        roof = mode_product_roofline(p, prec, ms_launch, per_step, peaks, peak_src, traffic,
                                     computed_macs / dense_macs)
        roof["share_of_kernel_time"] = kd["ms"] / total_kernel_ms
        step_ms = tot_ms / args.steps / nts
        in_step = {"mode_product_ms_per_time_step": per_step * ms_launch,
                   "time_step_ms": step_ms, "fits": per_step * ms_launch <= step_ms}
    elif dom == "mode_product_simt":
        avg_s = kd["ms"] / kd["count"] / 1e3
        flops = kd["flops"] / kd["count"]
        # the dense GEMM rate in the kernel's type, measured here (the peaks
        # file holds only HBM and BF16): best of 5 torch.matmul at 4096^2
        gdt = torch.float64 if prec == wl.FP64 else torch.float32
        peak = measured_gemm_peak(gdt)
        achieved = flops / avg_s
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": f"measured {'FP64' if prec == wl.FP64 else 'FP32'} dense GEMM "
                               "(torch.matmul 4096^2, best of 5)",
                "duration_source": "event-bracketed launches (serialised)",
                "share_of_kernel_time": kd["ms"] / total_kernel_ms}
    else:
        avg_s = kd["ms"] / kd["count"] / 1e3
        bytes_ = kd["bytes"] / kd["count"]
        achieved = bytes_ / avg_s
        peak = peaks["hbm_gbs"] * 1e9
        roof = {"bound": "hbm", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom}

    # accuracy: against the oracle's whole-horizon solve (rank 0), and
    # against an FP64 GPU solve of the same data
    acc = {}
    if not args.no_check:
        p64 = p.replace(precision=wl.FP64)
        ur = u0.double().clone()
        vr = v0.double().clone()
        with adr.Plan(p64) as plan64:
            plan64.step(ur, vr, nts)
        torch.cuda.synchronize()
        du, mu = adr.max_abs_diff(uf, ur)
        dv, mv = adr.max_abs_diff(vf, vr)
        acc["max_rel_err_vs_fp64_gpu"] = max(du / mu, dv / mv)
        if oracle is not None:
            oj, idx = oracle
            Uo, Vo, osec = oj.result(idx)
            uo = torch.tensor(Uo, dtype=torch.float64, device="cuda")
            vo = torch.tensor(Vo, dtype=torch.float64, device="cuda")
            du, mu = adr.max_abs_diff(uf, uo)
            dv, mv = adr.max_abs_diff(vf, vo)
            acc["max_rel_err_vs_oracle"] = max(du / mu, dv / mv)
            du, mu = adr.max_abs_diff(ur, uo)
            dv, mv = adr.max_abs_diff(vr, vo)
            acc["fp64_gpu_vs_oracle"] = max(du / mu, dv / mv)
            acc["oracle_solve"] = {"steps": nts, "seconds": round(osec, 1),
                                   "threads": oj.threads}

    compare = None
    if with_compare and args.compare and args.compare not in ("none", args.precision):
        cp = PREC[args.compare]
        pc = p.replace(precision=cp)
        cdt = adr.state_dtype(cp)
        cu0 = torch.tensor(wl.round_to(u0n, cp), dtype=cdt, device="cuda")
        cv0 = torch.tensor(wl.round_to(v0n, cp), dtype=cdt, device="cuda")
        cu, cv = torch.empty_like(cu0), torch.empty_like(cv0)
        with adr.Plan(pc) as cplan:
            cms = []
            for k in range(1 + max(1, args.steps // 2)):
                cu.copy_(cu0)
                cv.copy_(cv0)
                flush.fill_(1.0)
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                cplan.step(cu, cv, nts)
                a1.record(stream)
                torch.cuda.synchronize()
                if k > 0:
                    cms.append(a0.elapsed_time(a1))
        compare = {"precision": args.compare, "ms_per_step": float(np.mean(cms)),
                   "value": npts * nts / (float(np.mean(cms)) / 1e3),
                   "speedup_of_headline": (float(np.mean(cms)) / (tot_ms / args.steps))}
        if oracle is not None:
            Uo, Vo, _ = oracle[0].result(oracle[1])
            du, mu = adr.max_abs_diff(cu, torch.tensor(Uo, dtype=torch.float64, device="cuda"))
            dv, mv = adr.max_abs_diff(cv, torch.tensor(Vo, dtype=torch.float64, device="cuda"))
            compare["max_rel_err_vs_oracle"] = max(du / mu, dv / mv)

    # the accurate mode (compensated state, double-float reactions) on the
    # same workload: rate and accuracy
    accurate = None
    if (with_compare and prec in (wl.BF16X3, wl.TF32X3) and p.scheme == wl.ETD2RKDS
            and int(getattr(p, "state", 0)) != wl.STATE_COMPENSATED):
        pc = p.replace(state=wl.STATE_COMPENSATED)
        with adr.Plan(pc, kernel=kernel) as aplan:
            ams = []
            for k in range(1 + max(1, args.steps // 2)):
                u.copy_(u0)
                v.copy_(v0)
                flush.fill_(1.0)
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                aplan.step(u, v, nts)  # a new call on the same buffers: lo restarts below
                a1.record(stream)
                torch.cuda.synchronize()
                aplan.reset_state()
                if k > 0:
                    ams.append(a0.elapsed_time(a1))
        accurate = {"state": "compensated", "ms_per_step": float(np.mean(ams)),
                    "value": npts * nts / (float(np.mean(ams)) / 1e3)}
        if oracle is not None:
            Uo, Vo, _ = oracle[0].result(oracle[1])
            du, mu = adr.max_abs_diff(u, torch.tensor(Uo, dtype=torch.float64, device="cuda"))
            dv, mv = adr.max_abs_diff(v, torch.tensor(Vo, dtype=torch.float64, device="cuda"))
            accurate["max_rel_err_vs_oracle"] = max(du / mu, dv / mv)

    plan.close()
    if rank != 0:
        return None
    state = {0: "auto (plain)", 1: "plain", 2: "compensated"}[int(getattr(p, "state", 0))]
    return {"metric": "point-steps/s", "value": value, "unit": "point-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[prec],
            "data": "synthetic (seeded SplitMix64 data)",
            "config": {"workload": p.name, "grid": list(p.n[: p.d]), "tau": p.tau,
                       "scheme": SCHEME_NAMES[p.scheme], "state": state,
                       "time_steps_per_bench_step": nts, "precision": PREC_NAME[prec],
                       "l2": "flushed between timed solves (256 MB write)",
                       "parallelism": f"replicas x{world}",
                       "kernel": {"chosen": kernel, "by": "adr_autotune" if tune_ms else "--kernel",
                                  "ms_per_step": {str(k): round(t, 4) for k, t in tune_ms.items()},
                                  "tuning_s": round(tune_s, 2)}},
            **acc, "plan_ms": plan_ms,
            "e2e": e2e, "gpu_launches": launches,
            "roofline": roof, "in_step_check": in_step, "clocks": clocks,
            "same_gpu_comparison": compare, "accurate_mode": accurate,
            "kernel_timing": "per-kernel shares from a second pass of the same solves; graph "
                             "chunks replayed with an event-record node before and after every "
                             "kernel (no host launch gaps; kernels serialised)",
            "kernels": {k: {"count": d["count"], "avg_us": 1e3 * d["ms"] / d["count"],
                            "share": d["ms"] / total_kernel_ms} for k, d in kern.items()}}


def run_batch(args):
    """512 independent 2D solves of uneven sizes advanced together by grouped
    launches (one bench step = all solves x 100 ETD2RKds steps)."""
    import torch
    import paper_2307_10684_gb300 as adr

    R = Replicas()
    world, rank, local = R.world, R.rank, R.local
    torch.cuda.set_device(local)
    prec = PREC[args.precision]
    probs = wl.batched_512(precision=prec)
    nts = args.time_steps or probs[0].nsteps
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plans = [adr.Plan(p) for p in probs]
    plan_ms = 1e3 * (time.perf_counter() - t0)
    # one kernel for the whole batch, chosen by timing the batch's grouped
    # launches with each kernel (the plans keep their matrix functions)
    t0 = time.perf_counter()
    if args.kernel == -2:
        kernel, tune_ms = adr.autotune_batch(plans)
    else:
        kernel, tune_ms = args.kernel, {}
        for pl in plans:
            pl.set_kernel(kernel)
    tune_s = time.perf_counter() - t0
    dt = adr.state_dtype(prec)
    init = []
    for p in probs:
        u0, v0 = wl.initial_data(p)
        init.append((torch.tensor(wl.round_to(u0, prec), dtype=dt, device="cuda"),
                     torch.tensor(wl.round_to(v0, prec), dtype=dt, device="cuda")))
    us = [torch.empty_like(a) for a, _ in init]
    vs = [torch.empty_like(b) for _, b in init]
    batch = adr.Batch(plans)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    npts = sum(p.npoints for p in probs)

    def one_solve():
        for (a, b), u, v in zip(init, us, vs):
            u.copy_(a)
            v.copy_(b)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(us, vs, nts)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()
    # accuracy: a sample of solves against FP64 GPU plans of the same data
    max_rel = None
    if not args.no_check:
        max_rel = 0.0
        sample = list(range(0, len(probs), 32))
        for i in sample:
            p64 = probs[i].replace(precision=wl.FP64)
            ur = init[i][0].double().clone()
            vr = init[i][1].double().clone()
            with adr.Plan(p64) as pl:
                pl.step(ur, vr, nts)
            du, mu = adr.max_abs_diff(us[i], ur)
            dv, mv = adr.max_abs_diff(vs[i], vr)
            max_rel = max(max_rel, du / mu, dv / mv)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    batch.set_timing(False)
    R.barrier()
    torch.cuda.synchronize()
    evs = [one_solve() for _ in range(args.steps)]
    torch.cuda.synchronize()
    R.barrier()
    launches = batch.stats()["launches"]
    clocks = sampler.stop()
    tot_ms = R.max(sum(a.elapsed_time(b) for a, b in evs))
    value = whole_job_rate(npts * nts * args.steps, world, tot_ms / 1e3)
    batch.set_timing(True)
    for _ in range(args.steps):
        one_solve()
    torch.cuda.synchronize()
    stats = batch.stats()
    batch.set_timing(False)
    # end to end: pinned host states copied in and out inside the timed region
    hin = [(a.cpu().pin_memory(), b.cpu().pin_memory()) for a, b in init]
    hout = [(torch.empty_like(a), torch.empty_like(b)) for a, b in hin]
    hout = [(a.pin_memory(), b.pin_memory()) for a, b in hout]
    torch.cuda.synchronize()
    R.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for (ha, hb), u, v in zip(hin, us, vs):
            u.copy_(ha, non_blocking=True)
            v.copy_(hb, non_blocking=True)
        batch.step(us, vs, nts)
        for (oa, ob), u, v in zip(hout, us, vs):
            oa.copy_(u, non_blocking=True)
            ob.copy_(v, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = R.max(time.perf_counter() - t0)
    nbytes = sum(a.numel() * a.element_size() * 2 for a, _ in hin)
    e2e = {"value": whole_job_rate(npts * nts * args.steps, world, e2e_s), "unit": "point-steps/s",
           "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes)}
    peaks, peak_src = load_peaks()
    kern = {k: d for k, d in stats["kernels"].items() if d["count"] > 0}
    kd = kern["mode_product_tc"] if "mode_product_tc" in kern else max(kern.values(), key=lambda d: d["ms"])
    roof = tc_roofline(kd, prec, peaks, peak_src, None)
    roof["kernel"] = "mode_product_tc (grouped over 512 solves)"
    roof["share_of_kernel_time"] = kd["ms"] / sum(d["ms"] for d in kern.values())
    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        from oracle import schemes
        cores = len(os.sched_getaffinity(0))
        sample = [probs[i] for i in range(0, len(probs), 64)]
        steps = max(1, args.cpu_sample // 8)
        tot = 0.0
        pts = 0
        for p in sample:
            u0, v0 = wl.initial_data(p)
            plan = schemes.make_plan(p)
            t1 = time.perf_counter()
            schemes.etd2rkds_solve(plan, wl.round_to(u0, prec), wl.round_to(v0, prec), steps)
            tot += time.perf_counter() - t1
            pts += p.npoints * steps
        cpu = {"value": pts / tot, "unit": "point-steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{steps} steps of each of {len(sample)} batch solves (every 64th)"}
    if rank == 0:
        line = {"metric": "point-steps/s", "value": value, "unit": "point-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE_NAME[prec],
                "data": "synthetic (seeded SplitMix64; 512 solves, seeds 1000+i)",
                "config": {"workload": "batched 512 2D solves, sides {64..512}, 100 steps",
                           "points": npts, "time_steps_per_bench_step": nts,
                           "precision": args.precision, "grouped": batch.grouped,
                           "l2": "flushed between timed solves (256 MB write)",
                           "parallelism": f"replicas x{world}",
                           "kernel": {"chosen": kernel, "by": "autotune_batch (whole batch)" if tune_ms else "--kernel",
                                      "ms_per_step": {str(k): round(t, 4) for k, t in tune_ms.items()},
                                      "tuning_s": round(tune_s, 2)}},
                "max_rel_err_vs_fp64": max_rel, "max_rel_err_sample": "every 32nd solve",
                "plan_ms": plan_ms, "e2e": e2e, "gpu_launches": launches,
                "kernel_timing": "second pass of the same solves; the graph chunks are replayed "
                                 "with an event-record node before and after every kernel "
                                 "(no host launch gaps; kernels serialised)",
                "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
                "kernels": {k: {"count": d["count"], "avg_us": 1e3 * d["ms"] / d["count"]}
                            for k, d in kern.items()}}
        print(json.dumps(line), flush=True)
    batch.close()
    for pl in plans:
        pl.close()
    R.close()


def run_serve(args):
    """Poisson request stream (seeded, 200 req/s) of mixed 2D/3D grids and
    models, served with continuous batching; reports p50/p99 latency and the
    served throughput beside the offered load."""
    import torch
    import paper_2307_10684_gb300 as adr
    from paper_2307_10684_gb300.serve import Request, Server

    R = Replicas()
    world, rank, local = R.world, R.rank, R.local
    torch.cuda.set_device(local)
    prec = PREC[args.precision]
    stream_reqs = wl.serving_stream(count=args.requests, rate=args.rate, precision=prec,
                                    seed=5 + rank)

    def make(i, t, p):
        def init(p=p):
            u0, v0 = wl.initial_data(p)
            return (np.asarray(wl.round_to(u0, prec), dtype=np.float32),
                    np.asarray(wl.round_to(v0, prec), dtype=np.float32))
        return Request(i, t, p, init, p.nsteps)

    reqs = [make(i, t, p) for i, (t, p) in enumerate(stream_reqs)]
    # deterministic accuracy sample: every 20th request that is small
    sample = [r.rid for r in reqs if r.rid % 20 == 0 and
              (r.problem.d == 2 and r.problem.npoints <= 256 * 256 or
               r.problem.d == 3 and r.problem.npoints <= 96 ** 3)]
    # warm-up: a few small requests through a throwaway server
    warm = [make(100000 + i, 0.0, wl.fhn_1024(precision=prec, n=64, nsteps=32)) for i in range(3)]
    Server(budget_bytes=2**32).run(warm)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    srv = Server(budget_bytes=int(args.budget_gb * 2**30), keep_ids=sample)
    R.barrier()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    # whole job: every rank serves its own request stream; the served rate is
    # the work of all ranks over the slowest rank's wall time, and the
    # latency percentiles are over all ranks' requests
    served = R.sum(sum(r.npoints * r.nsteps for r in res))
    wall_all = R.max(wall)
    lat = sorted(R.gather([r.latency for r in res if r.nsteps > 0]))
    summ = {"p50_s": percentile(lat, 0.50), "p99_s": percentile(lat, 0.99),
            "mean_s": sum(lat) / len(lat), "max_s": lat[-1],
            "served_point_steps_per_s": served / wall_all}
    offered = R.sum(sum(r.problem.npoints * r.nsteps for r in reqs))
    span = R.max(max(r.arrival for r in reqs))
    wall = wall_all
    # accuracy of the sampled requests against FP64 GPU solves of the same data
    # and the conditioning floor: an FP64 solve from data perturbed by 2^-24
    errs, floors, fp32_errs = [], [], []
    gen = torch.Generator(device="cuda").manual_seed(11)
    for rid in sample:
        req = reqs[rid]
        out = srv.results[rid]
        u0, v0 = req.init()
        ur = torch.tensor(u0, dtype=torch.float64, device="cuda")
        vr = torch.tensor(v0, dtype=torch.float64, device="cuda")
        up = ur * (1 + 2.0**-24 * (2 * torch.rand(ur.shape, generator=gen, device="cuda",
                                                  dtype=torch.float64) - 1))
        vp = vr * (1 + 2.0**-24 * (2 * torch.rand(vr.shape, generator=gen, device="cuda",
                                                  dtype=torch.float64) - 1))
        with adr.Plan(req.problem.replace(precision=wl.FP64)) as pl:
            pl.step(ur, vr, req.nsteps)
            pl.step(up, vp, req.nsteps)
        uf = torch.tensor(u0, dtype=torch.float32, device="cuda")
        vf = torch.tensor(v0, dtype=torch.float32, device="cuda")
        with adr.Plan(req.problem.replace(precision=wl.FP32)) as pl:
            pl.step(uf, vf, req.nsteps)
        au, mu = adr.max_abs_diff(uf, ur)
        av, mv = adr.max_abs_diff(vf, vr)
        fp32_errs.append(max(au / mu, av / mv))
        du, mu = adr.max_abs_diff(out.u.cuda().float().contiguous(), ur)
        dv, mv = adr.max_abs_diff(out.v.cuda().float().contiguous(), vr)
        errs.append(max(du / mu, dv / mv))
        fu, _ = adr.max_abs_diff(up, ur)
        fv, _ = adr.max_abs_diff(vp, vr)
        floors.append(max(fu / mu, fv / mv))
    errs, floors, fp32_errs = R.gather(errs), R.gather(floors), R.gather(fp32_errs)
    if rank == 0:
        line = {"metric": "served point-steps/s; p50/p99 solve latency",
                "value": summ["served_point_steps_per_s"], "unit": "point-steps/s",
                "n_gpus": world, "steps": len(reqs), "warmup": len(warm),
                "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[prec],
                "data": "synthetic Poisson request stream per rank (seed 5 + rank), "
                        "seeded initial data",
                "config": {"workload": f"serving, {len(reqs)} requests per GPU at {args.rate:g}/s, 2D sides "
                                       "128-1024, 3D sides 64-192, 3 models, horizons 50-1000",
                           "budget_gb": args.budget_gb, "chunk_steps": srv.chunk,
                           "planner_threads": srv.planners},
                "latency": {k: summ[k] for k in ("p50_s", "p99_s", "mean_s", "max_s")},
                "offered_point_steps_per_s": offered / span if span > 0 else None,
                "served_point_steps_per_s": summ["served_point_steps_per_s"],
                "wall_s": wall, "arrival_span_s": span,
                "max_rel_err_vs_fp64": max(errs) if errs else None,
                "max_rel_err_sample": f"{len(errs)} requests (every 20th with <=256^2 or <=96^3)",
                "sample_errors": [round(e, 9) for e in errs],
                "sample_fp64_floors": [round(f, 9) for f in floors],
                "sample_plain_fp32_errors": [round(e, 9) for e in fp32_errs],
                "sample_within_1e-5": sum(1 for e in errs if e <= 1e-5),
                "sample_within_2x_plain_fp32": sum(1 for e, f in zip(errs, fp32_errs)
                                                  if e <= max(1e-5, 2 * f)),
                "server_stats": dict(srv.stats), "clocks": clocks,
                "e2e": {"value": summ["served_point_steps_per_s"], "unit": "point-steps/s",
                        "note": "requests enter and leave through host memory"}}
        print(json.dumps(line), flush=True)
    R.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="fhn1024")
    ap.add_argument("--precision", default=None, choices=sorted(PREC),
                    help="default: fp64 for schnak64 (the plain-method FP64 workload), else bf16x3")
    ap.add_argument("--compare", default="fp32",
                    help="also time this precision on the same workload ('none' to skip)")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="ETD2RKds steps per bench step (default: the workload's)")
    ap.add_argument("--no-check", action="store_true", help="skip the accuracy solves")
    ap.add_argument("--oracle-check", type=int, default=1,
                    help="1: accuracy against the oracle's whole-horizon solve (spawned process)")
    ap.add_argument("--oracle-threads", type=int, default=12,
                    help="BLAS threads of the oracle process (the rest stay with the GPU process)")
    ap.add_argument("--secondary", default="bruss256",
                    help="with the default fhn1024 workload, also measure this single-solve "
                         "workload and report it under secondary_workload ('none' to skip)")
    ap.add_argument("--scheme", default="etd2rkds", choices=sorted(SCHEMES),
                    help="time-stepping scheme of the single-solve workloads (fhn1024, "
                         "bruss256, schnak64)")
    ap.add_argument("--kernel", type=int, default=-2, choices=[-2, -1, 0, 1, 2, 3, 4],
                    help="tensor-core kernel: -2 autotune (default), -1 plan default, 0..4 fixed")
    ap.add_argument("--cpu-sample", type=int, default=40)
    ap.add_argument("--ref-sample", type=int, default=20)
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: requests per GPU")
    ap.add_argument("--rate", type=float, default=200.0,
                    help="serving workload: mean Poisson arrival rate (requests/s)")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serving: device-memory budget")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "schnak64" else "bf16x3"

    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload == "batch512":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return

    import torch

    R = Replicas()
    world, rank, local = R.world, R.rank, R.local
    prec = PREC[args.precision]
    p = workload(args.workload, prec).replace(scheme=SCHEMES[args.scheme])
    nts = args.time_steps or p.nsteps
    # the oracle's solves of the timed workloads, for the accuracy fields: a
    # spawned process (rank 0, one replica) running while the GPU works
    second = None
    if args.workload == "fhn1024" and args.secondary != "none":
        second = workload(args.secondary, prec).replace(scheme=SCHEMES[args.scheme])
    jobs = []
    if rank == 0 and not args.no_check and args.oracle_check:
        jobs.append((p, nts))
        if second is not None:
            jobs.append((second, second.nsteps))
    oj = OracleJobs(jobs, threads=args.oracle_threads) if jobs else None
    torch.cuda.set_device(local)
    line = run_single(args, p, nts, R, with_compare=True, oracle=(oj, 0) if oj else None)
    if second is not None:
        sub = run_single(args, second, second.nsteps, R, with_compare=False,
                         oracle=(oj, 1) if oj and len(jobs) > 1 else None)
        if line is not None and sub is not None:
            for k in ("n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline",
                      "cpu_baseline"):
                sub.pop(k, None)
            line["secondary_workload"] = sub
    if oj:
        oj.close()
    if rank == 0 and line is not None and world == 1 and args.cpu_sample > 0:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_sample)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    R.close()


if __name__ == "__main__":
    main()
