"""Python binding of libadr_gb300 (the C ABI declared in include/adr.h).

Argument marshalling only: every step of the ETD2RKds path runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  The
binding raises if the compiled library is missing; there is no fallback.

Usage::

    import paper_2307_10684_gb300 as adr
    plan = adr.Plan(problem)          # problem: any object with the adr_problem fields
    plan.step(u, v, nsteps)           # u, v: contiguous CUDA tensors, updated in place
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from . import _abi
from ._abi import (ADR_OK, ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA, ADR_EUNSUPPORTED,  # noqa: F401
                   ADR_ETIMEOUT, ADR_ENUMERIC, ADR_EBUSY, FP64, FP32, TF32X3, BF16X3,
                   SCHNAKENBERG, FHN, BRUSSELATOR, NO_REACTION, FHN_RHO, DIB, ETD2RKDS,
                   LAWSON2B, STATE_AUTO, STATE_PLAIN, STATE_COMPENSATED, AdrError, lib,
                   library_path)

__all__ = ["Plan", "Batch", "GeneralPlan", "AdrError", "lib", "library_path", "plan_bytes", "max_abs_diff",
           "make_problem", "state_dtype"]


def make_problem(p) -> _abi.AdrProblem:
    """adr_problem from an object with fields d, n, lo, hi, diff, adv, model,
    params, tau, precision (e.g. workloads.Problem)."""
    s = _abi.AdrProblem()
    s.d = int(p.d)
    s.model = int(p.model)
    s.precision = int(p.precision)
    s.scheme = int(getattr(p, "scheme", 0))
    def at(seq, i, default):
        return seq[i] if i < min(len(seq), max(int(p.d), 0)) else default

    for m in range(3):
        s.n[m] = int(at(p.n, m, 1))
        s.lo[m] = float(at(p.lo, m, 0.0))
        s.hi[m] = float(at(p.hi, m, 1.0))
    for c in range(2):
        s.diff[c] = float(p.diff[c])
        for m in range(3):
            s.adv[c][m] = float(at(p.adv[c], m, 0.0))
    if len(p.params) > 16:
        raise ValueError("at most 16 model parameters")
    for i in range(16):
        s.params[i] = float(p.params[i]) if i < len(p.params) else 0.0
    s.tau = float(p.tau)
    s.state = int(getattr(p, "state", 0))
    return s


def state_dtype(precision: int):
    import torch
    return torch.float64 if precision == FP64 else torch.float32


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """An adr_plan: FP64 matrix functions on the GPU, operands, workspace."""

    def __init__(self, problem, stream=None, kernel: int = -1):
        """kernel: tensor-core kernel variant (adr_tuning.kernel; -1 = the
        library's choice from the grid size, see autotune)."""
        self.problem = problem
        self.precision = int(problem.precision)
        self.shape = tuple(reversed([int(x) for x in problem.n[: problem.d]]))
        self._stream = stream
        self._p = _abi.AdrPlan()
        self._cprob = make_problem(problem)
        tuning = _abi.AdrTuning()
        tuning.kernel = int(kernel)
        _abi.check(lib().adr_plan_create_tuned(ctypes.byref(self._cprob), ctypes.byref(tuning),
                                               ctypes.c_void_p(_stream_handle(stream)),
                                               ctypes.byref(self._p)))

    def set_kernel(self, kernel: int):
        """adr_plan_set_kernel: switch the tensor-core kernel (see autotune)
        keeping the plan's matrix functions."""
        _abi.check(lib().adr_plan_set_kernel(self._p, int(kernel)))

    def set_stream(self, stream=None):
        """adr_plan_set_stream: later calls enqueue on `stream` (default: current)."""
        self._stream = stream
        _abi.check(lib().adr_plan_set_stream(self._p, ctypes.c_void_p(_stream_handle(stream))))

    def close(self):
        """adr_plan_destroy; raises (and keeps the plan) while a live Batch
        uses it."""
        if self._p:
            _abi.check(lib().adr_plan_destroy(self._p))
            self._p = _abi.AdrPlan()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check_state(self, x, device: bool):
        import torch
        if not isinstance(x, torch.Tensor):
            raise TypeError("state must be a torch.Tensor")
        if x.dtype != state_dtype(self.precision):
            raise TypeError(f"state dtype must be {state_dtype(self.precision)}")
        if not x.is_contiguous() or x.numel() != _abi.prod(self.shape):
            raise ValueError(f"state must be contiguous with {_abi.prod(self.shape)} elements")
        if device and not x.is_cuda:
            raise ValueError("state must be a CUDA tensor")

    def step(self, u, v, nsteps: int = 1):
        """adr_step: advance CUDA tensors u, v in place (asynchronous)."""
        self._check_state(u, True)
        self._check_state(v, True)
        _abi.check(lib().adr_step(self._p, ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(v.data_ptr()), ctypes.c_int64(int(nsteps))))

    def time_mode_products(self, u, v, reps: int = 32):
        """adr_plan_time_mode_products: (ms per mode-product launch inside a
        step, launches per step); u, v are scratch tensors (overwritten)."""
        self._check_state(u, True)
        self._check_state(v, True)
        ms = ctypes.c_double()
        n = ctypes.c_int32()
        _abi.check(lib().adr_plan_time_mode_products(self._p, ctypes.c_void_p(u.data_ptr()),
                                                     ctypes.c_void_p(v.data_ptr()), int(reps),
                                                     ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def mode_product_macs(self):
        """adr_plan_mode_product_macs: (dense, computed) multiply-adds of
        one step's mode products."""
        dense = ctypes.c_double()
        computed = ctypes.c_double()
        _abi.check(lib().adr_plan_mode_product_macs(self._p, ctypes.byref(dense),
                                                    ctypes.byref(computed)))
        return float(dense.value), float(computed.value)

    def set_indicators(self, enable: bool = True):
        """adr_plan_set_indicators: per-step indicators of Sec. 4 fused into
        the last product of every step."""
        _abi.check(lib().adr_plan_set_indicators(self._p, 1 if enable else 0))

    def indicator_log(self, max_steps: int = 4096):
        """adr_plan_indicator_log: numpy [steps, 4] of (<U>, <V>, ||dU||_F,
        ||dV||_F), oldest step first."""
        import numpy as np
        out = np.zeros((max(int(max_steps), 1), 4), dtype=np.float64)
        n = ctypes.c_int64()
        _abi.check(lib().adr_plan_indicator_log(
            self._p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_steps),
            ctypes.byref(n)))
        return out[: n.value].copy()

    def run(self, u, v, t_end: float, tol: float = 0.0, check_every: int = 32):
        """adr_run: step until t_end or until the increment indicator <= tol;
        returns (steps taken, indicators of the last step)."""
        self._check_state(u, True)
        self._check_state(v, True)
        steps = ctypes.c_int64()
        last = (ctypes.c_double * 4)()
        _abi.check(lib().adr_run(self._p, ctypes.c_void_p(u.data_ptr()),
                                 ctypes.c_void_p(v.data_ptr()), float(t_end), float(tol),
                                 int(check_every), ctypes.byref(steps), last))
        return int(steps.value), [float(x) for x in last]

    def reset_state(self):
        """adr_plan_reset_state: restart the compensated state's low-order
        words (after writing new values into buffers already stepped)."""
        _abi.check(lib().adr_plan_reset_state(self._p))

    def solve(self, u0, v0, uT, vT, nsteps: int):
        """adr_solve: tensors may live on the host (pinned) or the device."""
        for x in (u0, v0, uT, vT):
            self._check_state(x, False)
        _abi.check(lib().adr_solve(self._p, ctypes.c_void_p(u0.data_ptr()),
                                   ctypes.c_void_p(v0.data_ptr()), ctypes.c_void_p(uT.data_ptr()),
                                   ctypes.c_void_p(vT.data_ptr()), ctypes.c_int64(int(nsteps))))

    def matrix(self, which: int, component: int, mu: int):
        """FP64 plan matrix (0 = A, 1 = e^(tau A), 2 = phi_1, 3 = phi_2) as numpy."""
        import numpy as np
        n = int(self.problem.n[mu])
        out = np.empty((n, n), dtype=np.float64)
        _abi.check(lib().adr_plan_matrix(self._p, int(which), int(component), int(mu),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def indicators(self, u_prev, v_prev, u, v):
        """adr_indicators: (<U>, <V>, ||U - U_prev||_F, ||V - V_prev||_F)."""
        for x in (u_prev, v_prev, u, v):
            self._check_state(x, True)
        out = (ctypes.c_double * 4)()
        _abi.check(lib().adr_indicators(self._p, ctypes.c_void_p(u_prev.data_ptr()),
                                        ctypes.c_void_p(v_prev.data_ptr()),
                                        ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(v.data_ptr()), out))
        return tuple(float(x) for x in out)

    def set_timing(self, enable: bool):
        _abi.check(lib().adr_plan_set_timing(self._p, 1 if enable else 0))

    def stats(self) -> dict:
        st = _abi.AdrStats()
        _abi.check(lib().adr_plan_stats(self._p, ctypes.byref(st)))
        return _stats_dict(st)


class GeneralPlan:
    """adr_plan_create_general: m = 1..4 components, dense directional
    matrices A[c][mu] (numpy n_mu x n_mu), polynomial reaction terms
    (comp, exponents, coef) each adding coef * prod_j u_j^e_j to g^comp."""

    def __init__(self, A, terms, tau: float, precision: int = FP64, stream=None):
        import numpy as np
        self.m = len(A)
        self.d = len(A[0])
        self.n = [int(A[0][mu].shape[0]) for mu in range(self.d)]
        self.shape = tuple(reversed(self.n))
        self.precision = int(precision)
        gp = _abi.AdrGeneralProblem()
        gp.d, gp.m, gp.precision, gp.nterms = self.d, self.m, self.precision, len(terms)
        for mu in range(3):
            gp.n[mu] = self.n[mu] if mu < self.d else 1
        keep = []
        for c in range(self.m):
            for mu in range(self.d):
                a = np.ascontiguousarray(A[c][mu], dtype=np.float64)
                if a.shape != (self.n[mu], self.n[mu]):
                    raise ValueError("A[c][mu] must be n_mu x n_mu for every component")
                keep.append(a)
                gp.A[c][mu] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        T = (_abi.AdrTerm * max(1, len(terms)))()
        for i, (c, exps, coef) in enumerate(terms):
            T[i].comp = int(c)
            for j in range(4):
                T[i].pow[j] = int(exps[j]) if j < len(exps) else 0
            T[i].coef = float(coef)
        gp.terms = ctypes.cast(T, ctypes.POINTER(_abi.AdrTerm))
        gp.tau = float(tau)
        self._p = _abi.AdrPlan()
        _abi.check(lib().adr_plan_create_general(ctypes.byref(gp),
                                                 ctypes.c_void_p(_stream_handle(stream)),
                                                 ctypes.byref(self._p)))

    def step(self, states, nsteps: int = 1):
        """adr_step_general: advance the m CUDA tensors in place."""
        import torch
        dt = state_dtype(self.precision)
        if len(states) != self.m:
            raise ValueError("one state tensor per component")
        for x in states:
            if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == dt and
                    x.is_contiguous() and tuple(x.shape) == self.shape):
                raise ValueError(f"states must be contiguous CUDA {dt} tensors of shape {self.shape}")
        S = (ctypes.c_void_p * self.m)(*[x.data_ptr() for x in states])
        _abi.check(lib().adr_step_general(self._p, S, ctypes.c_int64(int(nsteps))))

    def matrix(self, which: int, component: int, mu: int):
        import numpy as np
        n = self.n[mu]
        out = np.empty((n, n), dtype=np.float64)
        _abi.check(lib().adr_plan_matrix(self._p, int(which), int(component), int(mu),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def close(self):
        if self._p:
            _abi.check(lib().adr_plan_destroy(self._p))
            self._p = _abi.AdrPlan()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _stats_dict(st) -> dict:
    kernels = {}
    for k in range(st.nkernels):
        kernels[st.name[k].value.decode()] = {
            "count": int(st.count[k]), "ms": float(st.ms[k]),
            "flops": float(st.flops[k]), "bytes": float(st.bytes[k])}
    return {"launches": int(st.launches), "steps": int(st.steps), "timing": bool(st.timing),
            "device_error": int(st.device_error), "shared_matrices": int(st.shared_matrices),
            "kernels": kernels}


_tuned = {}


def autotune(problem, nsteps: int = 32, stream=None, cache: bool = True):
    """adr_autotune: time every tensor-core kernel variant on this problem's
    grid (scratch state, nsteps steps each) and return (best kernel, {kernel:
    ms per step}).  Results are cached per (d, grid, precision, scheme) in
    this process.  FP32 / FP64 problems return (-1, {})."""
    key = (int(problem.d), tuple(int(x) for x in problem.n[: problem.d]),
           int(problem.precision), int(getattr(problem, "scheme", 0)))
    if cache and key in _tuned:
        return _tuned[key]
    cp = make_problem(problem)
    best = _abi.AdrTuning()
    ms = (ctypes.c_float * 8)()
    _abi.check(lib().adr_autotune(ctypes.byref(cp), ctypes.c_void_p(_stream_handle(stream)),
                                  int(nsteps), ctypes.byref(best), ms))
    out = (int(best.kernel), {k: float(ms[k]) for k in range(8) if ms[k] >= 0})
    if cache:
        _tuned[key] = out
    return out


def selftest_bounded_wait(arrive: bool, limit_ns: int = 20_000_000, stream=None):
    """adr_selftest_bounded_wait: (device error code, ns waited) of one
    bounded mbarrier wait that is (arrive=True) or is not satisfied."""
    code = ctypes.c_int32()
    waited = ctypes.c_int64()
    _abi.check(lib().adr_selftest_bounded_wait(ctypes.c_void_p(_stream_handle(stream)),
                                               1 if arrive else 0, ctypes.c_int64(int(limit_ns)),
                                               ctypes.byref(code), ctypes.byref(waited)))
    return int(code.value), int(waited.value)


def autotune_batch(plans, nsteps: int = 8, stream=None):
    """Kernel choice for a batch: every tensor-core kernel is timed on the
    grouped launches of the whole batch (its plans switched with
    adr_plan_set_kernel, zero-filled scratch states, two warm-up steps, then
    nsteps timed with CUDA events); the plans are left on the fastest kernel,
    which is returned with {kernel: ms per step}."""
    import torch
    plans = list(plans)
    if not plans or plans[0].precision not in (BF16X3, TF32X3):
        return -1, {}
    cands = [1] if plans[0].precision == TF32X3 else [0, 1, 2, 3, 4]
    st = torch.cuda.current_stream() if stream is None else stream
    us = [torch.zeros(pl.shape, dtype=torch.float32, device="cuda") for pl in plans]
    vs = [torch.zeros(pl.shape, dtype=torch.float32, device="cuda") for pl in plans]
    times = {}
    for k in cands:
        for pl in plans:
            pl.set_kernel(k)
        b = Batch(plans, stream=st)
        b.step(us, vs, 2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.step(us, vs, nsteps)
        e1.record(st)
        e1.synchronize()
        times[k] = e0.elapsed_time(e1) / nsteps
        b.close()
    best = min(times, key=times.get)
    for pl in plans:
        pl.set_kernel(best)
    return best, times


class Batch:
    """An adr_batch over existing plans (kept alive by this object)."""

    def __init__(self, plans, stream=None):
        self.plans = list(plans)
        arr = (_abi.AdrPlan * len(self.plans))(*[p._p for p in self.plans])
        self._b = ctypes.c_void_p()
        _abi.check(lib().adr_batch_create(arr, len(self.plans),
                                          ctypes.c_void_p(_stream_handle(stream)),
                                          ctypes.byref(self._b)))

    @property
    def grouped(self) -> bool:
        return bool(lib().adr_batch_is_grouped(self._b))

    def step(self, us, vs, nsteps=1):
        """Advance every solve i's CUDA tensors (us[i], vs[i]) in place by
        nsteps[i] steps (one int: the same for every solve)."""
        if len(us) != len(self.plans) or len(vs) != len(self.plans):
            raise ValueError("one (u, v) pair per plan")
        for p, u, v in zip(self.plans, us, vs):
            p._check_state(u, True)
            p._check_state(v, True)
        ns = ([int(n) for n in nsteps] if hasattr(nsteps, "__len__")
              else [int(nsteps)] * len(us))
        if len(ns) != len(us):
            raise ValueError("one horizon per plan")
        U = (ctypes.c_void_p * len(us))(*[u.data_ptr() for u in us])
        V = (ctypes.c_void_p * len(vs))(*[v.data_ptr() for v in vs])
        H = (ctypes.c_int64 * len(ns))(*ns)
        _abi.check(lib().adr_batch_step(self._b, U, V, H))

    def set_timing(self, enable: bool):
        _abi.check(lib().adr_batch_set_timing(self._b, 1 if enable else 0))

    def stats(self) -> dict:
        st = _abi.AdrStats()
        _abi.check(lib().adr_batch_stats(self._b, ctypes.byref(st)))
        return _stats_dict(st)

    def close(self):
        if self._b:
            lib().adr_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def plan_bytes(problem):
    s = make_problem(problem)
    sb = ctypes.c_size_t()
    cb = ctypes.c_size_t()
    _abi.check(lib().adr_plan_bytes(ctypes.byref(s), ctypes.byref(sb), ctypes.byref(cb)))
    return int(sb.value), int(cb.value)


def max_abs_diff(x, ref, stream=None):
    """(max |x - ref|, max |ref|) on the GPU in FP64; ref must be float64."""
    import torch
    if ref.dtype != torch.float64 or not ref.is_cuda or not x.is_cuda:
        raise TypeError("x, ref must be CUDA tensors, ref float64")
    if x.numel() != ref.numel() or not x.is_contiguous() or not ref.is_contiguous():
        raise ValueError("size / contiguity mismatch")
    out = (ctypes.c_double * 2)()
    _abi.check(lib().adr_max_abs_diff(ctypes.c_void_p(_stream_handle(stream)),
                                      ctypes.c_void_p(x.data_ptr()),
                                      1 if x.dtype == torch.float64 else 0,
                                      ctypes.c_void_p(ref.data_ptr()),
                                      ctypes.c_int64(x.numel()), out))
    return float(out[0]), float(out[1])
