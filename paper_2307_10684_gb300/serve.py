"""Continuous-batching server for ETD2RKds solves on one GPU.

Requests (an ADR problem plus its initial data and horizon) arrive over time.
The server:

* admits a waiting request when its plan and state fit in the device-memory
  budget (sizes from ``adr_plan_bytes``), building the plan (FP64 matrix
  functions on the GPU) on a planner thread, so that stepping continues
  meanwhile;
* keeps every admitted solve's state and matrices resident, and each tick
  advances all active solves of a dimension in one grouped batch call
  (``adr_batch_step``), each by ``chunk`` steps or what it has left;
* retires finished solves without stalling the stepping loop: the results
  are copied to page-locked host memory asynchronously, and a request is
  complete when its copy event has fired (its latency is that moment minus
  its arrival); plans are destroyed on a separate thread, because freeing
  device memory synchronises the device.

PyTorch supplies device memory, streams and events; every step runs in the
library's kernels through the C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

from . import BF16X3, ETD2RKDS, STATE_AUTO, STATE_COMPENSATED, TF32X3, Batch, Plan, plan_bytes, \
    state_dtype


def served_problem(p):
    """The problem as the server plans it.  A solve advances in ticks (one
    call per tick), so a tensor-core ETD2RKds solve carries its compensated
    state across calls (ADR_STATE_COMPENSATED): the server owns the state
    buffers for the solve's whole life and writes nothing into them between
    ticks, which is the condition that mode asks of its caller."""
    if (getattr(p, "state", STATE_AUTO) == STATE_AUTO and int(p.precision) in (BF16X3, TF32X3)
            and int(getattr(p, "scheme", ETD2RKDS)) == ETD2RKDS):
        return dataclasses.replace(p, state=STATE_COMPENSATED)
    return p


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds after the start of the run
    problem: object           # adr_problem fields (workloads.Problem)
    init: Callable            # () -> (u0, v0) host arrays of the problem's shape
    nsteps: int


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    nsteps: int
    npoints: int
    u: object = None          # host tensors (when keep_results)
    v: object = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Slot:
    def __init__(self, req: Request, plan: Plan, u, v, admitted: float, nbytes: int):
        self.req = req
        self.plan = plan
        self.u = u
        self.v = v
        self.admitted = admitted
        self.left = req.nsteps
        self.nbytes = nbytes


class Server:
    """One-GPU continuous-batching ETD2RKds server.

    budget_bytes: device memory the server may hold for plans and states.
    chunk: steps per tick for batched solves (32 = one captured graph chunk).
    planners: threads that build plans (FP64 matrix functions) concurrently.
    """

    def __init__(self, budget_bytes: int, chunk: int = 32, max_active: int = 1024,
                 keep_results: bool = False, keep_ids=None, planners: int = 3):
        import torch
        self.device = torch.cuda.current_device()
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.planners = max(1, int(planners))
        self.max_active = int(max_active)
        self.keep = keep_results
        self.keep_ids = set(keep_ids or ())
        self.stream = torch.cuda.current_stream()
        self.used = 0
        self.active: List[_Slot] = []
        self.results: Dict[int, Result] = {}
        self.stats = collections.Counter()

    # ---------------------------------------------------------------- planner
    def _planner(self, inq: "queue.Queue", outq: "queue.Queue"):
        import torch
        torch.cuda.set_device(self.device)
        pstream = torch.cuda.Stream()
        while True:
            item = inq.get()
            if item is None:
                return
            req, nbytes = item
            try:
                with torch.cuda.stream(pstream):
                    plan = Plan(served_problem(req.problem), stream=pstream)
                dt = state_dtype(plan.precision)
                u0, v0 = req.init()
                hu = torch.as_tensor(u0, dtype=dt).pin_memory()
                hv = torch.as_tensor(v0, dtype=dt).pin_memory()
                outq.put((req, plan, nbytes, (hu, hv), None))
            except Exception as exc:  # reported, request dropped
                outq.put((req, None, nbytes, None, exc))

    # ---------------------------------------------------------------- reaper
    @staticmethod
    def _reaper(q: "queue.Queue"):
        while True:
            item = q.get()
            if item is None:
                return
            try:
                item.close()
            except Exception:  # a failed teardown must not stop the server
                pass

    # ---------------------------------------------------------------- run
    def run(self, requests: Sequence[Request], clock: Optional[Callable[[], float]] = None):
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        arrivals = collections.deque(reqs)
        waiting: "collections.deque[Tuple[Request, int]]" = collections.deque()
        inq: "queue.Queue" = queue.Queue()
        outq: "queue.Queue" = queue.Queue()
        planners = [threading.Thread(target=self._planner, args=(inq, outq), daemon=True)
                    for _ in range(self.planners)]
        for th in planners:
            th.start()
        reapq: "queue.Queue" = queue.Queue()
        reaper = threading.Thread(target=self._reaper, args=(reapq,), daemon=True)
        reaper.start()
        retiring: List[Tuple[_Slot, object, object, object]] = []  # (slot, event, host u, host v)
        t0 = time.perf_counter()
        now = clock or (lambda: time.perf_counter() - t0)
        in_planning = 0
        batches: Dict[int, Tuple[Tuple[int, ...], Batch]] = {}
        total = len(reqs)
        while len(self.results) < total:
            t = now()
            # solves whose result copies have landed are complete
            if retiring:
                still = []
                for s, ev, hu, hv in retiring:
                    if not ev.query():
                        still.append((s, ev, hu, hv))
                        continue
                    res = Result(s.req.rid, s.req.arrival, s.admitted, now(), s.req.nsteps,
                                 int(s.u.numel()))
                    if hu is not None:
                        res.u, res.v = hu, hv
                    self.results[s.req.rid] = res
                    self.used -= s.nbytes   # its memory goes back once the reaper frees it
                    reapq.put(s.plan)
                retiring = still
            # arrivals join the waiting queue with their memory demand
            while arrivals and arrivals[0].arrival <= t:
                r = arrivals.popleft()
                sb, cb = plan_bytes(served_problem(r.problem))
                waiting.append((r, sb + cb))
            # admission by memory budget, in arrival order
            while waiting and len(self.active) + in_planning < self.max_active:
                r, nbytes = waiting[0]
                if self.used + nbytes > self.budget and (self.active or in_planning):
                    self.stats["admission_deferred"] += 1
                    break
                waiting.popleft()
                self.used += nbytes
                inq.put((r, nbytes))
                in_planning += 1
            # plans that are ready become active slots
            changed = False
            while True:
                try:
                    r, plan, nbytes, host, exc = outq.get_nowait()
                except queue.Empty:
                    break
                in_planning -= 1
                if exc is not None:
                    self.used -= nbytes
                    self.stats["plan_failed"] += 1
                    self.results[r.rid] = Result(r.rid, r.arrival, now(), now(), 0, 0)
                    continue
                plan.set_stream(self.stream)   # all stepping on the server's stream
                u = host[0].to("cuda", non_blocking=True)
                v = host[1].to("cuda", non_blocking=True)
                self.active.append(_Slot(r, plan, u, v, now(), nbytes))
                changed = True
            if not self.active:
                if in_planning == 0 and not waiting and arrivals and not retiring:
                    time.sleep(max(0.0, min(0.002, arrivals[0].arrival - now())))
                else:
                    time.sleep(0.0005)
                continue
            # one tick: every active solve of a dimension in one batch call,
            # each advancing min(chunk, its steps left); a solve whose horizon
            # ends inside the tick drops out of the grouped work there
            groups: Dict[int, List[_Slot]] = collections.defaultdict(list)
            for s in self.active:
                groups[s.req.problem.d].append(s)
            for d, slots in groups.items():
                steps = [min(self.chunk, s.left) for s in slots]
                if len(slots) == 1:  # a group of one steps its plan (and its graph) directly
                    s = slots[0]
                    s.plan.step(s.u, s.v, steps[0])
                    s.left -= steps[0]
                    self.stats["single_ticks"] += 1
                    continue
                key = tuple(id(s) for s in slots)
                if d not in batches or batches[d][0] != key:
                    if d in batches:
                        batches[d][1].close()
                    batches[d] = (key, Batch([s.plan for s in slots]))
                    self.stats["batch_rebuilds"] += 1
                batches[d][1].step([s.u for s in slots], [s.v for s in slots], steps)
                for s, n in zip(slots, steps):
                    s.left -= n
                    if n < self.chunk:
                        self.stats["tail_steps"] += n
                self.stats["ticks"] += 1
            # retire finished solves: copy results out asynchronously
            done = [s for s in self.active if s.left == 0]
            for s in done:
                hu = hv = None
                if self.keep or s.req.rid in self.keep_ids:
                    hu = torch.empty(s.u.shape, dtype=s.u.dtype, pin_memory=True)
                    hv = torch.empty(s.v.shape, dtype=s.v.dtype, pin_memory=True)
                    hu.copy_(s.u, non_blocking=True)
                    hv.copy_(s.v, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(self.stream)
                retiring.append((s, ev, hu, hv))
                self.active.remove(s)
                for d in list(batches):
                    if any(id(s) == k for k in batches[d][0]):
                        batches[d][1].close()   # stream-ordered; does not synchronise
                        del batches[d]
        for _ in planners:
            inq.put(None)
        for th in planners:
            th.join(timeout=10)
        for _, b in batches.values():
            b.close()
        reapq.put(None)
        reaper.join(timeout=60)
        return [self.results[r.rid] for r in reqs]


def latency_summary(results: Sequence[Result], wall_s: float) -> dict:
    lat = sorted(r.latency for r in results if r.nsteps > 0)
    if not lat:
        return {}

    def pct(q):
        i = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[i]

    served = sum(r.npoints * r.nsteps for r in results)
    return {"requests": len(results), "p50_s": pct(0.50), "p99_s": pct(0.99),
            "mean_s": sum(lat) / len(lat), "max_s": lat[-1], "wall_s": wall_s,
            "served_point_steps_per_s": served / wall_s}
