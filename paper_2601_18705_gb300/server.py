"""Continuous-batching server for SN-like DLR solves.

Requests (a TRT problem and a number of time steps) arrive over time.  The
server admits a request when a slot is free and its device footprint fits the
HBM budget, keeps every admitted request's state (X, S, W, T) resident on the
GPU between steps, and advances all admitted requests together: one batched
DLR step (one launch per kernel for the whole batch, one persistent
source-iteration launch) per tick.  Requests that arrive while others run
join at the next tick; a request leaves as soon as its last step is done, and
its memory is freed for the queue.  Latency = completion - arrival.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import DLR_MIXED, DlrError, Solver, footprint_bytes, problem_from_case, step_batch


@dataclass
class Request:
    rid: int
    arrival: float               # seconds after the start of the run
    case: dict                   # workloads case dict
    steps: int
    precision: int = DLR_MIXED
    spec: object = None
    footprint: int = 0
    solver: Solver = None
    admitted: float = None
    done_steps: int = 0
    finished: float = None
    result_T: np.ndarray = None


@dataclass
class ServeReport:
    latencies: list = field(default_factory=list)
    steps_total: int = 0
    updates_total: int = 0
    wall: float = 0.0
    ticks: int = 0
    max_active: int = 0
    admission_waits: int = 0
    peak_bytes: int = 0
    failures: list = field(default_factory=list)  # (request id, step, status)

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "steps_per_s": self.steps_total / self.wall,
                "cell_angle_updates_per_s": self.updates_total / self.wall,
                "wall_s": self.wall, "ticks": self.ticks, "max_active": self.max_active,
                "admission_waits": self.admission_waits, "peak_bytes": self.peak_bytes,
                "failed": len(self.failures),
                "failures": [list(f) for f in self.failures]}


class Server:
    """max_active: slots; hbm_budget: bytes of device state the admitted
    requests may hold together (0 = unlimited); keep_results: copy each
    request's final temperature to the host."""

    def __init__(self, *, max_active: int = 32, hbm_budget: int = 0, keep_results: bool = False,
                 stream=None, clock=time.perf_counter):
        import torch
        self.max_active = max_active
        self.hbm_budget = hbm_budget
        self.keep_results = keep_results
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.clock = clock

    def run(self, requests, *, realtime: bool = True) -> ServeReport:
        """Serves `requests` (sorted by arrival).  With realtime=False the
        arrival times are ignored (all requests are queued at the start)."""
        rep = ServeReport()
        queue = sorted(requests, key=lambda q: q.arrival)
        for q in queue:
            if q.spec is None:
                q.spec = problem_from_case(q.case, precision=q.precision, allow_nonpositive=1)
            q.footprint = footprint_bytes(q.spec)
        pending, active = list(queue), []
        used = 0
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            # admission: arrived requests, in order, while slots and memory allow
            while pending and (not realtime or pending[0].arrival <= now):
                q = pending[0]
                if len(active) >= self.max_active or (
                        self.hbm_budget and used + q.footprint > self.hbm_budget and active):
                    rep.admission_waits += 1
                    break
                pending.pop(0)
                q.solver = Solver(q.spec, stream=self.stream)
                q.admitted = now
                used += q.footprint
                rep.peak_bytes = max(rep.peak_bytes, used)
                active.append(q)
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival - (self.clock() - t0))))
                continue
            rep.max_active = max(rep.max_active, len(active))
            try:
                step_batch([q.solver for q in active], 1)
                self.stream.synchronize()  # one tick at a time: admission and latency follow the GPU
            except DlrError:
                # a request failed on the device (sticky status): drop it, keep serving the rest
                keep = []
                for q in active:
                    status = q.solver.stats()["status"]
                    if status != 0:
                        rep.failures.append((q.rid, q.done_steps, status))
                        q.solver.close()
                        q.solver = None
                        used -= q.footprint
                    else:
                        keep.append(q)
                if len(keep) == len(active):
                    raise
                active = keep
                continue
            rep.ticks += 1
            for q in active:
                q.done_steps += 1
            finished = [q for q in active if q.done_steps >= q.steps]
            if finished:
                t_done = self.clock() - t0
                for q in finished:
                    st = q.solver.stats()
                    rep.updates_total += st["cell_angle_updates"]
                    rep.steps_total += st["steps"]
                    if self.keep_results:
                        q.result_T = q.solver.T()
                    q.solver.close()
                    q.solver = None
                    q.finished = t_done
                    rep.latencies.append(q.finished - q.arrival if realtime else q.finished)
                    used -= q.footprint
                active = [q for q in active if q.done_steps < q.steps]
        self.stream.synchronize()
        rep.wall = self.clock() - t0
        return rep
