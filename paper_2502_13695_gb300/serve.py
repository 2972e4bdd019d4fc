"""Request loop with continuous batching over simulations resident on one GPU.

Requests (a workload configuration and a step count) arrive over time.  A
request is admitted as soon as its state fits the device-memory budget next
to the running ones (the arena size comes from pic_query); every admitted
simulation keeps its fields, particles and RNG state on the device until it
finishes.  Running simulations advance together in quanta of 32 steps from
one CUDA graph (pic_batch_*, rebuilt when the running set changes), so the
work of requests that arrived at different times overlaps on the GPU; a
request whose remaining steps are fewer than a quantum finishes alone.  A
finished request returns its FP64 diagnostics and is released.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from . import pic

QUANTUM = 32


@dataclass
class Request:
    rid: int
    cfg: dict
    steps: int
    arrival_s: float = 0.0


@dataclass
class Result:
    rid: int
    arrival_s: float
    admit_s: float
    done_s: float
    diagnostics: dict = field(default_factory=dict)

    @property
    def time_to_result_s(self) -> float:
        return self.done_s - self.arrival_s


class Server:
    def __init__(self, budget_bytes: float, quantum: int = QUANTUM, keep_state=False):
        self.budget = float(budget_bytes)
        self.quantum = int(quantum)
        self.keep_state = keep_state
        self.used = 0.0
        self.active = collections.OrderedDict()  # rid -> [req, sim, remaining, admit_s, bytes]
        self._batch = None
        self._batch_ids = ()

    # -- internals -----------------------------------------------------------
    def _rebatch(self):
        ids = tuple(rid for rid, a in self.active.items() if a[2] >= self.quantum)
        if ids == self._batch_ids:
            return
        if self._batch is not None:
            self._batch.close()
            self._batch = None
        self._batch_ids = ids
        if ids:
            self._batch = pic.Batch([self.active[r][1] for r in ids])

    def _admit(self, req: Request, now: float) -> bool:
        import torch
        need = float(pic.query(req.cfg)["arena_bytes"])
        if need > self.budget:
            raise ValueError(f"request {req.rid} needs {need:.3g} B, above the whole budget")
        if self.used + need > self.budget:
            return False
        sim = pic.Simulation(req.cfg, stream=torch.cuda.Stream())
        self.active[req.rid] = [req, sim, req.steps, now, need]
        self.used += need
        return True

    def _retire(self, rid, now, results):
        req, sim, _, admit_s, need = self.active.pop(rid)
        sim.sync()
        d = sim.diagnostics()
        if self.keep_state:
            d["fields"] = sim.fields()
        results.append(Result(rid, req.arrival_s, admit_s, now, d))
        sim.close()
        self.used -= need

    # -- public ------------------------------------------------------------------
    def run(self, requests, clock=None):
        """Serve `requests` (arrival_s relative to the start) in real time;
        returns the results in completion order."""
        clock = clock or time.perf_counter
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting = collections.deque()
        results = []
        t0 = clock()
        while pending or waiting or self.active:
            now = clock() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            while waiting and self._admit(waiting[0], now):
                waiting.popleft()
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(0.05, pending[0].arrival_s - now)))
                continue
            self._rebatch()
            if self._batch is not None:
                self._batch.step(self.quantum)
                for rid in self._batch_ids:
                    self.active[rid][2] -= self.quantum
            for rid, a in self.active.items():
                if rid not in self._batch_ids and 0 < a[2] < self.quantum:
                    a[1].step(a[2])
                    a[2] = 0
            if self._batch is not None:
                self._batch.sync()
            now = clock() - t0
            for rid in [r for r, a in self.active.items() if a[2] <= 0]:
                self._retire(rid, now, results)
        if self._batch is not None:
            self._batch.close()
            self._batch = None
            self._batch_ids = ()
        return results
