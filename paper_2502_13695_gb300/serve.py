"""Request loop with continuous batching over simulations resident on one GPU.

The loop itself is native (pic_serve_* in csrc/pic_serve.cpp): a host
worker thread admits submitted requests in submission order as soon as
their state fits the device-memory budget next to the running ones (the
arena size comes from pic_query; later requests may pass one that does not
fit until it has waited 1 s; the state lives in ranges of the server's own
device memory, reserved in chunks up to the budget), keeps every admitted simulation's fields,
particles and RNG state on the device until it finishes, advances the
running ones together in quanta of 32 steps from one CUDA graph
(pic_batch_*, rebuilt when the running set changes), lets a request with
fewer steps left than a quantum finish alone, and returns a finished
request's FP64 diagnostics.  This module submits requests at their arrival
times and collects the results (argument marshalling only).
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

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


def _bind(L):
    if getattr(L, "_serve_bound", False):
        return L
    vp, P = ctypes.c_void_p, ctypes.POINTER
    L.pic_serve_create.argtypes = [ctypes.c_double, ctypes.c_int, P(vp)]
    L.pic_serve_submit.argtypes = [vp, P(pic.Grid), P(pic.Material), P(pic.Pulse),
                                   ctypes.c_uint64, ctypes.c_longlong, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, vp,
                                   P(ctypes.c_longlong)]
    L.pic_serve_poll.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, P(ctypes.c_int),
                                 P(pic.Diag), P(ctypes.c_double)]
    L.pic_serve_destroy.argtypes = [vp]
    L._serve_bound = True
    return L


class Server:
    def __init__(self, budget_bytes: float, quantum: int = QUANTUM, keep_state=False):
        self.budget = float(budget_bytes)
        self.quantum = int(quantum)
        self.keep_state = keep_state

    def run(self, requests, clock=None):
        """Serve `requests` (arrival_s relative to the start) in real time;
        returns the results in completion order.  Times are seconds from the
        start on the server's steady clock."""
        clock = clock or time.perf_counter
        L = _bind(pic.lib())
        srv = ctypes.c_void_p()
        pic._check(L.pic_serve_create(self.budget, self.quantum, ctypes.byref(srv)))
        t0 = clock()
        try:
            return self._loop(L, srv, requests, clock, t0)
        finally:
            L.pic_serve_destroy(srv)

    def _loop(self, L, srv, requests, clock, t0):
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
        out = {}  # ticket -> (request, structs kept alive, fields buffer)
        results = []
        while pending or out:
            now = clock() - t0
            while pending and pending[0].arrival_s <= now:
                req = pending.popleft()
                g, m, p, keep = pic.c_structs(req.cfg)
                F = None
                if self.keep_state:
                    F = np.zeros((15, req.cfg["nz"] + 1, req.cfg["ny"], req.cfg["nx"]))
                t = ctypes.c_longlong()
                pic._check(L.pic_serve_submit(srv, ctypes.byref(g), ctypes.byref(m),
                                              ctypes.byref(p), int(req.cfg["seed"]),
                                              int(req.steps), 0, 0.0, 1.0, pic._ptr(F),
                                              ctypes.byref(t)))
                out[t.value] = (req, (g, m, p, keep), F)
            for t in list(out):
                done, d = ctypes.c_int(), pic.Diag()
                times = (ctypes.c_double * 3)()
                rc = L.pic_serve_poll(srv, t, 0, ctypes.byref(done), ctypes.byref(d), times)
                if not done.value:
                    pic._check(rc)
                    continue
                req, _, F = out.pop(t)
                pic._check(rc)
                diag = pic.diag_dict(d)
                diag["spectrum"] = np.zeros(0)
                if F is not None:
                    diag["fields"] = F
                results.append(Result(req.rid, req.arrival_s, times[1], times[2], diag))
            wait = 1e-3
            if pending:
                wait = min(wait, max(0.0, pending[0].arrival_s - (clock() - t0)))
            time.sleep(wait)
        results.sort(key=lambda r: r.done_s)
        return results
