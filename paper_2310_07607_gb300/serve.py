"""Continuous-batching request loop for monodomain simulations (over mdl_batch_*).

Requests arrive over time; the loop admits every waiting request whose device-memory
footprint fits the batch budget (first fit over the queue, oldest first), steps all
resident simulations together -- the batch's fused rounds: each slot's adaptation and level
phases on its own stream, one sweep launch per global tick over every resident slot -- and
retires finished slots, recording time-to-result (completion minus arrival).  Requests still
running when the wall limit ends are reported with their progress and a projected
time-to-result from their own barrier rate.

Only scheduling lives here; every numerical step runs in libmdl's CUDA kernels.
"""
from __future__ import annotations

import math
import statistics
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

from .mdl import Batch, MdlError, Sim


@dataclass
class Request:
    rid: int
    prob: object
    horizon_ms: float
    arrival_s: float
    V0: Optional[np.ndarray] = None
    v0: Optional[np.ndarray] = None
    admitted_s: float = math.nan
    finished_s: float = math.nan
    slot: int = -1
    barriers_total: int = 0
    barriers_done: int = 0
    dof_updates: int = 0
    rc: int = 0
    result: Optional[dict] = None


def percentile(xs: List[float], q: float) -> float:
    if not xs:
        return math.nan
    s = sorted(xs)
    k = (len(s) - 1) * q
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return s[lo] + (s[hi] - s[lo]) * (k - lo)


class Server:
    def __init__(self, budget_bytes: int = 0, barriers_per_round: int = 8, autotune: bool = True,
                 on_result: Optional[Callable[[Request, Sim], dict]] = None):
        self.batch = Batch(budget_bytes, autotune)
        self.k = barriers_per_round
        self.waiting: deque = deque()
        self.active: Dict[int, Request] = {}
        self.done: List[Request] = []
        self.on_result = on_result
        self.rounds = 0
        self.busy_rounds = 0
        self.peak_bytes = 0
        self.peak_resident = 0
        self.queue_samples: List[int] = []
        self.t0 = None

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _admit(self):
        kept = deque()
        while self.waiting:
            req = self.waiting.popleft()
            try:
                slot = self.batch.admit(req.prob, req.horizon_ms, req.V0, req.v0)
            except MdlError as e:
                if e.code == -3:          # does not fit now: keep waiting
                    kept.append(req)
                    continue
                req.rc = e.code
                req.finished_s = self.now()
                self.done.append(req)
                continue
            req.slot = slot
            req.admitted_s = self.now()
            g, _, _ = self.batch.slot(slot)
            t, nb, dt = g.time()
            req.barriers_total = int(math.floor(req.horizon_ms / dt + 1e-9))
            self.active[slot] = req
        self.waiting = kept

    def _retire(self):
        for slot in self.batch.poll():
            req = self.active.pop(slot)
            g, state, rc = self.batch.slot(slot)
            st = g.stats()
            req.barriers_done = g.time()[1]
            req.dof_updates = st["dof_updates"]
            req.rc = rc
            req.finished_s = self.now()
            if self.on_result is not None and rc == 0:
                req.result = self.on_result(req, g)
            self.batch.release(slot)
            self.done.append(req)

    def round(self):
        self._admit()
        used, budget, resident = self.batch.usage()
        self.peak_bytes = max(self.peak_bytes, used)
        self.peak_resident = max(self.peak_resident, resident)
        self.queue_samples.append(len(self.waiting))
        if self.active:
            self.batch.step(self.k)
            self.busy_rounds += 1
        self.rounds += 1
        self._retire()

    def run(self, requests: List[Request], wall_limit_s: float, drain: bool = False) -> dict:
        """Replay arrivals in real time (arrival_s relative to the start) for wall_limit_s."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        i = 0
        self.t0 = time.perf_counter()
        while True:
            now = self.now()
            while i < len(pending) and pending[i].arrival_s <= now:
                self.submit(pending[i])
                i += 1
            if now >= wall_limit_s and not drain:
                break
            if not self.active and not self.waiting:
                if i >= len(pending):
                    break                       # nothing left to serve
                time.sleep(min(0.001, max(0.0, pending[i].arrival_s - now)))
                continue
            self.round()
        return self.report(wall=self.now(), arrived=i, offered=len(pending))

    def report(self, wall: float, arrived: int, offered: int) -> dict:
        ok = [r for r in self.done if r.rc == 0]
        ttr = [r.finished_s - r.arrival_s for r in ok]
        prog = []
        proj = []
        for r in self.active.values():
            g, _, _ = self.batch.slot(r.slot)
            nb = g.time()[1]
            elapsed = self.now() - r.admitted_s
            frac = nb / max(1, r.barriers_total)
            prog.append(frac)
            if nb > 0:
                rate = nb / max(elapsed, 1e-9)
                proj.append((r.admitted_s - r.arrival_s) + r.barriers_total / rate)
        return {
            "offered": offered, "arrived": arrived, "completed": len(ok),
            "failed": len([r for r in self.done if r.rc != 0]),
            "running": len(self.active), "waiting": len(self.waiting),
            "wall_s": wall, "sims_per_s": len(ok) / wall if wall > 0 else 0.0,
            "ttr_p50_s": percentile(ttr, 0.5), "ttr_p99_s": percentile(ttr, 0.99),
            "running_progress_mean": float(np.mean(prog)) if prog else None,
            "projected_ttr_p50_s": percentile(proj, 0.5) if proj else None,
            "projected_ttr_p99_s": percentile(proj, 0.99) if proj else None,
            "busy_fraction": self.busy_rounds / max(1, self.rounds),
            "peak_resident": self.peak_resident, "peak_bytes": self.peak_bytes,
            "queue_mean": float(np.mean(self.queue_samples)) if self.queue_samples else 0.0,
            "dof_updates_completed": int(sum(r.dof_updates for r in ok)),
        }

    def close(self):
        self.batch.close()
