"""Continuous-batching server for rheology jobs on one GPU.

Jobs (a lattice size, rho0, a shear rate, a step count, a seed) arrive over
time.  Each is admitted into the lattice pool (``lb_pool_*``) as soon as its
device footprint fits the pool's arena, stays resident on the device, and is
stepped together with every other resident job by one persistent launch per
time step; finished jobs hand back their result and free their memory, which
lets queued jobs in.  The per-site arithmetic does not depend on which jobs
share a launch, so a job's result is the same alone and in any mix.

Shear jobs are plane-Couette lattices (walls moving at +-U with shear rate
2U/ny); their result carries the time-averaged wall stress and the effective
viscosity.  Scheduling is host-side bookkeeping only; every step runs in the
library's kernels.
"""
from __future__ import annotations

import collections
import json
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


@dataclass
class Job:
    """One request.  `spec` keys: nx, ny, rho0, shear_rate, steps, seed."""
    spec: dict
    arrival: float
    id: int = -1
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[dict] = None
    error: Optional[str] = None
    _slot: int = -1

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival

    @property
    def done(self) -> bool:
        return self.finished is not None


@dataclass
class Stats:
    """Job counts: every admitted job ends once, as finished (a result),
    failed (an error) or cancelled; site_updates counts finished jobs only."""
    admitted: int = 0
    finished: int = 0
    failed: int = 0
    refused_nomem: int = 0
    cancelled: int = 0
    site_updates: int = 0
    quanta: int = 0


class Server:
    """Admit queued jobs while their footprint fits, run one quantum of
    steps for every resident job, collect the finished ones; repeat.

    `pool` is a ``paper_0807_4471_gb300.Pool`` (or an object with the same
    admit/run/poll/stress/fields/release/footprint methods); `make_params`
    turns a job spec into the library's ``lb_params``.  Queued jobs are
    admitted in arrival order; a later, smaller job may go ahead of one that
    does not fit yet (backfill) unless the head of the queue has waited more
    than `max_bypass` quanta.  With `log_path`, every job that ends
    (finished, failed or cancelled) appends one JSON line: id, spec,
    arrival / admission / end times, latency, steps and result or error."""

    def __init__(self, pool, make_params: Callable[[dict], object], quantum: int = 100,
                 keep_fields: bool = False, max_bypass: int = 20,
                 clock: Callable[[], float] = time.perf_counter, log_path: Optional[str] = None):
        self.pool = pool
        self.make_params = make_params
        self.quantum = int(quantum)
        self.keep_fields = keep_fields
        self.max_bypass = max_bypass
        self.clock = clock
        self.log_path = log_path
        self.queue: collections.deque[Job] = collections.deque()
        self.running: dict[int, Job] = {}
        self.done: list[Job] = []
        self.stats = Stats()
        self._next_id = 0
        self._head_wait = 0

    # ----------------------------------------------------------- requests
    def submit(self, spec: dict, arrival: Optional[float] = None) -> Job:
        job = Job(spec=dict(spec), arrival=self.clock() if arrival is None else arrival,
                  id=self._next_id)
        self._next_id += 1
        self.queue.append(job)
        return job

    def cancel(self, job: Job) -> bool:
        """Withdraw a queued job, or stop a running one and free its memory
        (between quanta: no kernel of the pool is in flight then).  Returns
        False if the job had already ended."""
        if job.done:
            return False
        if job in self.queue:
            self.queue.remove(job)
        elif job._slot in self.running and self.running[job._slot] is job:
            self.pool.release(job._slot)
            del self.running[job._slot]
        else:
            return False
        job.error = "cancelled"
        job.finished = self.clock()
        self.done.append(job)
        self.stats.cancelled += 1
        self._log(job)
        return True

    def _log(self, job: Job):
        if not self.log_path:
            return
        rec = dict(id=job.id, spec=job.spec, arrival=job.arrival, admitted=job.admitted,
                   finished=job.finished, latency=job.latency, error=job.error,
                   result=None if job.result is None else
                   {k: v for k, v in job.result.items() if k != "fields"})
        with open(self.log_path, "a") as fh:
            fh.write(json.dumps(rec) + "\n")

    # ------------------------------------------------------------ serving
    def _admit(self):
        from . import LB_ERR_INVALID, LB_ERR_NOMEM, LbError
        admitted_any = False
        bypass_ok = self._head_wait <= self.max_bypass
        for job in list(self.queue):
            p = self.make_params(job.spec)
            try:
                job._slot = self.pool.admit(p, int(job.spec.get("seed", 0)),
                                            int(job.spec["steps"]))
            except LbError as e:
                if e.status == LB_ERR_NOMEM:
                    self.stats.refused_nomem += 1
                    if not bypass_ok:
                        break          # keep the head's turn
                    continue
                if e.status == LB_ERR_INVALID and len(self.running) > 0:
                    continue           # pool full of jobs: wait for a slot
                job.error = str(e)
                job.finished = self.clock()
                self.queue.remove(job)
                self.done.append(job)
                self.stats.failed += 1
                self._log(job)
                continue
            job.admitted = self.clock()
            self.queue.remove(job)
            self.running[job._slot] = job
            self.stats.admitted += 1
            admitted_any = True
        if self.queue and not admitted_any:
            self._head_wait += 1
        else:
            self._head_wait = 0

    def _collect(self):
        from . import LbError
        for slot, job in list(self.running.items()):
            steps, finished = self.pool.poll(slot)
            if not finished:
                continue
            try:
                res = dict(self.pool.stress(slot))
                if self.keep_fields:
                    res["fields"] = self.pool.fields(slot)
                job.result = res
            except LbError as e:
                job.error = str(e)
            self.pool.release(slot)
            job.finished = self.clock()
            del self.running[slot]
            self.done.append(job)
            if job.error is None:
                self.stats.finished += 1
                self.stats.site_updates += int(job.spec["nx"]) * int(job.spec["ny"]) * steps
            else:   # its steps produced no result: neither finished nor counted
                self.stats.failed += 1
            self._log(job)

    def step(self) -> int:
        """One scheduling round.  Returns the number of resident jobs."""
        self._admit()
        if self.running:
            self.pool.run(self.quantum)
            self.stats.quanta += 1
        self._collect()
        return len(self.running)

    def idle(self) -> bool:
        return not self.queue and not self.running

    def run_until_idle(self, max_rounds: int = 10 ** 9):
        for _ in range(max_rounds):
            if self.idle():
                return
            self.step()

    def replay(self, stream: list[tuple[float, dict]], time_scale: float = 1.0):
        """Serve an arrival stream [(arrival offset in s, spec)] in real time:
        each job is submitted once the clock passes its arrival offset (times
        time_scale); returns the jobs in submission order."""
        t0 = self.clock()
        pending = collections.deque(sorted(stream, key=lambda a: a[0]))
        jobs = []
        while pending or not self.idle():
            now = self.clock() - t0
            while pending and pending[0][0] * time_scale <= now:
                off, spec = pending.popleft()
                jobs.append(self.submit(spec, arrival=t0 + off * time_scale))
            if self.idle():
                if pending:   # nothing to do until the next arrival
                    wait = pending[0][0] * time_scale - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            self.step()
        return jobs


def percentile(values, q: float) -> float:
    v = np.asarray(sorted(values), dtype=float)
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, q))


def job_params(lb, shared_kwargs: dict, precision: str = "fp16") -> Callable[[dict], object]:
    """Map a job spec to lb_params: periodic if shear_rate == 0, else Couette
    with wall speed shear_rate * ny / 2 and the linear initial profile."""
    def make(spec: dict):
        rate = float(spec.get("shear_rate", 0.0))
        ny = int(spec["ny"])
        kw = dict(shared_kwargs)
        kw.update(rho0=float(spec.get("rho0", kw.get("rho0", 0.70))))
        if rate > 0:
            kw.update(boundary=1, u_wall=rate * ny / 2.0, init_shear=1)
        return lb.make_params(int(spec["nx"]), ny, precision, **kw)
    return make
