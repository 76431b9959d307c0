"""Continuous batching of droplet cases on one GPU.

Cases arrive over time; each runs until its deformation factor D (Eq. 63)
is steady, |D(t) - D(t - C)| / C < tol with C = check_every steps, or until
max_steps.  The server keeps every admitted case resident in one batch
(ehdlb_batch_*): it admits waiting cases first come, first served while the
batch's device-memory budget has room for them, steps all resident cases
together C steps at a time, reads every case's D with one device launch and
retires the steady ones, whose memory the next waiting case can then take.
``serve_one_by_one`` runs the same stream with one lattice at a time, the
plain way.

Only scheduling lives here; every step of every case runs in the library.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from . import ehdlb


@dataclass
class Case:
    """One request: its lattice, physical parameters and arrival time (s)."""
    t: float
    nx: int
    ny: int
    d_mm: float
    dpsi_kV: float
    eps_r: float
    mu_r: float
    key: int = 0

    def params(self, sweeps: int) -> ehdlb.ehdlb_params:
        p = ehdlb.ehdlb_params_from_physical(self.nx, self.ny, self.d_mm, self.dpsi_kV, self.eps_r, self.mu_r)
        p.sweeps_min = p.sweeps_max = sweeps
        return p


@dataclass
class Result:
    key: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    D: float
    steady: bool

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    case: Case
    admitted: float
    steps: int = 0
    D_prev: float | None = None


@dataclass
class Server:
    """Continuous batching over one ehdlb batch (or any object with the same
    add / remove / step / deformation methods)."""
    batch: object
    sweeps: int = 20
    check_every: int = 1000
    max_steps: int = 50000
    tol: float = 1e-6
    clock: object = time.perf_counter
    sleep: object = time.sleep
    waiting: collections.deque = field(default_factory=collections.deque)
    active: dict = field(default_factory=dict)
    results: list = field(default_factory=list)

    def _admit(self, now: float):
        while self.waiting:
            case = self.waiting[0]
            cid = self.batch.add(case.nx, case.ny, case.params(self.sweeps))
            if cid is None:          # no room: wait for a case to retire
                break
            self.waiting.popleft()
            self.active[cid] = _Active(case, now)

    def _advance(self, now_fn):
        ids = list(self.active)
        self.batch.step(self.check_every)
        D = self.batch.deformation(ids)
        now = now_fn()
        for cid, d in zip(ids, D):
            a = self.active[cid]
            a.steps += self.check_every
            steady = a.D_prev is not None and abs(d - a.D_prev) / self.check_every < self.tol
            if steady or a.steps >= self.max_steps:
                self.results.append(Result(a.case.key, a.case.t, a.admitted, now, a.steps, float(d), steady))
                self.batch.remove(cid)
                del self.active[cid]
            else:
                a.D_prev = float(d)

    def run(self, cases: list[Case]) -> list[Result]:
        """Serve cases (sorted by arrival time, seconds from the call) in real time."""
        start = self.clock()
        now_fn = lambda: self.clock() - start
        pending = collections.deque(sorted(cases, key=lambda c: c.t))
        while pending or self.waiting or self.active:
            now = now_fn()
            while pending and pending[0].t <= now:
                self.waiting.append(pending.popleft())
            self._admit(now)
            if self.active:
                self._advance(now_fn)
            elif pending:
                self.sleep(max(0.0, pending[0].t - now_fn()))
            elif self.waiting:
                raise RuntimeError("a waiting case does not fit in an empty batch")
        return self.results


def serve_one_by_one(cases: list[Case], sweeps: int = 20, check_every: int = 1000, max_steps: int = 50000,
                     tol: float = 1e-6, precision=ehdlb.FP32, clock=time.perf_counter,
                     sleep=time.sleep) -> list[Result]:
    """The same stream served one lattice at a time, first come, first served."""
    start = clock()
    out = []
    for case in sorted(cases, key=lambda c: c.t):
        now = clock() - start
        if case.t > now:
            sleep(case.t - now)
        admitted = clock() - start
        lat = ehdlb.Lattice(case.nx, case.ny, case.params(sweeps), precision=precision)
        steps, D_prev, steady, d = 0, None, False, 0.0
        while steps < max_steps:
            lat.step(check_every)
            steps += check_every
            d = lat.deformation()
            if D_prev is not None and abs(d - D_prev) / check_every < tol:
                steady = True
                break
            D_prev = d
        lat.close()
        out.append(Result(case.key, case.t, admitted, clock() - start, steps, d, steady))
    return out


def percentile(values, q: float) -> float:
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = sorted(values)
    if not v:
        return float("nan")
    pos = (len(v) - 1) * q / 100.0
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)
