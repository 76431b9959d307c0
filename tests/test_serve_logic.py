"""Scheduling of the serving loop on the CPU, against a scripted batch.

The fake batch holds at most `slots` cases, and each case's deformation
approaches its final value exponentially with the steps it has taken, so the
step at which it becomes steady is known in closed form.
"""
import math

from paper_2501_04920_gb300.serve import Case, Server, percentile


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeBatch:
    def __init__(self, slots, clock, secs_per_step, tau):
        self.slots, self.clock, self.secs_per_step, self.tau = slots, clock, secs_per_step, tau
        self.cases, self.next_id, self.max_active, self.order = {}, 0, 0, []

    def add(self, nx, ny, params):
        if len(self.cases) >= self.slots:
            return None
        cid = self.next_id
        self.next_id += 1
        self.cases[cid] = [0, nx]
        self.order.append(nx)
        self.max_active = max(self.max_active, len(self.cases))
        return cid

    def remove(self, cid):
        del self.cases[cid]

    def step(self, n):
        for c in self.cases.values():
            c[0] += n
        self.clock.t += n * self.secs_per_step

    def deformation(self, ids):
        return [0.1 * (1.0 - math.exp(-self.cases[i][0] / self.tau)) for i in ids]


def make_cases(n, gap):
    # the lattice width labels each case (it is what FakeBatch records)
    return [Case(t=i * gap, nx=64 + 8 * i, ny=64, d_mm=1.0, dpsi_kV=1.0, eps_r=2.0, mu_r=2.0, key=i)
            for i in range(n)]


def steady_step(check, tau, tol):
    # first multiple of check at which |D(s) - D(s - check)| / check < tol
    s = 2 * check
    while abs(0.1 * (math.exp(-(s - check) / tau) - math.exp(-s / tau))) / check >= tol:
        s += check
    return s


def test_continuous_batching_admits_fifo_within_the_slots_and_retires_steady_cases():
    clock = FakeClock()
    fb = FakeBatch(slots=3, clock=clock, secs_per_step=1e-3, tau=800.0)
    srv = Server(fb, check_every=100, max_steps=100000, tol=1e-6, clock=clock, sleep=clock.sleep)
    cases = make_cases(8, gap=0.05)
    res = srv.run(cases)
    assert len(res) == 8 and not srv.active and not srv.waiting
    assert fb.max_active == 3
    assert fb.order == [c.nx for c in cases]            # first come, first served
    expect = steady_step(100, 800.0, 1e-6)
    for r in res:
        assert r.steady and r.steps == expect
        assert r.finished >= r.admitted >= r.arrival
    lat = [r.latency for r in res]
    assert percentile(lat, 50) <= percentile(lat, 99) <= max(lat)


def test_cases_stop_at_max_steps_and_idle_server_waits_for_arrivals():
    clock = FakeClock()
    fb = FakeBatch(slots=2, clock=clock, secs_per_step=1e-3, tau=1e9)   # never steady
    srv = Server(fb, check_every=50, max_steps=200, tol=1e-12, clock=clock, sleep=clock.sleep)
    res = srv.run([Case(t=5.0, nx=64, ny=64, d_mm=1.0, dpsi_kV=1.0, eps_r=2.0, mu_r=2.0, key=7)])
    (r,) = res
    assert not r.steady and r.steps == 200
    assert r.admitted >= 5.0                         # slept until the arrival
    assert abs(r.finished - r.admitted - 0.2) < 1e-9   # 200 steps of 1 ms


def test_percentile_interpolates_order_statistics():
    v = list(range(101))
    assert percentile(v, 50) == 50 and percentile(v, 99) == 99
    assert percentile([1.0, 3.0], 50) == 2.0
