"""The serving loop's scheduling on the CPU, with a fake backend whose lattices
report prescribed force sums: admission under the memory budget, continuous
re-batching, convergence on consecutive window means, the step cap, and
rejection of requests that can never fit."""
import math

import numpy as np
import pytest

from paper_2110_00967_gb300 import serve as S
from paper_2110_00967_gb300 import workloads as W


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-3)


class FakeLattice:
    """Window k (0-based) reports Cd = cd(k), Cl = cl(k) for both estimators."""

    def __init__(self, req, cd, cl, log):
        self.req, self.cd, self.cl, self.log = req, cd, cl, log
        self.k = -1
        self.closed = False

    def sums(self):
        q = 0.5 * S.U0 ** 2 * self.req.nx * 200.0 / 2048.0
        n = 1000
        fx, fy = self.cd(self.k) * q * n, self.cl(self.k) * q * n
        return np.array([fx, fy, 0.0, fx, fy, 0.0]), np.array([n, n])

    def reset_sums(self):
        pass

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self, lats, clock, log):
        self.lats, self.clock, self.log = lats, clock, log
        log.append(sorted(l.req.rid for l in lats))

    def step(self, n):
        assert n == 1000
        for l in self.lats:
            l.k += 1
        self.clock.t += 0.01 * len(self.lats)

    def close(self):
        pass


class FakeBackend:
    def __init__(self, clock, behaviour):
        self.clock, self.behaviour = clock, behaviour
        self.batches, self.live = [], []
        self.peak = 0

    def nbytes(self, req):
        return req.nx * req.ny  # bytes proportional to the grid

    def make(self, req):
        cd, cl = self.behaviour(req)
        lat = FakeLattice(req, cd, cl, None)
        self.live.append(lat)
        self.peak = max(self.peak, sum(self.nbytes(l.req) for l in self.live if not l.closed))
        return lat

    def batch(self, lats):
        return FakeBatch(lats, self.clock, self.batches)


def converging_after(k):
    """Window means that settle (exactly) from window k on."""
    return (lambda w: 1.0 + (0.0 if w >= k else 0.1 / (w + 1)),
            lambda w: 0.5 + (0.0 if w >= k else 0.05 / (w + 1)))


def test_admission_convergence_and_rebatching():
    reqs = W.serving_requests(24, rate=50.0)
    clock = Clock()
    be = FakeBackend(clock, lambda r: converging_after(2 + r.rid % 4))
    budget = 2 * 2048 * 1024  # two of the largest grids at most
    srv = S.Server(be, memory_bytes=budget, window=1000, tol=1e-4, cap=50_000)
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert [r.rid for r in res] == [r.rid for r in reqs]
    assert all(r.converged and not r.rejected for r in res)
    for r, q in zip(res, reqs):
        # window k (0-based) covers steps 1000 k .. 1000 (k + 1); the means settle at
        # window 2 + rid % 4 and the next window sees no change
        assert r.steps == 1000 * (2 + q.rid % 4 + 2)
        assert math.isclose(r.cd, 1.0) and math.isclose(r.cl, 0.5)
        assert r.start >= r.arrival - 1e-12 and r.finish > r.start
    assert be.peak <= budget
    assert all(l.closed for l in be.live)
    # the batch was re-formed as requests came and went, never with a retired one
    assert len(be.batches) > 1
    assert any(len(b) > 1 for b in be.batches)


def test_cap_and_rejection():
    reqs = [W.Request(0, 0.0, 3.0, 512, 256), W.Request(1, 0.0, 7.0, 2048, 1024),
            W.Request(2, 0.1, 9.0, 768, 384)]
    clock = Clock()
    be = FakeBackend(clock, lambda r: (lambda w: 1.0 + 0.01 * w, lambda w: 0.2))  # never settles
    srv = S.Server(be, memory_bytes=1024 * 512, window=1000, tol=1e-4, cap=5000)
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert res[1].rejected and res[1].steps == 0  # larger than the whole budget
    for r in (res[0], res[2]):
        assert not r.rejected and not r.converged and r.steps == 5000
    summ = S.summary(res, clock.t, 0.0)
    assert summ["rejected"] == 1 and summ["capped"] == 2 and summ["converged"] == 0
    # capped requests are no solves: they count only as completed
    assert summ["solves_per_s"] == 0.0 and summ["completed_per_s"] == 2 / clock.t
    assert math.isnan(summ["p50_s"]) and summ["p50_all_s"] > 0


def test_coefficients_from_sums():
    chord = 200.0
    q = 0.5 * S.U0 ** 2 * chord
    cd, cl, cds, cls = S.coefficients([2 * q * 10, -q * 10, 0, 3 * q * 5, q * 5, 0], [10, 5], chord)
    assert (cd, cl, cds, cls) == pytest.approx((2.0, -1.0, 3.0, 1.0))
    assert all(math.isnan(x) for x in S.coefficients([0] * 6, [0, 0], chord))


def test_one_at_a_time():
    reqs = W.serving_requests(6, rate=100.0)
    clock = Clock()
    be = FakeBackend(clock, lambda r: converging_after(1))
    srv = S.Server(be, memory_bytes=1 << 40, window=1000, cap=50_000, max_active=1)
    res = srv.run(reqs, clock=clock, sleep=clock.sleep)
    assert all(len(b) == 1 for b in be.batches) and all(r.converged for r in res)
    order = sorted(res, key=lambda r: r.start)
    assert all(a.finish <= b.start + 1e-12 for a, b in zip(order, order[1:]))
