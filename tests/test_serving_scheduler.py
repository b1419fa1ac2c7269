"""Continuous-batching scheduler of serve.py driven by a CPU fake backend (no GPU)."""
import time

import numpy as np

from paper_2401_10287_gb300 import serve

import workloads as W


class _Handle:
    def __init__(self, key):
        self.key = key
        self.busy = False
        self.capacity = 0


class _Event:
    def __init__(self, t_done):
        self.t_done = t_done


class FakeBackend:
    """Each chunk takes (walkers x electrons) microseconds of simulated device time."""

    def __init__(self):
        self.handles = {}
        self.created = 0
        self.destroyed = 0
        self.log = []

    def new_stream(self):
        return object()

    def acquire(self, req):
        for h in self.handles.setdefault(req.key, []):
            if not h.busy:
                h.busy = True
                return h, False
        h = _Handle(req.key)
        h.busy = True
        self.handles[req.key].append(h)
        self.created += 1
        return h, True

    def release(self, req, handle):
        handle.busy = False

    def destroy(self, key, handle):
        self.handles[key].remove(handle)
        self.destroyed += 1

    def workspace_bytes(self, handle, n):
        return max(n, handle.capacity) * 1000

    def job_bytes(self, req):
        return req.n_walkers * 10

    def grow(self, handle, n):
        handle.capacity = max(handle.capacity, n)

    def _later(self, req, scale=1.0):
        return _Event(time.perf_counter() + scale * req.n_walkers * (req.n_up + req.n_down) * 1e-7)

    def start(self, job, stream):
        self.log.append(("start", job.req.job_id))
        return self._later(job.req, 0.1)

    def mcmc_chunk(self, job, stream, offset, steps):
        return self._later(job.req, steps * 0.1)

    def energy(self, job, stream):
        return self._later(job.req)

    def collect(self, job):
        return -float(job.req.n_up + job.req.n_down), 0.01, 0.5

    @staticmethod
    def done(ev):
        return time.perf_counter() >= ev.t_done

    def free(self, job):
        pass


def _requests(n=60, rate=2000.0):
    jobs = W.serving_jobs(n_jobs=n, rate_per_s=rate, seed=4, mcmc_steps=20)
    return serve.requests_from_jobs(jobs)


def test_all_jobs_complete_fifo_and_budget():
    reqs = _requests()
    be = FakeBackend()
    budget = 12_000_000
    srv = serve.Server(be, memory_budget=budget, slots=4)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    assert srv.peak_footprint <= budget
    assert srv.max_concurrent > 1                 # work of several jobs was in flight together
    admitted = [jid for _, kind, jid in srv.events if kind == "admit"]
    electrons = {r.job_id: r.n_up + r.n_down for r in reqs}
    order = [r.job_id for r in sorted(reqs, key=lambda r: r.arrival_s) if electrons[r.job_id] > 0]
    assert admitted == order                      # first come, first served
    for r in res:
        assert r.done_s >= r.admit_s >= r.arrival_s - 1e-9
        if electrons[r.job_id] > 0:
            assert r.energy == -electrons[r.job_id]


def test_zero_electron_job_returns_nuclear_repulsion():
    h_plus = W.atom(1, 1)
    req = serve.Request(0, 0.0, h_plus.nuclei, h_plus.charges, 0, 0, 300)
    res = serve.Server(FakeBackend(), memory_budget=10 ** 9, slots=2).run([req])
    assert res[0].energy == 0.0


def test_tight_budget_serialises_and_evicts():
    reqs = _requests(30)
    be = FakeBackend()
    biggest = max(be.workspace_bytes(_Handle("x"), r.n_walkers) + be.job_bytes(r) for r in reqs)
    srv = serve.Server(be, memory_budget=biggest + 1, slots=4)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    assert srv.peak_footprint <= biggest + 1
    assert srv.evictions > 0


def test_summary_percentiles():
    res = [serve.Result(i, 0.0, 0.0, 0.0, 100, 0.0, 0.0, (i + 1) * 0.001) for i in range(100)]
    summ = serve.summarize(res, 1.0)
    assert abs(summ["latency_ms"]["p50"] - 50.5) < 1e-9
    assert summ["jobs"] == 100 and summ["walker_energies_per_s"] == 100 * 100
