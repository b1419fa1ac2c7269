"""Continuous-batching VMC energy server over the C ABI.

A job is one VMC energy estimate: electrons placed by Algorithm 1, `mcmc_steps`
Metropolis steps on |psi|^2, then the mean local energy (Eqs. 1-3) of its walkers.
Jobs arrive over time; the server

* admits a waiting job (first come, first served) as soon as a slot (a CUDA stream) is
  free and the device-memory footprint of everything admitted, counted with
  ``fn_workspace_bytes`` plus the job's own tensors, stays within the budget;
* keeps one library handle (and its workspace and parameters) per molecule resident
  and reuses it for later jobs of the same molecule;
* enqueues each admitted job's work in chunks (a few Metropolis steps at a time) on the
  job's own stream, so work of different jobs overlaps on the device, and polls CUDA
  events to learn when a chunk is done;
* records latency from arrival to the moment the job's energy is on the host.

The device work is behind a small backend interface; `LibraryBackend` runs it through
``libfnvmc.so``.  Any other backend with the same methods (the tests use a CPU fake)
drives the same scheduler.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Deque, Dict, List, Optional, Tuple

import numpy as np

from . import api

CHUNK_STEPS = 10


@dataclass
class Request:
    job_id: int
    arrival_s: float
    nuclei: np.ndarray
    charges: np.ndarray
    n_up: int
    n_down: int
    n_walkers: int
    mcmc_steps: int = 50
    step_size: float = 0.02
    init_std: float = 1.0
    seed: int = 0
    key: str = ""


@dataclass
class Result:
    job_id: int
    energy: float
    stderr: float
    acceptance: float
    n_walkers: int
    arrival_s: float
    admit_s: float
    done_s: float

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class _Active:
    """Book-keeping of one admitted job."""

    def __init__(self, req: Request, slot: int, handle, footprint: int, admit_s: float):
        self.req = req
        self.slot = slot
        self.handle = handle
        self.footprint = footprint
        self.admit_s = admit_s
        self.steps_done = 0
        self.stage = "start"
        self.state = None
        self.pending = None


class LibraryBackend:
    """Runs jobs through libfnvmc.so; one torch stream per slot."""

    def __init__(self, cfg: api.NetConfig, param_seed: int = 4, device: str = "cuda"):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.param_seed = param_seed
        self.device = device
        self.handles: Dict[str, List[Tuple[api.System, object]]] = collections.defaultdict(list)
        self.params: Dict[str, object] = {}

    # -- resources -------------------------------------------------------------------
    def new_stream(self):
        return self.torch.cuda.Stream()

    def acquire(self, req: Request):
        """(handle, is_new): an idle handle for the molecule, or a new one (not yet allocated)."""
        for h in self.handles[req.key]:
            if not h.busy:
                h.busy = True
                return h, False
        h = api.System(req.nuclei, req.charges, req.n_up, req.n_down, self.cfg)
        h.busy = True
        h.capacity = 0
        self.handles[req.key].append(h)
        if req.key not in self.params:
            self.params[req.key] = h.init_params(self.param_seed)
        return h, True

    def release(self, req: Request, handle):
        handle.busy = False

    def destroy(self, key: str, handle):
        # the library frees the handle's device memory in the order of the handle's last
        # stream; nothing here waits for the device
        self.handles[key].remove(handle)
        handle.close()

    def workspace_bytes(self, handle, n_walkers: int) -> int:
        """Workspace the handle holds once it has served n_walkers (it never shrinks)."""
        return handle.workspace_bytes(max(n_walkers, handle.capacity))

    def job_bytes(self, req: Request) -> int:
        per = 8 if self.cfg.precision == api.FP64 else 4
        return req.n_walkers * ((req.n_up + req.n_down) * 3 * per + 8 * 4)

    def grow(self, handle, n_walkers: int):
        handle.capacity = max(handle.capacity, n_walkers)

    # -- work ------------------------------------------------------------------------
    def start(self, job: _Active, stream):
        torch = self.torch
        h, req = job.handle, job.req
        with torch.cuda.stream(stream):
            walkers, _ = h.init_walkers(req.n_walkers, req.seed, req.init_std, stream=stream)
            lp, _ = h.log_psi(self.params[req.key], walkers, stream=stream)
            acc = torch.zeros(1, dtype=torch.int64, device=self.device)
        job.state = {"walkers": walkers, "log_psi": lp, "accepted": acc}
        return self._mark(stream)

    def mcmc_chunk(self, job: _Active, stream, offset: int, steps: int):
        h, req, st = job.handle, job.req, job.state
        h.mcmc_steps(self.params[req.key], st["walkers"], st["log_psi"], steps, req.step_size, req.seed,
                     step_offset=offset, accept_count=st["accepted"], stream=stream)
        return self._mark(stream)

    def energy(self, job: _Active, stream):
        torch = self.torch
        h, req, st = job.handle, job.req, job.state
        with torch.cuda.stream(stream):
            e, _, _ = h.local_energy(self.params[req.key], st["walkers"], stream=stream)
            # Eq. 1: mean local energy and its variance, in the library
            stats = h.energy_stats(h.energy_moments(e, stream=stream), stream=stream)
            host = torch.empty(4, dtype=torch.float64, pin_memory=True)
            host[:3].copy_(stats, non_blocking=True)
            host[3:].copy_(st["accepted"], non_blocking=True)
        st["host"] = host
        return self._mark(stream)

    def collect(self, job: _Active):
        _, m, v, acc = (float(x) for x in job.state["host"])
        req = job.req
        return m, math.sqrt(max(v, 0.0) / req.n_walkers), acc / max(1, req.mcmc_steps * req.n_walkers)

    def _mark(self, stream):
        ev = self.torch.cuda.Event()
        ev.record(stream)
        return ev

    @staticmethod
    def done(event) -> bool:
        return event.query()

    def free(self, job: _Active):
        job.state = None


class Server:
    """Continuous batching with admission by device-memory footprint."""

    def __init__(self, backend, memory_budget: int, slots: int = 8, clock: Callable[[], float] = time.perf_counter,
                 chunk_steps: int = CHUNK_STEPS):
        self.backend = backend
        self.budget = int(memory_budget)
        self.slots = slots
        self.clock = clock
        self.chunk_steps = chunk_steps
        self.streams = [backend.new_stream() for _ in range(slots)]
        self.peak_footprint = 0
        self.max_concurrent = 0
        self.evictions = 0
        self.events: List[Tuple[float, str, int]] = []

    def run(self, requests: List[Request], realtime: bool = True) -> List[Result]:
        """Serves every request; arrivals are replayed against the clock when `realtime`."""
        t0 = self.clock()
        order = sorted(requests, key=lambda r: r.arrival_s)
        incoming: Deque[Request] = collections.deque(order)
        waiting: Deque[Request] = collections.deque()
        active: Dict[int, _Active] = {}
        free_slots = list(range(self.slots))
        used = 0                      # resident workspaces + tensors of active jobs
        resident: Dict[int, tuple] = {}
        keys: Dict[int, str] = {}
        last_use: Dict[int, float] = collections.defaultdict(float)
        results: List[Result] = []

        def now():
            return self.clock() - t0

        while incoming or waiting or active:
            t = now()
            while incoming and (not realtime or incoming[0].arrival_s <= t):
                r = incoming.popleft()
                if r.n_up + r.n_down == 0:
                    # no electrons: the energy is the nuclear repulsion, zero for one nucleus
                    results.append(Result(r.job_id, _nuclear_repulsion(r), 0.0, 0.0, r.n_walkers, r.arrival_s,
                                          max(t, r.arrival_s), max(t, r.arrival_s)))
                    continue
                waiting.append(r)
            # admission: first come first served, while a slot and memory are free
            while waiting and free_slots:
                r = waiting[0]
                handle, is_new = self.backend.acquire(r)
                ws_now = resident.get(id(handle), (None, 0))[1]
                ws_need = self.backend.workspace_bytes(handle, r.n_walkers)
                delta = ws_need - ws_now + self.backend.job_bytes(r)
                # make room by evicting idle handles, least recently used first
                while used + delta > self.budget:
                    idle = [(last_use[k], k) for k, (h, _) in resident.items()
                            if not h.busy and h is not handle]
                    if not idle:
                        break
                    _, k = min(idle)
                    h_old, b_old = resident.pop(k)
                    self.backend.destroy(keys[k], h_old)
                    used -= b_old
                    self.evictions += 1
                if used + delta > self.budget and active:
                    self.backend.release(r, handle)
                    if is_new:
                        self.backend.destroy(r.key, handle)
                    break
                waiting.popleft()
                slot = free_slots.pop()
                job = _Active(r, slot, handle, self.backend.job_bytes(r), now())
                resident[id(handle)] = (handle, ws_need)
                keys[id(handle)] = r.key
                self.backend.grow(handle, r.n_walkers)
                used += delta
                self.peak_footprint = max(self.peak_footprint, used)
                job.pending = self.backend.start(job, self.streams[slot])
                job.stage = "mcmc"
                active[r.job_id] = job
                self.max_concurrent = max(self.max_concurrent, len(active))
                self.events.append((job.admit_s, "admit", r.job_id))
            progressed = False
            for jid in list(active):
                job = active[jid]
                if not self.backend.done(job.pending):
                    continue
                progressed = True
                req = job.req
                stream = self.streams[job.slot]
                if job.stage == "mcmc" and job.steps_done < req.mcmc_steps:
                    k = min(self.chunk_steps, req.mcmc_steps - job.steps_done)
                    job.pending = self.backend.mcmc_chunk(job, stream, job.steps_done, k)
                    job.steps_done += k
                elif job.stage == "mcmc":
                    job.pending = self.backend.energy(job, stream)
                    job.stage = "energy"
                else:
                    e, se, acc = self.backend.collect(job)
                    results.append(Result(jid, e, se, acc, req.n_walkers, req.arrival_s, job.admit_s, now()))
                    self.events.append((now(), "done", jid))
                    self.backend.free(job)
                    self.backend.release(req, job.handle)
                    last_use[id(job.handle)] = now()
                    used -= job.footprint
                    free_slots.append(job.slot)
                    del active[jid]
            if not progressed:
                time.sleep(0.0002)
        results.sort(key=lambda r: r.job_id)
        return results


def _nuclear_repulsion(r: Request) -> float:
    e = 0.0
    for a in range(len(r.charges)):
        for b in range(a + 1, len(r.charges)):
            e += r.charges[a] * r.charges[b] / float(np.linalg.norm(r.nuclei[a] - r.nuclei[b]))
    return e


def summarize(results: List[Result], wall_s: float) -> dict:
    lat = np.array([r.latency_s for r in results]) * 1e3
    walkers = sum(r.n_walkers for r in results)
    return {"jobs": len(results), "wall_s": wall_s, "jobs_per_s": len(results) / wall_s,
            "walker_energies_per_s": walkers / wall_s,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())}}


def shard_requests(requests: List[Request], rank: int, world: int) -> List[Request]:
    """The requests one GPU serves when the stream is split by job across `world` GPUs (one
    process per GPU): the i-th arrival goes to GPU i mod world.  Whole jobs move, so no
    collective runs while serving; each GPU keeps its own admission budget and slots."""
    order = sorted(requests, key=lambda r: (r.arrival_s, r.job_id))
    return [r for i, r in enumerate(order) if i % world == rank]


def gather_results(results: List[Result], group=None) -> List[Result]:
    """Every rank's results, on every rank (torch.distributed object all-gather after serving),
    for a summary of the whole stream."""
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, results, group=group)
    return sorted((r for part in parts for r in part), key=lambda r: r.job_id)


def requests_from_jobs(jobs) -> List[Request]:
    """Requests from job descriptions carrying .system (nuclei, charges, spins, name)."""
    out = []
    for j in jobs:
        s = j.system
        out.append(Request(j.job_id, j.arrival_s, np.asarray(s.nuclei, np.float64), np.asarray(s.charges, np.float64),
                           s.n_up, s.n_down, j.n_walkers, j.mcmc_steps, j.step_size, j.init_std, j.seed,
                           key=f"{s.name}:{s.n_up}:{s.n_down}"))
    return out
