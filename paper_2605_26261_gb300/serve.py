"""Request loop for FTLM jobs: continuous batching over CUDA streams.

A job is one whole FTLM run of a cluster (sites N, bond list J_ij, Zeeman field h):
every S^z >= 0 sector (mirrored), R chains of M Lanczos steps each, then E, C, chi
and <S^z> on a temperature grid (Eq. 6-9; the field enters as -h S^z per sector).
Jobs arrive at any time.  The engine keeps a fixed number of slots, each a CUDA
stream; whenever a slot is free it takes the waiting jobs at the head of the queue
(up to `max_group` of them, and no more chains than `max_group_rows` rows of
vectors) and plans them as ONE ftlm_batch: the small sectors of all these jobs
share one persistent launch, the large ones run on the batch's side streams.  The
group is admitted to the device only when its exact footprint (sector tables +
batch workspace + outputs) fits both the engine's memory budget and the free
device memory; until then it waits with its slot.  Groups on different slots run
concurrently, so jobs that arrive while others are on the GPU start as soon as a
slot and memory free up, and their kernels overlap those already running.

Every kernel of a job has a launch shape fixed by the job's own sectors (grids by
sector dimension, one CTA per small-sector unit, fixed-order reductions), so its
results are bit-identical whether it runs alone or in a group, on any slot.

Everything on the device goes through the C ABI of libftlm (ftlm.py); this module
only schedules.  Host clocks (time.perf_counter) stamp arrival, start and finish.
"""
import collections
import dataclasses
import math
import time

import numpy as np
import torch

from . import ftlm, inputs


@dataclasses.dataclass
class Job:
    """One FTLM request.  bonds = (bi, bj, J) host arrays; h = field (units of J)."""
    job_id: int
    N: int
    bonds: tuple
    h: float = 0.0
    seed: int = 1
    arrival: float = 0.0        # host time the request arrived (engine clock)
    start: float = None         # host time its group was launched
    finish: float = None        # host time its results were on the host
    result: np.ndarray = None   # (4, nT): E, C, chi, mag
    updates: int = 0            # H.v matrix-element updates its chains applied

    @property
    def latency(self):
        return None if self.finish is None else self.finish - self.arrival


class _Group:
    def __init__(self, jobs):
        self.jobs = jobs
        self.bases = []         # per job: list of Basis
        self.batch = None
        self.outs = []          # per job: (4, nT) device tensor
        self.host = None        # pinned (n_jobs, 4, nT)
        self.meff_host = None   # pinned (sectors, R): chain lengths
        self.event = None
        self.footprint = 0


class Engine:
    """Continuous-batching FTLM server on the current CUDA device.

    slots           concurrent groups (CUDA streams)
    R, M            chains per sector and Lanczos steps
    dtype           vector storage (reductions are FP64)
    block, streams  ftlm_batch block width and side streams (0: library defaults)
    T               temperature grid (host array)
    g               g-factor of chi
    memory_budget   bytes the engine may hold on the device (default: 80 % of the
                    free memory when the engine starts)
    max_group       jobs planned into one batch at most
    max_group_rows  sum over the group's sectors of D at most (keeps a group's
                    latency bounded; the head job is always taken)
    """

    def __init__(self, slots=4, R=8, M=80, dtype=torch.float32, block=8, streams=2, T=None, g=2.0,
                 dist=ftlm.GAUSS, memory_budget=None, max_group=8, max_group_rows=1 << 22):
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.R, self.M, self.dtype, self.block, self.streams = R, M, dtype, block, streams
        self.g, self.dist = g, dist
        T = np.asarray(T if T is not None else np.logspace(-2, 1, 200), dtype=np.float64)
        self.nT = len(T)
        self.T = torch.as_tensor(T, device=self.dev)
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(memory_budget if memory_budget is not None else 0.8 * free)
        self.in_use = 0
        self.max_group, self.max_group_rows = max_group, max_group_rows
        self.slots = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.busy = [None] * slots       # _Group running on the slot
        self.parked = [None] * slots     # _Group planned on the slot, waiting for memory
        self.waiting = collections.deque()
        self.finished = []
        self.stats = {"groups": 0, "max_group": 0, "max_busy": 0, "parked_polls": 0}
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    # ------------------------------------------------------------------ queue
    def submit(self, job):
        if job.arrival is None:
            job.arrival = self.now()
        self.waiting.append(job)

    def idle(self):
        return not self.waiting and all(g is None for g in self.busy) and all(g is None for g in self.parked)

    # --------------------------------------------------------------- planning
    def _take_group(self):
        grp = _Group(take_group(self.waiting, self.max_group, self.max_group_rows))
        self.stats["groups"] += 1
        self.stats["max_group"] = max(self.stats["max_group"], len(grp.jobs))
        return grp

    def _plan(self, grp, stream):
        entries = []
        with torch.cuda.stream(stream):
            for job in grp.jobs:
                bs = [ftlm.Basis(job.N, tz, job.bonds, stream=stream) for tz in ftlm.computed_two_sz(job.N)]
                grp.bases.append(bs)
                entries += [(b, self.R, job.seed, 0) for b in bs]
            grp.batch = ftlm.Batch(entries, self.M, self.dist, self.dtype, self.block, self.streams,
                                   stream=stream, lazy=True)
        tables = sum(b.table_bytes for bs in grp.bases for b in bs)
        outs = len(entries) * self.R * (2 * self.M * 8 + 4) + len(grp.jobs) * 4 * self.nT * 8
        grp.footprint = tables + grp.batch.workspace_bytes + outs

    def _fits(self, grp):
        if self.in_use + grp.footprint > self.budget and self.in_use > 0:
            return False
        free, _ = torch.cuda.mem_get_info(self.dev)
        return grp.footprint <= free or self.in_use == 0

    def _launch(self, grp, stream):
        now = self.now()
        with torch.cuda.stream(stream):
            results = grp.batch.run(stream)
            k = 0
            for job, bs in zip(grp.jobs, grp.bases):
                res = results[k:k + len(bs)]
                k += len(bs)
                out = torch.empty((4, self.nT), dtype=torch.float64, device=self.dev)
                ftlm.ftlm_thermo([b.two_sz for b in bs], [b.dim for b in bs], self.R, self.M,
                                 [r["theta"] for r in res], [r["weight"] for r in res], [r["m_eff"] for r in res],
                                 True, self.g, job.h, self.T, out[0], out[1], out[2], out[3], stream=stream)
                grp.outs.append(out)
                job.start = now
            grp.host = torch.empty((len(grp.jobs), 4, self.nT), dtype=torch.float64).pin_memory()
            for i, out in enumerate(grp.outs):
                grp.host[i].copy_(out, non_blocking=True)
            grp.meff_host = torch.empty((len(results), self.R), dtype=torch.int32).pin_memory()
            for i, r in enumerate(results):
                grp.meff_host[i].copy_(r["m_eff"], non_blocking=True)
            grp.event = torch.cuda.Event()
            grp.event.record(stream)
        self.in_use += grp.footprint

    def _retire(self, slot):
        grp = self.busy[slot]
        now = self.now()
        meff = grp.meff_host.numpy()
        k = 0
        for i, (job, bs) in enumerate(zip(grp.jobs, grp.bases)):
            job.result = grp.host[i].numpy().copy()
            job.finish = now
            job.updates = int(sum(int(meff[k + j].sum()) * b.updates for j, b in enumerate(bs)))
            k += len(bs)
            self.finished.append(job)
        # the group's work is complete: release in the slot's stream order, no wait
        stream = self.slots[slot]
        grp.batch.release(stream)
        for bs in grp.bases:
            for b in bs:
                b.release(stream)
        self.in_use -= grp.footprint
        self.busy[slot] = None

    # ------------------------------------------------------------------- loop
    def poll(self):
        """Retire finished groups, then plan and admit waiting work.  Returns True if
        anything changed."""
        changed = False
        for s in range(len(self.slots)):
            if self.busy[s] is not None and self.busy[s].event.query():
                self._retire(s)
                changed = True
        for s in range(len(self.slots)):
            if self.busy[s] is not None:
                continue
            if self.parked[s] is None and self.waiting:
                grp = self._take_group()
                self._plan(grp, self.slots[s])
                self.parked[s] = grp
                changed = True
            grp = self.parked[s]
            if grp is not None:
                if self._fits(grp):
                    self._launch(grp, self.slots[s])
                    self.busy[s], self.parked[s] = grp, None
                    changed = True
                else:
                    self.stats["parked_polls"] += 1
        self.stats["max_busy"] = max(self.stats["max_busy"], sum(g is not None for g in self.busy))
        return changed

    def run(self, jobs, arrivals=None, sleep=2e-4):
        """Serve `jobs`; arrivals[i] = seconds after the start at which job i is
        submitted (default: all at once).  Returns the finished jobs in order of
        completion."""
        arrivals = np.zeros(len(jobs)) if arrivals is None else np.asarray(arrivals, dtype=np.float64)
        order = np.argsort(arrivals, kind="stable")
        self.t0 = time.perf_counter()
        nxt = 0
        while nxt < len(jobs) or not self.idle():
            t = self.now()
            while nxt < len(jobs) and arrivals[order[nxt]] <= t:
                job = jobs[order[nxt]]
                job.arrival = float(arrivals[order[nxt]])
                self.submit(job)
                nxt += 1
            if not self.poll():
                time.sleep(sleep)
        return self.finished


def sector_rows(N):
    """Sum of the dimensions of the S^z >= 0 sectors of N spins 1/2."""
    return sum(math.comb(N, (N + tz) // 2) for tz in ftlm.computed_two_sz(N))


def take_group(waiting, max_group, max_rows):
    """Pop the next group off the FIFO `waiting` (a deque of jobs with .N): the head
    job always, then following jobs while the group has fewer than max_group jobs
    and its summed sector rows stay within max_rows.  Order is kept."""
    jobs = [waiting.popleft()]
    rows = sector_rows(jobs[0].N)
    while waiting and len(jobs) < max_group:
        r = sector_rows(waiting[0].N)
        if rows + r > max_rows:
            break
        jobs.append(waiting.popleft())
        rows += r
    return jobs


def poisson_jobs(n, rate, seed=4, sizes=(16, 18, 20, 22, 24, 26)):
    """Jobs and arrival times of inputs.serving_requests (seeded)."""
    reqs, arrivals = inputs.serving_requests(n, rate, seed, sizes)
    jobs = [Job(job_id=i, N=r["N"], bonds=r["bonds"], h=r["h"], seed=1000 + i) for i, r in enumerate(reqs)]
    return jobs, arrivals
