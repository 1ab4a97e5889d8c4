"""Request loop for FTLM jobs: chain-level continuous batching.

A job is one whole FTLM run of a cluster (sites N, bond list J_ij, Zeeman field h):
every S^z >= 0 sector (mirrored), R chains of M Lanczos steps each, then E, C, chi
and <S^z> on a temperature grid (Eq. 6-9; the field enters as -h S^z per sector).
Jobs arrive at any time.  The chains of every large sector on the device advance
together through one continuous flow (ftlm_flow_*): the flow visits its sectors in
waves of at most 256 MB of vectors (L2-sized) and runs a few Lanczos steps of each
wave with one multi-sector H.v launch per rank kind and one update launch per step,
whatever step each sector is at.  Between passes the loop admits the sectors of
waiting jobs, in arrival order, as long as their device memory fits in the flow's
workspace (so a job that arrives while others are at step 40 starts its step 1 in
the next pass), and collects the sectors that finished.  A job's small sectors run
all their steps in one persistent launch on a side stream as soon as the job
starts.  When every sector of a job is done, its thermodynamic sums are queued and
its results read back to pinned host memory.

Every unit of chains reduces its own tiles in a fixed order, so a job's results are
bit-identical whether it runs alone or among other jobs, and whenever it was
admitted.  The flow's Lanczos steps are queued on one stream and its Ritz steps run
on the flow's own stream; a job's thermodynamic sums and result copies go on a
third stream that waits for the job's outputs, so neither holds up the next
steps.  Sector tables are built on a high-priority side stream without a host
wait (the flow's stream and the small batches' stream wait for an event instead:
the host never blocks on the busy device to admit a job) and released in the sums
stream's order once the job's sums are queued.

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
    start: float = None         # host time its first sector was admitted
    finish: float = None        # host time its results were on the host
    result: np.ndarray = None   # (4, nT): E, C, chi, mag
    updates: int = 0            # H.v matrix-element updates its chains applied

    @property
    def latency(self):
        return None if self.finish is None else self.finish - self.arrival


class AdmissionQueue:
    """Waiting jobs in arrival order.  admit(start, try_add) starts the head job
    (start(job), once) and offers its sectors to try_add(job, index) one at a time;
    it stops at the first refusal (so no job's sector overtakes an earlier job's), or
    before starting a new job when max_jobs jobs are in flight."""

    def __init__(self, max_jobs=None):
        self.jobs = collections.deque()  # [job, sector indices not yet admitted, started]
        self.max_jobs = max_jobs
        self.in_flight = 0               # started jobs not yet finished

    def push(self, job, sectors):
        self.jobs.append([job, list(sectors), False])

    def admit(self, start, try_add):
        """Returns the (job, sector) pairs admitted by this call."""
        admitted = []
        while self.jobs:
            entry = self.jobs[0]
            job, rest, started = entry
            if not started:
                if self.max_jobs is not None and self.in_flight >= self.max_jobs:
                    break
                start(job)
                entry[2] = True
                self.in_flight += 1
            while rest:
                if not try_add(job, rest[0]):
                    return admitted
                admitted.append((job, rest.pop(0)))
            self.jobs.popleft()
        return admitted

    def finished(self):
        self.in_flight -= 1

    def __len__(self):
        return len(self.jobs)


class Engine:
    """Continuous-batching FTLM server on the current CUDA device.

    R, M            chains per sector and Lanczos steps
    dtype           vector storage (reductions are FP64)
    block           chains per unit
    T               temperature grid (host array); g the g-factor of chi
    memory_budget   bytes of the flow's workspace (default: DEFAULT_BUDGET, at most
                    60 % of the free device memory when the engine starts); tables
                    and the small sectors' batches come on top.  The workspace
                    bounds the sectors in flight: on the serving stream of 128 jobs
                    (N = 16 ... 26) a workspace that admits every waiting job at once
                    served fewer jobs per second (measured 11.7 / 12.6 / 13.8 / 13.5 /
                    12.4 jobs/s at 170 / 48 / 32 / 24 / 16 GB)
    max_units       units of chains the flow holds at once
    max_jobs        jobs in flight at once (None: as many as fit; 1: one at a time)
    steps_per_poll  Lanczos steps of each wave of the flow per admission pass
    depth           admission passes queued ahead of the device at most
    small_rows      sectors up to this dimension run in a job's own persistent batch
    flow_streams    wave streams of the flow (1..4)
    max_live_rows   rows of the flow's sectors in flight at most (None: no limit
                    beyond memory); the head job's sector is admitted into an empty
                    flow whatever its size.  A limit that still fills the GPU keeps
                    throughput and lets jobs finish in arrival order, instead of
                    all sharing the device until the end of the stream

    A job's sectors of at most small_rows rows run all their steps in one persistent
    launch (ftlm_batch, a CTA per block of chains) on a side stream as soon as the
    job starts; its larger sectors join the flow.
    """

    DEFAULT_BUDGET = 32 << 30  # bytes of the flow's workspace

    def __init__(self, R=8, M=80, dtype=torch.float32, block=8, T=None, g=2.0, dist=ftlm.GAUSS,
                 memory_budget=None, max_units=512, max_jobs=None, steps_per_poll=20, depth=2,
                 small_rows=1 << 15, flow_streams=4, max_live_rows=None):
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.R, self.M, self.dtype, self.block = R, M, dtype, block
        self.g, self.dist = g, dist
        T = np.asarray(T if T is not None else np.logspace(-2, 1, 200), dtype=np.float64)
        self.nT = len(T)
        self.T = torch.as_tensor(T, device=self.dev)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            memory_budget = int(min(self.DEFAULT_BUDGET, 0.6 * free))
        self.stream = torch.cuda.Stream(self.dev)   # the flow's Lanczos steps
        # sector tables (built without a host wait; the streams that use them wait
        # for an event), high priority so that they run as soon as SMs free up
        self.side = torch.cuda.Stream(self.dev, priority=-1)
        self.plans = torch.cuda.Stream(self.dev)    # batch plan uploads (copies only)
        self.small = torch.cuda.Stream(self.dev)    # the small sectors' persistent batches
        self.tstream = torch.cuda.Stream(self.dev)  # thermodynamic sums and result copies
        self.flow = ftlm.Flow(M, dist, dtype, block, max_units, memory_budget, stream=self.stream,
                              streams=flow_streams)
        self.queue = AdmissionQueue(max_jobs)
        self.steps_per_poll, self.depth, self.small_rows = steps_per_poll, depth, small_rows
        self.max_live_rows, self.live_rows = max_live_rows, 0
        self.running = {}     # id(job) -> state dict (jobs need not have distinct job_id)
        self.closing = []
        self.finished = []
        self.inflight = collections.deque()
        self.stats = {"polls": 0, "max_jobs_in_flight": 0, "max_units": 0, "refusals": 0, "small_sectors": 0,
                      "flow_sectors": 0, "host_s": {"admit": 0.0, "step": 0.0, "wait": 0.0, "collect": 0.0,
                                                     "tables": 0.0, "small_batch": 0.0}}
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, job):
        job._two_sz = ftlm.computed_two_sz(job.N)
        dims = [math.comb(job.N, (job.N + tz) // 2) for tz in job._two_sz]
        job._large = [k for k, d in enumerate(dims) if d > self.small_rows]
        self.queue.push(job, job._large)

    def idle(self):
        return not len(self.queue) and not self.running and not self.closing

    # ----------------------------------------------------------------- admission
    def _start(self, job):
        """Tables of every sector; the small sectors' batch on its own stream."""
        n = len(job._two_sz)
        st = {"job": job, "bases": [None] * n, "outs": [None] * n, "left": len(job._large), "batch": None,
              "small_ev": None}
        self.running[id(job)] = st
        t0 = time.perf_counter()
        st["bases"] = ftlm.Basis.sectors(job.N, job._two_sz, job.bonds, stream=self.side, wait=False)
        tables = torch.cuda.Event()
        tables.record(self.side)
        self.stream.wait_event(tables)  # the flow's next step call forks after this point
        small = [k for k in range(n) if k not in job._large]
        t1 = time.perf_counter()
        if small:
            self.small.wait_event(tables)
            with torch.cuda.stream(self.small):
                batch = ftlm.Batch([(st["bases"][k], self.R, job.seed, 0) for k in small], self.M, self.dist,
                                   self.dtype, self.block, 1, stream=self.plans)
                res = batch.run(self.small)
                ev = torch.cuda.Event()
                ev.record(self.small)
            for k, r in zip(small, res):
                st["outs"][k] = r
            st["batch"], st["small_ev"] = batch, ev
            self.stats["small_sectors"] += len(small)
        h = self.stats["host_s"]
        h["tables"] += t1 - t0
        h["small_batch"] += time.perf_counter() - t1
        job.start = self.now()
        if not job._large:
            self._close(st)

    def _try_add(self, job, k):
        st = self.running[id(job)]
        d = st["bases"][k].dim
        if self.max_live_rows is not None and self.live_rows > 0 and self.live_rows + d > self.max_live_rows:
            return False
        t = self.flow.add(st["bases"][k], self.R, job.seed, 0, owner=(id(job), k))
        if t is None:
            self.stats["refusals"] += 1
            if self.flow.status()["units"] == 0:
                raise RuntimeError(f"job {job.job_id}: a sector of N = {job.N} does not fit in an empty flow")
            return False
        self.stats["flow_sectors"] += 1
        self.live_rows += d
        return True

    # ------------------------------------------------------------------- collect
    def _collect(self):
        for ticket, out, (key, k) in self.flow.done(self.tstream):
            st = self.running[key]
            st["outs"][k] = out
            self.live_rows -= st["bases"][k].dim
            st["left"] -= 1
            if st["left"] == 0:
                self._close(st)

    def _close(self, st):
        job = st["job"]
        bs, outs = st["bases"], st["outs"]
        with torch.cuda.stream(self.tstream):
            if st["small_ev"] is not None:
                self.tstream.wait_event(st["small_ev"])
            res = torch.empty((4, self.nT), dtype=torch.float64, device=self.dev)
            ftlm.ftlm_thermo([b.two_sz for b in bs], [b.dim for b in bs], self.R, self.M,
                             [o["theta"] for o in outs], [o["weight"] for o in outs], [o["m_eff"] for o in outs],
                             True, self.g, job.h, self.T, res[0], res[1], res[2], res[3], stream=self.tstream)
            host = torch.empty((4, self.nT), dtype=torch.float64).pin_memory()
            host.copy_(res, non_blocking=True)
            meff = torch.empty((len(outs), self.R), dtype=torch.int32).pin_memory()
            for k, o in enumerate(outs):
                meff[k].copy_(o["m_eff"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.tstream)
        # the flow's last use of the tables precedes its outputs, which tstream waited for
        for b in bs:
            b.release(self.tstream)
        self.closing.append((job, ev, host, meff, [b.updates for b in bs], res, outs, st["batch"]))
        del self.running[id(job)]

    def _retire(self):
        keep = []
        for entry in self.closing:
            job, ev, host, meff, upd = entry[:5]
            if ev.query():
                job.result = host.numpy().copy()
                job.finish = self.now()
                m = meff.numpy()
                job.updates = int(sum(int(m[k].sum()) * upd[k] for k in range(len(upd))))
                if entry[7] is not None:  # its work is done: release in stream order, no device-wide wait
                    entry[7].release(self.tstream)
                self.finished.append(job)
                self.queue.finished()  # a job is in flight until its results are on the host
            else:
                keep.append(entry)
        self.closing = keep

    # ---------------------------------------------------------------------- loop
    def poll(self):
        """Admit, queue one pass of the flow, collect.  Returns True if it queued work.
        Host seconds spent admitting (tables, small batches), queueing passes,
        waiting for the device and collecting accumulate in stats["host_s"]."""
        t0 = time.perf_counter()
        self.queue.admit(self._start, self._try_add)
        self.stats["max_jobs_in_flight"] = max(self.stats["max_jobs_in_flight"], len(self.running) + len(self.closing))
        st = self.flow.status()
        self.stats["max_units"] = max(self.stats["max_units"], st["units"])
        busy = st["units"] > 0
        t1 = t2 = time.perf_counter()
        if busy:
            self.flow.step(self.steps_per_poll, self.stream)
            self.stats["polls"] += 1
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.inflight.append(ev)
            t2 = time.perf_counter()
            while len(self.inflight) > self.depth:
                self.inflight.popleft().synchronize()
        t3 = time.perf_counter()
        self._collect()
        self._retire()
        h = self.stats["host_s"]
        h["admit"] += t1 - t0
        h["step"] += t2 - t1
        h["wait"] += t3 - t2
        h["collect"] += time.perf_counter() - t3
        return busy

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
                if self.closing:
                    self.closing[0][1].synchronize()
                else:
                    time.sleep(sleep)
        return self.finished

    def close(self):
        self.flow.close()


def sector_rows(N):
    """Sum of the dimensions of the S^z >= 0 sectors of N spins 1/2."""
    return sum(math.comb(N, (N + tz) // 2) for tz in ftlm.computed_two_sz(N))


def poisson_jobs(n, rate, seed=4, sizes=(16, 18, 20, 22, 24, 26)):
    """Jobs and arrival times of inputs.serving_requests (seeded)."""
    reqs, arrivals = inputs.serving_requests(n, rate, seed, sizes)
    jobs = [Job(job_id=i, N=r["N"], bonds=r["bonds"], h=r["h"], seed=1000 + i) for i, r in enumerate(reqs)]
    return jobs, arrivals
