"""FTLM benchmark on one GB300 (or N independent replicas).

Workload (default): spin-1/2 icosidodecahedron, N = 30 sites, 60 bonds, J = 1,
S^z = 0 sector (D = 155 117 520); R = 8 Rademacher start vectors, M = 100 Lanczos
steps, FP32 vectors with FP64 reductions; thermodynamics on 200 temperatures in
[0.01, 10].  One step = one whole FTLM job through the C ABI: sector setup,
8 chains x 100 fused H.v + update launches, Ritz step, thermodynamic sums.

metric value = H.v matrix-element updates applied per second over the timed steps
(updates per H.v = D + 2 sum_b C(N-2, K-1), Eq. 10 at s = 1/2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload icosidodecahedron|ring34] [--mode auto|clt|cr] [--dtype f32|f64]

--impl reference times the FP64 CPU oracle on the same workload (bounded row
samples of its H.v) on the host cores.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·v Gupdates/s & %HBM roofline at N=30 S^z=0; FTLM jobs/s, p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0
WORKLOADS = {
    "icosidodecahedron": dict(N=30, desc="icosidodecahedron N=30 S^z=0 (D=155117520, 60 bonds, J=1)",
                              paper=(124.0, "paper GPU-CLT, 124 s for this job on RTX 4000 Ada (Table 3)")),
    "ring34": dict(N=34, desc="ring N=34 S^z=0 (D=2333606220, 34 bonds, J=1)"),
    # general local spin, the icosahedron systems of Table 3 (R = 24, N_L = 100)
    "icosahedron_s1": dict(N=12, two_s=2, sectors="all", R=24, M=100,
                           desc="spin-1 icosahedron N=12 (30 bonds, J=1), every S^z >= 0 sector (mirrored)",
                           paper=(0.21, "paper GPU-CR, 0.21 s for this job on RTX 4000 Ada (Table 3)")),
    "icosahedron_s3/2": dict(N=12, two_s=3, sectors="all", R=24, M=100,
                             desc="spin-3/2 icosahedron N=12 (30 bonds, J=1), every S^z >= 0 sector (mirrored)",
                             paper=(14.6, "paper GPU-CR, 14.6 s for this job on RTX 4000 Ada (Table 3)")),
    "icosahedron_s2": dict(N=12, two_s=4, sectors="zero", R=24, M=100,
                           desc="spin-2 icosahedron N=12 (30 bonds, J=1) S^z=0 (D=19611175)",
                           paper=(34.8, "paper GPU-CR, 34.8 s for this job on RTX 4000 Ada (Table 3)")),
    "icosahedron_s3": dict(N=12, two_s=6, sectors="zero", R=8, M=100,
                           desc="spin-3 icosahedron N=12 (30 bonds, J=1) S^z=0 (D=786588243)"),
    # a smaller sector of the same kind (4-regular-like random graph) for detailed
    # counter captures that must stay within a few GB of device memory
    "random28": dict(N=28, desc="random graph N=28 (degrees 3-5, J~U[0.5,1.5], seed 28) S^z=0 (D=40116600)"),
    "serving": dict(N=26, desc="Poisson stream (200 jobs/s, seeded) of FTLM jobs: rings or 2-leg ladders, N uniform "
                               "in {16,...,26} even, J~U[0.2,1.5], h~U[0,2], every S^z sector, R=8 Gaussian, M=80, "
                               "f32 vectors"),
    "precision": dict(N=24, sectors="all", R=64, M=150,
                      desc="4x6 periodic J1-J2 lattice N=24 (J1=1, J2=0.5, 96 bonds), every S^z >= 0 sector, "
                           "R=64 Rademacher, M=150: FP32 vs FP64 vectors, sigma_emp over seeds, ghost counts"),
    "clusters256": dict(N=22, desc="256 random clusters, N uniform in {18,20,22}, degrees 3-5, J~U[0.5,1.5], "
                                   "every S^z >= 0 sector (mirrored), R=16 Rademacher, M=100, f32 vectors"),
}
PROFILES = os.path.join(ROOT, "profiles")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=list(WORKLOADS), default="icosidodecahedron")
    p.add_argument("--mode", choices=["auto", "clt", "cr"], default="auto")
    p.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    p.add_argument("--R", type=int, default=0, help="chains per sector (default: the workload's)")
    p.add_argument("--M", type=int, default=0, help="Lanczos steps (default: the workload's)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--jobs", type=int, default=128, help="serving: requests in the timed stream")
    p.add_argument("--steps-per-poll", type=int, default=20,
                   help="serving: Lanczos steps of each flow wave between admission passes of the request loop")
    p.add_argument("--seeds", type=int, default=8, help="precision: independent FTLM runs for sigma_emp")
    p.add_argument("--clusters", type=int, default=256, help="clusters256: use the first n clusters (profiling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="default workload: skip the FP64 one-vector job and the serving stream")
    p.add_argument("--serving-jobs", type=int, default=64, help="requests of the serving stream in the default line")
    p.add_argument("--live-rows", type=int, default=0,
                   help="serving: rows of flow sectors in flight at most (0: no limit beyond memory)")
    p.add_argument("--two-sz", type=int, default=0, help="sector 2 S^z of single-sector workloads (profiling)")
    p.add_argument("--schedule", choices=["auto", "one_walk", "split"], default="auto",
                   help="walks of the Lanczos H.v (ftlm_basis_set_schedule)")
    p.add_argument("--rows-per-tile", type=int, default=0, help="high patterns per tile of the split's walk B")
    p.add_argument("--hv-only", action="store_true",
                   help="time plain ftlm_hv launches on the workload (kernel microbenchmark)")
    p.add_argument("--block", type=int, default=0,
                   help="with --hv-only: vectors per launch (ftlm_hv_block, 1/4/8/16); with clusters256: "
                        "fixed block width instead of the autotuner")
    return p.parse_args()


def bonds_of(name):
    from paper_2605_26261_gb300 import inputs

    if name == "icosidodecahedron":
        return inputs.icosidodecahedron()
    if name == "random28":
        return inputs.random_graph(28, seed=28)
    if name.startswith("icosahedron_"):
        return inputs.icosahedron()
    if name == "precision":
        return inputs.square_j1j2(4, 6, 1.0, 0.5)
    if name == "clusters256":  # the CPU sample: the first N = 22 cluster of the set
        return next(b for N, b in inputs.cluster_set(256, seed=256) if N == 22)
    if name == "serving":  # the CPU sample: the first N = 26 request of the stream
        reqs, _ = inputs.serving_requests(128, 200.0, seed=4)
        return next(r["bonds"] for r in reqs if r["N"] == 26)
    return inputs.ring(34)


def sector_model_bytes(updates, D, dtype_bytes, clt, lanczos=True, B=1):
    """Algorithmic bytes of one H.v launch on B interleaved vectors under the
    sector model: every gather of the B entries of a source row costs whole 32-byte
    sectors (ceil(B * size / 32) of them), plus the row streams x[t] and y[t] (and
    the u_{j-1} read of the fused Lanczos epilogue) for B vectors; CLT adds one
    32-byte sector per table lookup and the 4-byte basis[t] read."""
    n_off = updates - D
    sectors = -(-B * dtype_bytes // 32)
    b = 32 * sectors * n_off + (2 + (1 if lanczos else 0)) * dtype_bytes * B * D
    if clt:
        b += 32 * n_off + 4 * D
    return b


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Device sources of each H.v kernel family: a committed ncu summary holds DRAM
# traffic for the sources it was taken on.
KERNEL_SOURCES = {
    "hv": ("hv.cu", "walka.cu", "walkb.cu", "epi.cuh", "rows.cuh", "vec.cuh", "reduce.cuh", "ftlm_internal.cuh"),
    "spin": ("spin.cu", "spin_rows.cuh", "epi.cuh", "vec.cuh", "reduce.cuh", "ftlm_internal.cuh"),
}


def kernel_fingerprint(family="hv"):
    """Hash of the family's device sources without their comments and blank lines
    (an edit of a comment leaves the compiled kernels, and so the counters, as they
    were)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2605_26261_gb300", "csrc")
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(d, f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = line.split("//", 1)[0].rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_bytes_per_row(workload, mode_name, dtype, schedule, family="hv"):
    """DRAM bytes per sector row of one Lanczos H.v step (all its launches) from a
    committed ncu summary (profiles/*.md) taken on the current sources of the kernel
    family, for this workload, rank mode, dtype and H.v schedule; else None.  The
    captures run on smaller sectors of the same cluster (a few GB on the device) and
    give bytes per row, which the caller scales by the sector dimension."""
    import glob

    want = kernel_fingerprint(family)
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        text = open(path).read()
        fp = re.search(rf"kernel_fingerprint\[{family}\]:\s*(\w+)", text)
        if not fp or fp.group(1) != want:
            continue
        m = re.search(rf"dram_bytes_per_row\[{re.escape(workload)},{mode_name},{dtype},{schedule}\]:\s*([0-9.eE+]+)",
                      text)
        if m:
            return float(m.group(1))
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        return False

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        load = [s for s in sm if smax and s > 0.3 * smax] or sm
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_over_ranks(updates, ms, device, world):
    """Whole-job totals over replicas: updates summed over ranks, the timed region's
    duration taken as the maximum over ranks."""
    import torch
    import torch.distributed as dist

    if world <= 1:
        return float(updates), float(ms)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return u.item(), t.item()


# ---------------------------------------------------------------------- oracle
class OracleSampler:
    """Times the FP64 CPU oracle's H.v on bounded, evenly spread samples of rows."""

    def __init__(self, workload, seed=5):
        import math

        import oracle as o

        self.o = o
        N = WORKLOADS[workload]["N"]
        self.N, self.two_s = N, WORKLOADS[workload].get("two_s", 1)
        # beyond these sizes the oracle cannot enumerate the S^z = 0 sector in host memory
        self.ok = N <= 30 if self.two_s == 1 else (self.two_s + 1) ** N <= 5**12
        if not self.ok:
            return
        self.bonds = bonds_of(workload)
        if self.two_s == 1:
            self.b = o.basis(N, N // 2)
            self.D = len(self.b)
            self.upd_per_row = (self.D + 2 * len(self.bonds[2]) * math.comb(N - 2, N // 2 - 1)) / self.D
        else:
            A = o.spin.sector_A(N, self.two_s, (N * self.two_s) % 2)
            self.b = o.spin.basis(N, self.two_s, A)
            self.D = len(self.b)
            self.upd_per_row = o.spin.nnz(N, self.two_s, A, len(self.bonds[2])) / self.D
        self.x = np.random.default_rng(seed).standard_normal(self.D)

    def _run(self, rows_per_chunk, offset, passes=1):
        starts = (np.linspace(0, self.D - rows_per_chunk - 64, 64) + offset).astype(np.int64)
        out = np.empty(rows_per_chunk)
        t = time.perf_counter()
        for _ in range(passes):
            for s in starts:
                if self.two_s == 1:
                    self.o.hv_range(self.bonds, self.b, self.x, int(s), int(s) + rows_per_chunk, out=out)
                else:
                    self.o.spin.hv_range(self.N, self.two_s, self.bonds, self.b, self.x, int(s),
                                         int(s) + rows_per_chunk, out=out)
        return time.perf_counter() - t, passes * 64 * rows_per_chunk

    def sample(self, seconds, offset=0, single_thread_share=0.2):
        """OpenMP over all host cores for about `seconds`, and one thread for a
        share of it (the oracle's two builds of the CPU baseline plan)."""
        self._run(256, offset)  # thread pool and first touch
        t0, n0 = self._run(1024, offset)
        want = seconds / (t0 / n0)  # rows that take about `seconds`
        rows_chunk = int(max(256, min(want / 64, (self.D - 128) // 64)))
        passes = max(1, int(want / (64 * rows_chunk)))
        t1, n1 = self._run(rows_chunk, offset, passes)
        cores = self.o.num_threads()
        out = {"updates_per_s": n1 * self.upd_per_row / t1, "rows": n1, "seconds": t1, "cores": cores, "D": self.D}
        if single_thread_share > 0 and cores > 1:
            self.o.set_num_threads(1)
            try:
                chunk1 = max(64, int(rows_chunk * single_thread_share / cores))
                t2, n2 = self._run(chunk1, offset)
                out["single_thread_updates_per_s"] = n2 * self.upd_per_row / t2
            finally:
                self.o.set_num_threads(cores)
        return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    samples = []
    sampler = OracleSampler(args.workload)
    if not sampler.ok:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the FP64 CPU oracle cannot enumerate this sector in host memory"}))
        return
    per_step = max(1.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        res = sampler.sample(per_step, offset=i)
        if i >= args.warmup:
            samples.append(res["updates_per_s"])
    v = statistics.median(samples) / 1e9
    sample = (f"FP64 oracle H.v (binary-search index map) on {res['rows']} rows per step, 64 evenly "
              f"spread chunks of the D={res['D']} sector; median of {args.steps} steps")
    unit = "Gupdates/s"
    if args.workload == "serving":
        # the request loop's unit: the oracle's H.v rate over the mean updates of a
        # job of the same request stream (every sector, 8 chains of min(80, D) steps)
        import math

        from paper_2605_26261_gb300 import inputs

        reqs, _ = inputs.serving_requests(args.jobs, 200.0, seed=4)
        tot = 0
        for r in reqs:
            N, nb = r["N"], len(r["bonds"][2])
            for K in range((N + 1) // 2, N + 1):
                D = math.comb(N, K)
                tot += 8 * min(80, D) * (D + 2 * nb * math.comb(N - 2, K - 1))
        v = v * 1e9 / (tot / len(reqs))
        unit = "jobs/s"
        sample += f"; jobs/s = that rate / {tot / len(reqs):.3e} updates per job of the request stream"
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["desc"], "parallelism": "host threads"},
        "cpu_baseline": {"value": v, "unit": unit, "cores": res["cores"], "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2605_26261_gb300 import ftlm, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    wl = WORKLOADS[args.workload]
    N, two_s = wl["N"], wl.get("two_s", 1)
    bonds = bonds_of(args.workload)
    mode = {"auto": ftlm.RANK_AUTO, "clt": ftlm.RANK_CLT, "cr": ftlm.RANK_CR}[args.mode]
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    R = args.R or wl.get("R", 8)
    M = args.M or wl.get("M", 100)
    sectors = [args.two_sz] if wl.get("sectors", "zero") == "zero" else ftlm.computed_two_sz(N, two_s)
    T_host = inputs.log_t_grid(200)
    T = torch.as_tensor(T_host, device=dev)

    sched = {"auto": ftlm.HV_AUTO, "one_walk": ftlm.HV_ONE_WALK, "split": ftlm.HV_SPLIT}[args.schedule]

    def basis(tz, bl=bonds):
        b = ftlm.Basis(N, tz, bl, mode, two_s=two_s)
        if sched != ftlm.HV_AUTO or args.rows_per_tile:
            b.set_schedule(sched, args.rows_per_tile)
        return b

    info = {}  # two_sz -> (D, updates per H.v, rank mode)
    work_bytes = 0
    for tz in sectors:
        with basis(tz) as b:
            info[tz] = (b.dim, b.updates, b.mode)
            work_bytes = max(work_bytes, ftlm.ftlm_lanczos_workspace_bytes(b.handle, R, M, dt))
    work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
    outs = {tz: (torch.empty((R, M), dtype=torch.float64, device=dev),
                 torch.empty((R, M), dtype=torch.float64, device=dev),
                 torch.empty(R, dtype=torch.int32, device=dev)) for tz in sectors}
    obs = {k: torch.empty_like(T) for k in ("E", "C", "chi", "mag")}
    # a job over several sectors runs as one batch (all sectors advance together);
    # one sector runs through ftlm_lanczos
    batch_block = args.block or (16 if R % 16 == 0 else (8 if R % 8 == 0 else 4))

    def job(bl, release_stream):
        if len(sectors) == 1:
            b = basis(sectors[0], bl)
            th, w, me = outs[sectors[0]]
            ftlm.ftlm_lanczos(b.handle, R, M, 1, ftlm.RADEMACHER, dt, work, th, w, me)
            b.release(release_stream)  # tables go back to the pool after the chains, no wait
        else:
            bs = [basis(tz, bl) for tz in sectors]
            batch = ftlm.Batch([(b, R, 1, 0) for b in bs], M, ftlm.RADEMACHER, dt, batch_block)
            for tz, r in zip(sectors, batch.run()):
                for dst, k in zip(outs[tz], ("theta", "weight", "m_eff")):
                    dst.copy_(r[k])
            batch.release(release_stream)
            for b in bs:
                b.release(release_stream)
        ftlm.ftlm_thermo(sectors, [info[tz][0] for tz in sectors], R, M, [outs[tz][0] for tz in sectors],
                         [outs[tz][1] for tz in sectors], [outs[tz][2] for tz in sectors], True, 2.0, 0.0, T,
                         obs["E"], obs["C"], obs["chi"], obs["mag"])

    def step():
        job(bonds, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ftlm.ftlm_profile_read()  # drop anything recorded so far
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ftlm.ftlm_profile_enable(True)
    launches0 = ftlm.ftlm_launch_count()
    with ClockSampler(local) as clocks:
        ev[0].record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    ftlm.ftlm_profile_enable(False)
    launches_timed = ftlm.ftlm_launch_count() - launches0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    hv_n, hv_vec, hv_ms, up_n, up_ms = ftlm.ftlm_profile_read()
    updates_step = sum(int(outs[tz][2].sum().item()) * info[tz][1] for tz in sectors)

    all_updates, max_ms = aggregate_over_ranks(updates_step * args.steps, total_ms, dev, world)
    value = all_updates / (max_ms / 1e3) / 1e9

    # end-to-end through the public API with host buffers (one job per step):
    # bond list and T grid from (pinned) host memory, results read back to pinned host memory
    e2e = None
    if rank == 0 or world == 1:
        T_pin = torch.as_tensor(T_host).pin_memory()
        host = {tz: [torch.empty((R, M), dtype=torch.float64).pin_memory(),
                     torch.empty((R, M), dtype=torch.float64).pin_memory(),
                     torch.empty(R, dtype=torch.int32).pin_memory()] for tz in sectors}
        obs_host = [torch.empty(200, dtype=torch.float64).pin_memory() for _ in range(3)]
        bl_host = tuple(np.ascontiguousarray(a) for a in bonds)
        n_e2e = max(1, min(2, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            T.copy_(T_pin, non_blocking=True)
            job(bl_host, stream)
            for tz in sectors:
                for h_, d_ in zip(host[tz], outs[tz]):
                    h_.copy_(d_, non_blocking=True)
            for h_, k in zip(obs_host, ("E", "C", "chi")):
                h_.copy_(obs[k], non_blocking=True)
            torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / n_e2e
        h2d = sum(a.nbytes for a in bl_host) * len(sectors) + T_pin.numel() * 8
        d2h = len(sectors) * (2 * R * M * 8 + R * 4) + 3 * 200 * 8
        e2e_updates = sum(int(host[tz][2].sum()) * info[tz][1] for tz in sectors)
        e2e = {"value": e2e_updates / wall / 1e9, "unit": "Gupdates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * wall}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # the rest of the metric on the same GPU: the one-vector FP64 path on this job and
    # the request loop of the serving configuration
    extras = None
    if world == 1 and args.workload == "icosidodecahedron" and not args.no_extras and len(sectors) == 1:
        extras = {"fp64_b1": fp64_b1_job(N, bonds, mode, R, M, T, value), "serving": None}
        sv = serve_stream(args.serving_jobs, args.steps_per_poll, 3, local, live_rows=args.live_rows)
        sv.pop("_done"), sv.pop("_jobs")
        sv["workload"] = WORKLOADS["serving"]["desc"]
        extras["serving"] = sv
        del work
        # the other configurations, one measurement each
        extras["precision"] = precision_job(T)
        extras["clusters256"] = clusters_step(T)
        extras["ring34"] = ring34_job(T)

    peak, peak_src = peak_hbm()
    block = round(hv_vec / max(hv_n, 1))  # vectors per H.v launch (one block width per run)
    vsize = 4 if dt == torch.float32 else 8
    # algorithmic bytes of every H.v launch of the timed steps: per sector and block
    # of chains, min(M, D) launches of the sector model's bytes
    plan = []
    left = R
    if len(sectors) > 1:  # the batch: units of batch_block chains
        plan = [batch_block] * (-(-R // batch_block))
        left = 0
    for w_ in (16, 8, 4):
        if w_ <= (8 if dt == torch.float32 else 4):
            while left >= w_:
                plan.append(w_)
                left -= w_
    plan += [1] * left
    alg_total, launches_model, upd_total = 0.0, 0, 0
    for tz in sectors:
        D_, upd_, mode_ = info[tz]
        for w_ in plan:
            n_l = min(M, D_) * args.steps
            alg_total += n_l * sector_model_bytes(upd_, D_, vsize, mode_ == ftlm.RANK_CLT, B=w_)
            upd_total += n_l * w_ * upd_
            launches_model += n_l
    hv_s = hv_ms / 1e3
    D0, upd0, mode0 = info[sectors[0]]
    clt = mode0 == ftlm.RANK_CLT
    mode_name = "clt" if clt else "cr"
    family = "spin" if two_s > 1 else "hv"
    hv_avg_s = hv_s / max(hv_n, 1)
    # the walks the Lanczos H.v steps used (one launch, or walk A + walk B)
    schedule = "one_walk"
    if len(sectors) == 1 and two_s == 1 and mode0 == ftlm.RANK_CR:
        with basis(sectors[0]) as b_:
            if ftlm.ftlm_basis_hv_schedule(b_.handle, block, dt) == ftlm.HV_SPLIT:
                schedule = "split"
    kname = ("ms_hv_kernel" if len(sectors) > 1 else
             ("hv_kernel" if schedule == "one_walk" else "hv_kernel (walk A) + walk_b_kernel")
             if two_s == 1 else "hv_spin_kernel")
    # DRAM traffic of one H.v step from the committed capture of the current sources
    # (bytes per row on smaller sectors of the same cluster, scaled by D)
    bpr = (profiled_bytes_per_row(args.workload, mode_name, args.dtype, schedule, family)
           if len(sectors) == 1 else None)
    traffic = bpr * D0 if bpr else None
    # compulsory bytes of one step: x[t] read, u_{j-1} read and y written once per
    # row (B values each), plus the per-tile alpha sums of CR launches
    tiles = 0 if clt or len(sectors) > 1 else (D0 + 31) // 32
    compulsory = 3 * D0 * block * vsize + tiles * block * 8 if len(sectors) == 1 else None
    if traffic and hv_n:
        achieved, basis_note = traffic / hv_avg_s / 1e9, ("DRAM read + write bytes per H.v step (ncu capture "
                                                          "of the current sources, profiles/) / event-timed step")
    elif compulsory and hv_n:
        achieved, basis_note = compulsory / hv_avg_s / 1e9, ("compulsory bytes per H.v step (a lower bound on "
                                                             "its DRAM traffic: no capture of the current sources) "
                                                             "/ event-timed step")
    else:
        achieved, basis_note = None, "no per-step traffic for this workload"
    n_off = (upd0 - D0) * block  # off-diagonal gathers of one step (each row of B values)
    # the read rate that bounds the gathers: L2 (a 64 MB buffer, L2-resident) measured
    # here with the library's probe; gathers and row streams of one step move through L2
    l2_peak = peak_rows = peak_runs = None
    if hv_n:
        probe = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
        l2_peak = ftlm.ftlm_probe_read_bandwidth(probe, 40)
        peak_rows = ftlm.ftlm_probe_gather_bandwidth(probe, 1, 40)
        peak_runs = ftlm.ftlm_probe_gather_bandwidth(probe, 32, 40)
        del probe
    gather_bytes = n_off // block * 32 * max(1, block * vsize // 32)
    stream_bytes = (6 if schedule == "split" else 3) * D0 * block * vsize
    l2_achieved = (gather_bytes + stream_bytes) / hv_avg_s / 1e9 if hv_n else None
    # the gathers' own roofline: every bond has the same number of off-diagonal terms
    # at s = 1/2, so the high-high bonds' share of the gathers is their share of the
    # bonds; those move in runs of 32 consecutive rows per warp (1 KB), the others as
    # rows of their own; the fastest a step could gather at the probed rates
    gather_roof = None
    if hv_n and two_s == 1 and len(sectors) == 1 and peak_rows and peak_runs:
        lo_block = min(N, 14)
        n_hh = sum(1 for i, j in zip(bonds[0], bonds[1]) if min(i, j) >= lo_block)
        g_runs = gather_bytes * n_hh / len(bonds[0])
        t_min = (gather_bytes - g_runs) / (peak_rows * 1e9) + g_runs / (peak_runs * 1e9)
        gather_roof = {"peak_rows": peak_rows, "peak_runs_1KB": peak_runs, "unit": "GB/s",
                       "t_min_ms": 1e3 * t_min, "frac": t_min / hv_avg_s,
                       "basis": "gather bytes of one step at ftlm_probe_gather_bandwidth's rates on a 64 MB "
                                "L2-resident buffer (scattered 32-byte rows for the bonds touching the low digit "
                                f"block, 1 KB runs for the {n_hh} high-high bonds), this run; frac = that time / "
                                "the event-timed step"}
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak if achieved else None, "traffic": traffic,
        "achieved_basis": basis_note,
        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
        "kernel": f"{kname}<{'float' if dt == torch.float32 else 'double'}, {mode_name.upper()}, lanczos, "
                  f"B={block}>" + (" (one H.v step: both walks + alpha)" if schedule == "split" else ""),
        "schedule": schedule,
        "compulsory_bytes_per_launch": compulsory,
        "traffic_over_compulsory": traffic / compulsory if (traffic and compulsory) else None,
        "sector_model_bytes_per_launch": alg_total / max(hv_n, 1),
        "sector_model_ratio": (alg_total / hv_s / 1e9 / peak) if hv_n else None,
        "sector_model": "32 B per gathered row of B values + row streams (x, y, u_{j-1}); counts every gather "
                        "as a DRAM sector, so L2 hits push the ratio above 1: not a fraction of a roofline",
        "l2": {"achieved": l2_achieved, "peak": l2_peak, "unit": "GB/s",
               "frac": l2_achieved / l2_peak if (l2_achieved and l2_peak) else None,
               "bytes_per_launch": gather_bytes + stream_bytes,
               "basis": "gathers (one 32-byte sector per row of B values per off-diagonal term) + the row streams "
                        "of the step's walks, through L2 / event-timed step; peak = ftlm_probe_read_bandwidth on "
                        "a 64 MB L2-resident buffer, this run",
               "gathers": gather_roof},
        "hv_launches": hv_n, "sector_block_steps": launches_model, "vectors_per_launch": block,
        "hv_ms_avg": hv_avg_s * 1e3,
        "hv_Gupdates_per_s": upd_total / hv_s / 1e9 if hv_n else None,
        "update_ms_avg": up_ms / max(up_n, 1),
    }
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        sampler = OracleSampler(args.workload)
        res = sampler.sample(args.cpu_seconds) if sampler.ok else None
        if res:
            cpu = {"value": res["updates_per_s"] / 1e9, "unit": "Gupdates/s", "cores": res["cores"],
                   "kind": "oracle",
                   "sample": f"FP64 oracle H.v (binary-search index map) on {res['rows']} rows: 64 evenly "
                             f"spread chunks of the D={res['D']} sector, {res['seconds']:.1f} s",
                   "single_thread_value": res.get("single_thread_updates_per_s", 0.0) / 1e9}
    paper = wl.get("paper")
    vs = None
    if paper:  # the paper's best GPU wall time for this exact job (Table 3), as Gupdates/s
        paper_updates = sum(R * min(M, info[tz][0]) * info[tz][1] for tz in sectors)
        vs = value / (paper_updates / paper[0] / 1e9)
    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": vs, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": (wl["desc"] if sectors == [0] or len(sectors) > 1 else
                                re.sub(r"\(D=\d+", f"(D={D0}", wl["desc"].replace("S^z=0", f"2S^z={sectors[0]}"))) +
                               f", R={R} Rademacher, M={M}, 200-point T grid",
                   "sectors": len(sectors), "rank_mode": mode_name.upper(),
                   "vectors": f"{args.dtype} storage, FP64 reductions",
                   "l2": f"inputs larger than L2 (two blocks of {plan[0]} vectors of D={D0} elements, "
                         f"{2 * plan[0] * D0 * vsize / 1e9:.2f} GB)" if 2 * plan[0] * D0 * vsize > 129e6
                   else f"largest sector's two blocks ({2 * plan[0] * D0 * vsize / 1e6:.0f} MB) fit in L2",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "vs_baseline_ref": paper[1] if paper else None},
        "job_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                   "jobs_per_s": world * args.steps / (max_ms / 1e3),
                   "note": "the timed steps: this one job repeated back to back (not request latencies; "
                           "those are under serving)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_timed, "clocks": clocks.summary(),
    }
    if extras is not None:
        line.update(extras)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def fp64_b1_job(N, bonds, mode, R, M, T, value_f32):
    """The same FTLM job with FP64 vectors and every chain on its own (block width 1):
    the plain one-vector FP64 path, timed with CUDA events (one untimed short run first)."""
    import torch

    from paper_2605_26261_gb300 import ftlm

    dev = T.device
    ftlm.ftlm_lanczos_set_block(1)
    try:
        with ftlm.Basis(N, 0, bonds, mode) as b:
            work = torch.empty(ftlm.ftlm_lanczos_workspace_bytes(b.handle, R, M, torch.float64), dtype=torch.uint8,
                               device=dev)
            th = torch.empty((R, M), dtype=torch.float64, device=dev)
            w = torch.empty_like(th)
            me = torch.empty(R, dtype=torch.int32, device=dev)
            obs = [torch.empty_like(T) for _ in range(4)]
            ftlm.ftlm_lanczos(b.handle, R, 3, 1, ftlm.RADEMACHER, torch.float64, work, th, w, me)
            torch.cuda.synchronize()
            ftlm.ftlm_profile_read()
            ftlm.ftlm_profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ftlm.ftlm_lanczos(b.handle, R, M, 1, ftlm.RADEMACHER, torch.float64, work, th, w, me)
            ftlm.ftlm_thermo([0], [b.dim], R, M, [th], [w], [me], True, 2.0, 0.0, T, *obs)
            e1.record()
            torch.cuda.synchronize()
            ftlm.ftlm_profile_enable(False)
            hv_n, _, hv_ms, _, _ = ftlm.ftlm_profile_read()
            ms = e0.elapsed_time(e1)
            upd = int(me.sum().item()) * b.updates
            used = ftlm.ftlm_basis_hv_schedule(b.handle, 1, torch.float64)
    finally:
        ftlm.ftlm_lanczos_set_block(0)
    v = upd / (ms / 1e3) / 1e9
    return {"value": v, "unit": "Gupdates/s", "job_ms": ms, "hv_ms_avg": hv_ms / max(hv_n, 1),
            "schedule": "split" if used == ftlm.HV_SPLIT else "one_walk",
            "f32_block8_over_fp64_b1": value_f32 / v,
            "note": "same job, FP64 vectors, every chain alone (ftlm_lanczos_set_block(1))"}


def ring34_job(T):
    """The N = 34 ring S^z = 0 sector (D = 2 333 606 220, CR), 8 Rademacher chains as one
    FP32 block, M = 100: one whole job (sector setup, Lanczos, Ritz, thermodynamic sums)
    timed with CUDA events after a 3-step warm-up job."""
    import torch

    from paper_2605_26261_gb300 import ftlm

    dev = T.device
    torch.cuda.empty_cache()
    bonds = bonds_of("ring34")
    R, M = 8, 100
    with ftlm.Basis(34, 0, bonds, ftlm.RANK_CR) as b:
        work = torch.empty(ftlm.ftlm_lanczos_workspace_bytes(b.handle, R, M, torch.float32), dtype=torch.uint8,
                           device=dev)
        D, per_hv = b.dim, b.updates
        used = ftlm.ftlm_basis_hv_schedule(b.handle, 8, torch.float32)
    th = torch.empty((R, M), dtype=torch.float64, device=dev)
    w = torch.empty_like(th)
    me = torch.empty(R, dtype=torch.int32, device=dev)
    obs = [torch.empty_like(T) for _ in range(4)]

    def job(m):
        with ftlm.Basis(34, 0, bonds, ftlm.RANK_CR) as b:
            ftlm.ftlm_lanczos(b.handle, R, m, 1, ftlm.RADEMACHER, torch.float32, work, th, w, me)
            ftlm.ftlm_thermo([0], [D], R, M, [th], [w], [me], True, 2.0, 0.0, T, *obs)

    job(3)
    torch.cuda.synchronize()
    ftlm.ftlm_profile_read()
    ftlm.ftlm_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    job(M)
    e1.record()
    torch.cuda.synchronize()
    ftlm.ftlm_profile_enable(False)
    hv_n, hv_vec, hv_ms, up_n, up_ms = ftlm.ftlm_profile_read()
    ms = e0.elapsed_time(e1)
    upd = int(me.sum().item()) * per_hv
    del work
    torch.cuda.empty_cache()
    return {"value": upd / (ms / 1e3) / 1e9, "unit": "Gupdates/s", "job_ms": ms,
            "hv_ms_avg": hv_ms / max(hv_n, 1), "update_ms_avg": up_ms / max(up_n, 1),
            "schedule": "split" if used == ftlm.HV_SPLIT else "one_walk",
            "workload": WORKLOADS["ring34"]["desc"] + ", R=8 Rademacher (one block of 8 f32 vectors), M=100",
            "vectors_gb": 2 * D * R * 4 / 1e9}


def clusters_step(T):
    """The batched-cluster configuration in brief: every S^z >= 0 sector of the 256
    random clusters in one batch (R = 16 Rademacher, M = 100, FP32, the default plan:
    blocks of 8 chains, 2048-row H.v tiles), then the 256 thermodynamic sums; one
    untimed run, then one run timed with CUDA events."""
    import torch

    from paper_2605_26261_gb300 import ftlm, inputs

    R, M = 16, 100
    clusters = inputs.cluster_set(256, seed=256)
    bases = [[ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)] for N, bonds in clusters]
    entries = [(b, R, 1 + c, 0) for c, bs in enumerate(bases) for b in bs]
    outs = [[torch.empty_like(T) for _ in range(4)] for _ in clusters]
    with ftlm.Batch(entries, M, ftlm.RADEMACHER, torch.float32, 8) as batch:
        def step():
            res = batch.run()
            k = 0
            for c, bs in enumerate(bases):
                r = res[k:k + len(bs)]
                k += len(bs)
                ftlm.ftlm_thermo([b.two_sz for b in bs], [b.dim for b in bs], R, M, [x["theta"] for x in r],
                                 [x["weight"] for x in r], [x["m_eff"] for x in r], True, 2.0, 0.0, T, *outs[c])
            return res

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        upd = sum(int(r["m_eff"].sum().item()) * b.updates for (b, _, _, _), r in zip(entries, res))
    for bs in bases:
        for b in bs:
            b.close()
    return {"step_ms": ms, "clusters_per_s": len(clusters) / (ms / 1e3), "Gupdates_per_s": upd / (ms / 1e3) / 1e9,
            "sectors": len(entries), "workload": WORKLOADS["clusters256"]["desc"],
            "plan": "blocks of 8 chains, 2048-row H.v tiles, 16384-row streaming tiles (the autotuner's choice "
                    "on this set), eager (not graph-captured)"}


def precision_job(T):
    """The precision configuration in brief: the 4 x 6 J1-J2 lattice, every S^z >= 0
    sector in one batch, R = 64 Rademacher, M = 150, with FP32 and with FP64 vectors
    from the same seeds; job times and the largest FP32 - FP64 difference of E, C and
    chi over the 200 temperatures (relative where |O| >= 1e-6 max|O|, else absolute
    over max|O|)."""
    import numpy as np
    import torch

    from paper_2605_26261_gb300 import ftlm

    wl = WORKLOADS["precision"]
    N, R, M = wl["N"], wl["R"], wl["M"]
    bonds = bonds_of("precision")
    sectors = ftlm.computed_two_sz(N)
    bases = [ftlm.Basis(N, tz, bonds) for tz in sectors]
    per = {}
    for dt in (torch.float32, torch.float64):
        for rep in range(2 if dt == torch.float32 else 1):
            with ftlm.Batch([(b, R, 1, 0) for b in bases], M, ftlm.RADEMACHER, dt, 8) as batch:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                res = batch.run()
                obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], T, R, M)
                e1.record()
                torch.cuda.synchronize()
                upd = sum(int(r["m_eff"].sum().item()) * b.updates for b, r in zip(bases, res))
                per[dt] = (e0.elapsed_time(e1), upd, {k: obs[k].cpu().numpy() for k in ("E", "C", "chi")})
    for b in bases:
        b.close()
    diff = {}
    for k in ("E", "C", "chi"):
        a, ref = per[torch.float32][2][k], per[torch.float64][2][k]
        scale = np.max(np.abs(ref))
        band = np.abs(ref) >= 1e-6 * scale
        rel = np.abs(a[band] - ref[band]) / np.abs(ref[band])
        ab = np.abs(a[~band] - ref[~band]) / scale
        diff[k] = float(max(rel.max() if rel.size else 0.0, ab.max() if ab.size else 0.0))
    f32, f64 = per[torch.float32], per[torch.float64]
    return {"f32_job_ms": f32[0], "f32_Gupdates_per_s": f32[1] / (f32[0] / 1e3) / 1e9,
            "f64_job_ms": f64[0], "f64_Gupdates_per_s": f64[1] / (f64[0] / 1e3) / 1e9,
            "max_rel_diff_f32_vs_f64": diff, "workload": wl["desc"] if "desc" in wl else "precision",
            "note": "same seeded chains in FP32 and FP64 vector storage (FP64 reductions in both)"}


def run_clusters(args):
    """Many small clusters in one batch: every sector of 256 clusters through one
    ftlm_batch (persistent kernel for sectors up to 32768 states, side streams for
    the rest), then the thermodynamic sums of each cluster, captured once as a CUDA
    graph and replayed per step.  Block width and side-stream count come from
    ftlm_batch_autotune on a 24-cluster subset."""
    import torch

    import __graft_entry__
    from paper_2605_26261_gb300 import ftlm, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    R, M = 16, 100
    dt = torch.float32
    clusters = inputs.cluster_set(256, seed=256)[:args.clusters]
    T_host = inputs.log_t_grid(200)
    T = torch.as_tensor(T_host, device=dev)

    def make_bases(cl):
        return [[ftlm.Basis(N, tz, bonds) for tz in ftlm.computed_two_sz(N)] for N, bonds in cl]

    def entries_of(bases_per_cluster, first=0):
        return [(b, R, 1 + first + c, 0) for c, bs in enumerate(bases_per_cluster) for b in bs]

    t_setup = time.perf_counter()
    bases = make_bases(clusters)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    # autotune on 8 clusters of each size
    sub = []
    for n in (18, 20, 22):
        sub += [c for c, (N, _) in enumerate(clusters) if N == n][:8]
    t_tune = time.perf_counter()
    if args.block:
        plan, tried = ftlm.BatchPlan(args.block if args.block > 1 else 16, 4, 0, 0), []
    else:
        plan, tried = ftlm.autotune_plan(entries_of([bases[c] for c in sub]), M, ftlm.RADEMACHER, dt)
    block, streams = plan.block, plan.streams
    tune_s = time.perf_counter() - t_tune
    batch = ftlm.Batch(entries_of(bases), M, ftlm.RADEMACHER, dt, plan=plan)
    results = batch.results
    outs = [{k: torch.empty_like(T) for k in ("E", "C", "chi", "mag")} for _ in clusters]
    k0 = [0]
    for bs in bases:
        k0.append(k0[-1] + len(bs))

    def step():
        batch.run()
        for c, bs in enumerate(bases):
            res = results[k0[c]:k0[c + 1]]
            o = outs[c]
            ftlm.ftlm_thermo([b.two_sz for b in bs], [b.dim for b in bs], R, M, [r["theta"] for r in res],
                             [r["weight"] for r in res], [r["m_eff"] for r in res], True, 2.0, 0.0, T,
                             o["E"], o["C"], o["chi"], o["mag"])

    # one eager run with kernel timing on, for the H.v launch statistics
    ftlm.ftlm_profile_read()
    ftlm.ftlm_profile_enable(True)
    step()
    torch.cuda.synchronize()
    ftlm.ftlm_profile_enable(False)
    hv_n, hv_vec, hv_ms, up_n, up_ms = ftlm.ftlm_profile_read()

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    launches0 = ftlm.ftlm_launch_count()
    with torch.cuda.graph(graph, stream=side):
        step()
    launches_graph = ftlm.ftlm_launch_count() - launches0  # kernel nodes of one replay
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clocks:
        ev[0].record(stream)
        for i in range(args.steps):
            graph.replay()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = sum(step_ms)

    updates = 0
    alg_bytes = 0
    large_rows = small_rows = 0
    for c, bs in enumerate(bases):
        for b, r in zip(bs, results[k0[c]:k0[c + 1]]):
            steps = int(r["m_eff"].sum().item())
            updates += steps * b.updates
            # sector model per chain step, block of `block` interleaved f32 vectors
            alg_bytes += steps / block * sector_model_bytes(b.updates, b.dim, 4, b.mode == ftlm.RANK_CLT,
                                                            B=block)
            if b.dim > 32768:
                large_rows += b.dim
            else:
                small_rows += b.dim
    all_updates, max_ms = aggregate_over_ranks(updates * args.steps, total_ms, dev, world)
    value = all_updates / (max_ms / 1e3) / 1e9

    # end to end through the public API from host data: sector setup, plan, run,
    # thermodynamic sums, results to pinned host memory, release
    e2e = None
    if rank == 0:
        obs_host = torch.empty((len(clusters), 3, 200), dtype=torch.float64).pin_memory()
        T_pin = torch.as_tensor(T_host).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.copy_(T_pin, non_blocking=True)
        bases2 = make_bases(clusters)
        with ftlm.Batch(entries_of(bases2), M, ftlm.RADEMACHER, dt, plan=plan) as b2:
            res2 = b2.run()
            for c, bs in enumerate(bases2):
                res = res2[k0[c]:k0[c + 1]]
                o = outs[c]
                ftlm.ftlm_thermo([b.two_sz for b in bs], [b.dim for b in bs], R, M, [r["theta"] for r in res],
                                 [r["weight"] for r in res], [r["m_eff"] for r in res], True, 2.0, 0.0, T,
                                 o["E"], o["C"], o["chi"], o["mag"])
                for j, k in enumerate(("E", "C", "chi")):
                    obs_host[c, j].copy_(o[k], non_blocking=True)
            torch.cuda.synchronize()
        for bs in bases2:
            for b in bs:
                b.close()
        wall = time.perf_counter() - t0
        h2d = sum(bonds[0].nbytes + bonds[1].nbytes + bonds[2].nbytes for _, bonds in clusters) + T_pin.numel() * 8
        e2e = {"value": updates / wall / 1e9, "unit": "Gupdates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(obs_host.numel() * 8), "ms_per_step": 1e3 * wall,
               "clusters_per_s": len(clusters) / wall}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_src = peak_hbm()
    achieved = alg_bytes / (max_ms / args.steps / 1e3) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        res = OracleSampler(args.workload).sample(args.cpu_seconds)
        cpu = {"value": res["updates_per_s"] / 1e9, "unit": "Gupdates/s", "cores": res["cores"], "kind": "oracle",
               "sample": f"FP64 oracle H.v on {res['rows']} rows (64 evenly spread chunks) of the S^z=0 sector "
                         f"(D={res['D']}) of the first N=22 cluster, {res['seconds']:.1f} s"}
    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["clusters256"]["desc"] if len(clusters) == 256 else
                   f"the first {len(clusters)} clusters of " + WORKLOADS["clusters256"]["desc"],
                   "sectors": sum(len(bs) for bs in bases),
                   "rows_small_sectors": small_rows, "rows_large_sectors": large_rows,
                   "block": block, "side_streams": streams, "tile_rows": plan.tile_rows,
                   "stream_rows": plan.stream_rows,
                   "autotune": {f"B{k[0]}_s{k[1]}_t{k[2]}_u{k[3]}": round(v, 2) for k, v in tried},
                   "autotune_s": tune_s, "setup_s": setup_s,
                   "graph": "one CUDA graph per step: batch run + 256 thermodynamic launches",
                   "l2": "per-sector working sets are L2-sized (<= 90 MB); the whole step streams "
                         f"{2 * 16 * 4 * (small_rows + large_rows) / 1e9:.1f} GB of vectors",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "clusters_per_s": world * len(clusters) * args.steps / (max_ms / 1e3),
        "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                     else "fallback",
                     "kernel": "whole step (batch kernel + H.v launches of the large sectors)",
                     "model": "sector model summed over every H.v of the step / step time; sectors are "
                              "L2-resident, so the HBM model overstates the DRAM bytes",
                     "hv_launches_large": hv_n, "hv_ms_large": hv_ms, "update_ms_large": up_ms},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_graph * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def serve_stream(n_jobs, steps_per_poll, warmup, local=0, clocks=None, live_rows=0):
    """The request loop (serve.Engine: chain-level continuous batching) on the seeded
    Poisson stream of FTLM jobs of the serving configuration: jobs/s (requests /
    makespan) and p50/p99 latency from arrival to results on the host, beside the
    same jobs run one at a time (one job in flight, all queued at once), the same
    jobs through the plain per-sector path one at a time, and a bit-for-bit
    comparison of every job's results in the first two runs."""
    import torch

    from paper_2605_26261_gb300 import ftlm, inputs, serve

    T = inputs.log_t_grid(200)
    R, M = 8, 80

    def engine(max_jobs, live=None):
        return serve.Engine(R=R, M=M, dtype=torch.float32, block=8, T=T, dist=ftlm.GAUSS, max_jobs=max_jobs,
                            steps_per_poll=steps_per_poll, max_live_rows=live)

    # warm-up: a few jobs of every size through a throwaway engine
    warm, _ = serve.poisson_jobs(max(warmup, 6), 200.0, seed=99)
    eng = engine(None)
    eng.run(warm)
    eng.close()
    torch.cuda.synchronize()

    jobs, arrivals = serve.poisson_jobs(n_jobs, 200.0, seed=4)
    launches0 = ftlm.ftlm_launch_count()
    eng = engine(None, live_rows or None)
    if clocks is not None:
        clocks.__enter__()
    try:
        done = eng.run(jobs, arrivals)
        torch.cuda.synchronize()
    finally:
        if clocks is not None:
            clocks.__exit__(None, None, None)
    stats = dict(eng.stats)
    eng.close()
    launches = ftlm.ftlm_launch_count() - launches0
    lat = np.array([j.latency for j in done]) * 1e3
    makespan = max(j.finish for j in done) - min(j.arrival for j in done)
    served = {j.job_id: j for j in done}

    alone_jobs, _ = serve.poisson_jobs(n_jobs, 200.0, seed=4)
    t0 = time.perf_counter()
    eng = engine(1)
    alone = eng.run(alone_jobs)
    torch.cuda.synchronize()
    eng.close()
    alone_s = time.perf_counter() - t0

    # the same jobs through the plain per-sector path of the library, one job at a
    # time: ftlm.run_ftlm (each sector through ftlm_lanczos in turn, then the sums),
    # results read back per job
    plain_jobs, _ = serve.poisson_jobs(n_jobs, 200.0, seed=4)
    Td = torch.as_tensor(T, device=torch.device("cuda", local))
    t0 = time.perf_counter()
    for j in plain_jobs:
        obs = ftlm.run_ftlm(j.N, j.bonds, R, M, Td, seed=j.seed, dist=ftlm.GAUSS, dtype=torch.float32, h=j.h)
        torch.stack([obs[k] for k in ("E", "C", "chi", "mag")]).cpu()
    plain_s = time.perf_counter() - t0
    same = sum(1 for j in alone if np.array_equal(j.result, served[j.job_id].result))
    worst = max((float(np.max(np.abs(j.result - served[j.job_id].result) /
                              np.maximum(np.abs(j.result), 1e-300)))
                 for j in alone if not np.array_equal(j.result, served[j.job_id].result)), default=0.0)
    alone_lat = np.array([j.latency for j in alone]) * 1e3
    return {"jobs": n_jobs, "steps_per_poll": steps_per_poll, "max_live_rows": live_rows or None,
            "jobs_per_s": n_jobs / makespan,
            "max_jobs_in_flight": stats["max_jobs_in_flight"], "max_units": stats["max_units"],
            "host_s": {k: round(v, 3) for k, v in stats["host_s"].items()}, "polls": stats["polls"],
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "makespan_s": makespan, "Gupdates_per_s": sum(j.updates for j in done) / makespan / 1e9,
            "one_at_a_time_jobs_per_s": n_jobs / alone_s,
            "plain_one_at_a_time_jobs_per_s": n_jobs / plain_s,
            "one_at_a_time_p50_ms": float(np.percentile(alone_lat, 50)),
            "one_at_a_time_p99_ms": float(np.percentile(alone_lat, 99)),
            "identical_alone_vs_mix": f"{same}/{n_jobs}", "max_rel_diff_alone_vs_mix": worst,
            "gpu_launches": launches,
            "_done": done, "_jobs": jobs}


def run_serving(args):
    """Serving configuration on its own (see serve_stream)."""
    import torch

    import __graft_entry__
    from paper_2605_26261_gb300 import ftlm, inputs, serve

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:  # replicas only: the request loop runs on rank 0's GPU
        return
    __graft_entry__.build()
    torch.cuda.set_device(local)
    n_jobs = args.jobs
    R = 8
    clocks = ClockSampler(local)
    sv = serve_stream(n_jobs, args.steps_per_poll, args.warmup, local, clocks, args.live_rows)
    done, jobs = sv.pop("_done"), sv.pop("_jobs")
    launches = sv["gpu_launches"]
    makespan = sv["makespan_s"]

    updates = sum(j.updates for j in done)
    value = len(done) / makespan
    peak, peak_src = peak_hbm()
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        res = OracleSampler("serving").sample(args.cpu_seconds)
        cpu = {"value": res["updates_per_s"] / 1e9, "unit": "Gupdates/s", "cores": res["cores"], "kind": "oracle",
               "sample": f"FP64 oracle H.v on {res['rows']} rows of the S^z=0 sector (D={res['D']}) of the first "
                         f"N=26 request, {res['seconds']:.1f} s (oracle Gupdates/s; GPU Gupdates/s of the served "
                         f"run: {updates / makespan / 1e9:.1f})"}
    h2d = sum(j.bonds[0].nbytes + j.bonds[1].nbytes + j.bonds[2].nbytes for j in jobs)
    line = {
        "metric": METRIC, "value": value, "unit": "jobs/s", "n_gpus": 1, "steps": n_jobs, "warmup": max(args.warmup, 6),
        "ms_per_step": 1e3 * makespan / n_jobs, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["serving"]["desc"], "jobs": n_jobs,
                   "steps_per_poll": args.steps_per_poll, "block": 8,
                   "batching": "chain level: sectors join the running multi-sector launches at Lanczos-step "
                               "boundaries (ftlm_flow)",
                   "admission": "first fit of each sector's units in the flow workspace (32 GB)" +
                                (f", at most {args.live_rows} rows of flow sectors in flight" if args.live_rows
                                 else ""),
                   "flow_streams": 4, "small_sectors": "D <= 32768: one persistent batch per job on a side stream",
                   "l2": "largest sectors (D=10400600, 8 f32 vectors) exceed L2",
                   "parallelism": "single GPU"},
        "p50_ms": sv["p50_ms"], "p99_ms": sv["p99_ms"],
        "makespan_s": makespan, "Gupdates_per_s": updates / makespan / 1e9,
        "one_at_a_time": {"jobs_per_s": sv["one_at_a_time_jobs_per_s"], "p50_ms": sv["one_at_a_time_p50_ms"],
                          "p99_ms": sv["one_at_a_time_p99_ms"],
                          "note": "same jobs and engine, one job in flight at a time, all queued at t=0"},
        "plain_one_at_a_time": {"jobs_per_s": sv["plain_one_at_a_time_jobs_per_s"],
                                "note": "same jobs through ftlm.run_ftlm (every sector through ftlm_lanczos in turn, "
                                        "then the sums), one job at a time"},
        "identical_alone_vs_mix": sv["identical_alone_vs_mix"],
        "max_rel_diff_alone_vs_mix": sv["max_rel_diff_alone_vs_mix"],
        "engine": {k: sv[k] for k in ("max_jobs_in_flight", "max_units", "polls", "host_s")},
        "roofline": {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "note": "request-loop line: the H.v kernel roofline is reported by the default workload"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "jobs/s", "h2d_bytes_per_step": int(h2d / n_jobs),
                "d2h_bytes_per_step": int(4 * 200 * 8 + 4 * R * 14),
                "note": "the request loop is end to end: bond lists from host memory, results to pinned host"},
        "gpu_launches": launches, "clocks": clocks.summary(),
    }
    print(json.dumps(line))


def run_precision(args):
    """FP32 vectors (FP64 reductions) against FP64 vectors on one FTLM job, the
    spread of FP32 estimates over independent seeds (Eq. 22), sigma_theo = O /
    sqrt(Z_eff), and Cullum-Willoughby ghost counts (Eq. 25) of FP32 and FP64
    chains from the same start vectors (S^z = 0 sector, first 16 chains)."""
    import torch

    import __graft_entry__
    from paper_2605_26261_gb300 import ftlm, inputs

    if int(os.environ.get("RANK", "0")) != 0:
        return
    __graft_entry__.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS["precision"]
    N, R, M = wl["N"], args.R or wl["R"], args.M or wl["M"]
    bonds = bonds_of("precision")
    T_host = inputs.log_t_grid(200)
    T = torch.as_tensor(T_host, device=dev)
    sectors = ftlm.computed_two_sz(N)
    bases = [ftlm.Basis(N, tz, bonds) for tz in sectors]

    def job(dt, seed):
        with ftlm.Batch([(b, R, seed, 0) for b in bases], M, ftlm.RADEMACHER, dt, 8) as batch:
            res = batch.run()
            obs = ftlm.thermo([(b.two_sz, b.dim, r) for b, r in zip(bases, res)], T, R, M)
            Z = torch.empty_like(T)
            ftlm.ftlm_partition(sectors, [b.dim for b in bases], R, M, [r["theta"] for r in res],
                                [r["weight"] for r in res], [r["m_eff"] for r in res], True, 0.0, T, Z)
            torch.cuda.synchronize()
            upd = sum(int(r["m_eff"].sum().item()) * b.updates for b, r in zip(bases, res))
            return {k: obs[k].cpu().numpy() for k in ("E", "C", "chi")} | {"Z": Z.cpu().numpy()}, upd

    for _ in range(max(1, args.warmup)):
        job(torch.float32, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        l0 = ftlm.ftlm_launch_count()
        ev0.record()
        o32, upd = job(torch.float32, 1)
        ev1.record()
        torch.cuda.synchronize()
        ms32 = ev0.elapsed_time(ev1)
        launches = ftlm.ftlm_launch_count() - l0
        ev0.record()
        o64, upd64 = job(torch.float64, 1)
        ev1.record()
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
    seeds = [o32] + [job(torch.float32, 1 + s)[0] for s in range(1, args.seeds)]
    prec = {}
    for k in ("C", "chi"):
        stack = np.stack([x[k] for x in seeds])
        mean = stack.mean(0)
        sig = np.sqrt(np.sum((stack - mean) ** 2, 0) / len(seeds))  # Eq. 22
        d = np.abs(o32[k] - o64[k])
        sig_theo = np.abs(o64[k]) / np.sqrt(o64["Z"] * len(seeds))  # pooled R_eff = N_s R
        band = np.abs(o64[k]) >= 1e-6 * np.max(np.abs(o64[k]))
        prec[k] = {"max_abs_fp32_minus_fp64": float(d.max()),
                   "max_rel_fp32_minus_fp64": float(np.max(d[band] / np.abs(o64[k][band]))),
                   "max_ratio_diff_over_sigma_emp": float(np.max(d[band] / sig[band])),
                   "median_sigma_emp": float(np.median(sig[band])),
                   "median_sigma_theo_pooled": float(np.median(sig_theo[band]))}
    # ghosts of the same chains in FP32 and FP64 (the S^z = 0 sector)
    gh = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        res = ftlm.lanczos(bases[0], 16, M, seed=1, dist=ftlm.RADEMACHER, dtype=dt, keep_coeffs=True)
        g = ftlm.ghosts(res, c_tau=1.0, u=2.0**-24)
        gh[name] = int(g["count"].sum().item())
    for b in bases:
        b.close()
    cpu = None
    if not args.no_cpu_baseline:
        r = OracleSampler("precision").sample(args.cpu_seconds)
        cpu = {"value": r["updates_per_s"] / 1e9, "unit": "Gupdates/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"FP64 oracle H.v on {r['rows']} rows of the S^z=0 sector (D={r['D']}), "
                         f"{r['seconds']:.1f} s"}
    peak, peak_src = peak_hbm()
    value = upd / (ms32 / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "sectors": len(sectors), "seeds": args.seeds, "block": 8,
                   "fp64_job_ms": ms64, "fp64_Gupdates_per_s": upd64 / (ms64 / 1e3) / 1e9,
                   "parallelism": "single GPU"},
        "precision": prec,
        "ghosts_S0_16_chains": {"f32": gh["f32"], "f64": gh["f64"], "c_tau": 1.0, "u": "2^-24"},
        "roofline": {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "note": "precision line: the H.v kernel roofline is reported by the default workload"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 4 * 200 * 8,
                "note": "sector tables resident; observables read back to the host every job"},
        "gpu_launches": launches, "clocks": clocks.summary(),
    }
    print(json.dumps(line))


def run_hv_only(args):
    """Kernel microbenchmark: W + K plain H.v launches on the workload's sector."""
    import torch

    import __graft_entry__
    from paper_2605_26261_gb300 import ftlm, inputs

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N = WORKLOADS[args.workload]["N"]
    bonds = bonds_of(args.workload)
    mode = {"auto": ftlm.RANK_AUTO, "clt": ftlm.RANK_CLT, "cr": ftlm.RANK_CR}[args.mode]
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    B = args.block or 1
    with ftlm.Basis(N, 0, bonds, mode) as b:
        x = inputs.hashed_vector_torch(b.dim * B, dt, dev)
        y = torch.empty_like(x)

        def once():
            if B == 1:
                ftlm.ftlm_hv(b.handle, x, y)
            else:
                ftlm.ftlm_hv_block(b.handle, B, x, y)

        for _ in range(args.warmup):
            once()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record()
        for i in range(args.steps):
            once()
            ev[i + 1].record()
        torch.cuda.synchronize()
        ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        clt = b.mode == ftlm.RANK_CLT
        med = statistics.median(ms)
        print(json.dumps({"hv_only": True, "workload": args.workload, "mode": "clt" if clt else "cr",
                          "dtype": args.dtype, "block": B, "ms": ms, "ms_median": med,
                          "Gupdates_per_s": B * b.updates / med * 1e-6, "D": b.dim,
                          "updates_per_vector": b.updates}))


def main():
    args = parse_args()
    if args.hv_only:
        run_hv_only(args)
    elif args.workload == "clusters256" and args.impl == "ours":
        run_clusters(args)
    elif args.workload == "serving" and args.impl == "ours":
        run_serving(args)
    elif args.workload == "precision" and args.impl == "ours":
        run_precision(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
