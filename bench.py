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
PAPER_GUPS = 800 * 4969109520 / 124.0 / 1e9  # paper's GPU-CLT run of this workload (124 s, RTX 4000 Ada)
FALLBACK_HBM_GBS = 6800.0
WORKLOADS = {
    "icosidodecahedron": dict(N=30, desc="icosidodecahedron N=30 S^z=0 (D=155117520, 60 bonds, J=1)"),
    "ring34": dict(N=34, desc="ring N=34 S^z=0 (D=2333606220, 34 bonds, J=1)"),
}
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "hv_kernel_icosidodecahedron.md")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=list(WORKLOADS), default="icosidodecahedron")
    p.add_argument("--mode", choices=["auto", "clt", "cr"], default="auto")
    p.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    p.add_argument("--R", type=int, default=8)
    p.add_argument("--M", type=int, default=100)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--hv-only", action="store_true",
                   help="time plain ftlm_hv launches on the workload (kernel microbenchmark)")
    p.add_argument("--block", type=int, default=1,
                   help="with --hv-only: vectors per launch (ftlm_hv_block, 1/4/8/16)")
    return p.parse_args()


def bonds_of(name):
    from paper_2605_26261_gb300 import inputs

    return inputs.icosidodecahedron() if name == "icosidodecahedron" else inputs.ring(34)


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


def kernel_fingerprint():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2605_26261_gb300", "csrc")
    for f in ("hv.cu", "reduce.cuh", "ftlm_internal.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(mode_name, dtype):
    """DRAM bytes per H.v launch from the committed ncu summary, if it was taken on
    the current kernel source for this mode and dtype; else None."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    fp = re.search(r"kernel_fingerprint:\s*(\w+)", text)
    if not fp or fp.group(1) != kernel_fingerprint():
        return None
    m = re.search(rf"dram_bytes_per_launch\[{mode_name},{dtype}\]:\s*([0-9.eE+]+)", text)
    return float(m.group(1)) if m else None


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
        self.ok = N <= 30  # beyond that the oracle cannot enumerate the sector in host memory
        if not self.ok:
            return
        self.bonds = bonds_of(workload)
        self.b = o.basis(N, N // 2)
        self.D = len(self.b)
        self.upd_per_row = (self.D + 2 * len(self.bonds[2]) * math.comb(N - 2, N // 2 - 1)) / self.D
        self.x = np.random.default_rng(seed).standard_normal(self.D)

    def _run(self, rows_per_chunk, offset):
        starts = (np.linspace(0, self.D - rows_per_chunk - 64, 64) + offset).astype(np.int64)
        out = np.empty(rows_per_chunk)
        t = time.perf_counter()
        for s in starts:
            self.o.hv_range(self.bonds, self.b, self.x, int(s), int(s) + rows_per_chunk, out=out)
        return time.perf_counter() - t, 64 * rows_per_chunk

    def sample(self, seconds, offset=0):
        t0, n0 = self._run(256, offset)
        rows_chunk = max(256, int(seconds / (t0 / n0) / 64))
        t1, n1 = self._run(rows_chunk, offset)
        return {"updates_per_s": n1 * self.upd_per_row / t1, "rows": n1, "seconds": t1,
                "cores": self.o.num_threads(), "D": self.D}


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
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gupdates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["desc"], "parallelism": "host threads"},
        "cpu_baseline": {"value": v, "unit": "Gupdates/s", "cores": res["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
    N = wl["N"]
    bonds = bonds_of(args.workload)
    mode = {"auto": ftlm.RANK_AUTO, "clt": ftlm.RANK_CLT, "cr": ftlm.RANK_CR}[args.mode]
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    R, M = args.R, args.M
    T_host = inputs.log_t_grid(200)
    T = torch.as_tensor(T_host, device=dev)

    probe = ftlm.Basis(N, 0, bonds, mode)
    D, updates_hv, mode_used = probe.dim, probe.updates, probe.mode
    work_bytes = ftlm.ftlm_lanczos_workspace_bytes(probe.handle, R, M, dt)
    probe.close()
    work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
    theta = torch.empty((R, M), dtype=torch.float64, device=dev)
    weight = torch.empty_like(theta)
    m_eff = torch.empty(R, dtype=torch.int32, device=dev)
    obs = {k: torch.empty_like(T) for k in ("E", "C", "chi", "mag")}

    def step():
        with ftlm.Basis(N, 0, bonds, mode) as b:
            ftlm.ftlm_lanczos(b.handle, R, M, 1, ftlm.RADEMACHER, dt, work, theta, weight, m_eff)
            ftlm.ftlm_thermo([0], [D], R, M, [theta], [weight], [m_eff], True, 2.0, 0.0, T,
                             obs["E"], obs["C"], obs["chi"], obs["mag"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ftlm.ftlm_profile_read()  # drop anything recorded so far
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ftlm.ftlm_profile_enable(True)
    with ClockSampler(local) as clocks:
        ev[0].record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    ftlm.ftlm_profile_enable(False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    hv_n, hv_vec, hv_ms, up_n, up_ms = ftlm.ftlm_profile_read()
    chains_steps = int(m_eff.sum().item())
    updates_step = chains_steps * updates_hv
    # kernels per step: H.v and update launches (counted), per chain block a start
    # and an m_eff copy, the Ritz step, the thermodynamic sums, the coarse index
    # build of the sector setup, and for CLT the basis and CLT builds
    m_max = min(M, D)
    blocks = hv_n // max(1, args.steps * m_max)
    launches_step = ((hv_n + up_n) // args.steps + 2 * blocks + 2 + 1
                     + (2 if mode_used == ftlm.RANK_CLT else 0))

    all_updates, max_ms = aggregate_over_ranks(updates_step * args.steps, total_ms, dev, world)
    value = all_updates / (max_ms / 1e3) / 1e9

    # end-to-end through the public API with host buffers (one job per step):
    # bond list and T grid from (pinned) host memory, results read back to pinned host memory
    e2e = None
    if rank == 0 or world == 1:
        T_pin = torch.as_tensor(T_host).pin_memory()
        outs_host = [torch.empty((R, M), dtype=torch.float64).pin_memory() for _ in range(2)]
        me_host = torch.empty(R, dtype=torch.int32).pin_memory()
        obs_host = [torch.empty(200, dtype=torch.float64).pin_memory() for _ in range(3)]
        bi, bj, J = (np.ascontiguousarray(a) for a in bonds)
        n_e2e = max(1, min(2, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            T.copy_(T_pin, non_blocking=True)
            with ftlm.Basis(N, 0, (bi, bj, J), mode) as b:
                ftlm.ftlm_lanczos(b.handle, R, M, 1, ftlm.RADEMACHER, dt, work, theta, weight, m_eff)
                ftlm.ftlm_thermo([0], [D], R, M, [theta], [weight], [m_eff], True, 2.0, 0.0, T,
                                 obs["E"], obs["C"], obs["chi"], obs["mag"])
            outs_host[0].copy_(theta, non_blocking=True)
            outs_host[1].copy_(weight, non_blocking=True)
            me_host.copy_(m_eff, non_blocking=True)
            for h_, k in zip(obs_host, ("E", "C", "chi")):
                h_.copy_(obs[k], non_blocking=True)
            torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / n_e2e
        h2d = bi.nbytes + bj.nbytes + J.nbytes + T_pin.numel() * 8
        d2h = 2 * R * M * 8 + R * 4 + 3 * 200 * 8
        e2e = {"value": int(me_host.sum()) * updates_hv / wall / 1e9, "unit": "Gupdates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * wall}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_src = peak_hbm()
    hv_avg_s = hv_ms / max(hv_n, 1) / 1e3
    block = round(hv_vec / max(hv_n, 1))  # vectors per H.v launch (one block width per run)
    clt = mode_used == ftlm.RANK_CLT
    alg_bytes = sector_model_bytes(updates_hv, D, 4 if dt == torch.float32 else 8, clt, B=block)
    achieved = alg_bytes / hv_avg_s / 1e9 if hv_n else None
    mode_name = "clt" if clt else "cr"
    traffic = profiled_traffic(mode_name, args.dtype)
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak if achieved else None, "traffic": traffic,
        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
        "kernel": f"hv_kernel<{'float' if dt == torch.float32 else 'double'}, {mode_name.upper()}, lanczos, B={block}>",
        "model": "sector model: 32 B per gathered x element + row streams",
        "algorithmic_bytes_per_launch": alg_bytes,
        "hv_launches": hv_n, "vectors_per_launch": block, "hv_ms_avg": hv_avg_s * 1e3,
        "hv_Gupdates_per_s": block * updates_hv / hv_avg_s / 1e9 if hv_n else None,
        "dram_frac": (traffic / hv_avg_s / 1e9 / peak) if (traffic and hv_n) else None,
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
                             f"spread chunks of the D={res['D']} sector, {res['seconds']:.1f} s"}
    srt = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_GUPS, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": wl["desc"] + f", R={R} Rademacher, M={M}, 200-point T grid",
                   "rank_mode": mode_name.upper(), "vectors": f"{args.dtype} storage, FP64 reductions",
                   "l2": "inputs larger than L2 (two vectors of D elements, 620 MB each in f32)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "vs_baseline_ref": "paper GPU-CLT, 124 s for this job on RTX 4000 Ada (Table 3)"},
        "jobs_per_s": world * args.steps / (max_ms / 1e3),
        "p50_ms": srt[len(srt) // 2], "p99_ms": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_step * args.steps, "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


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
    B = args.block
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
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
