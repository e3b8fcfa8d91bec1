"""Benchmark: MD throughput of the d=6, N=32768 polydisperse harmonic system.

One bench step = 1000 velocity-Verlet timesteps (dt = 0.005, skin 0.3, with
the on-device rebuild trigger and list builds) of a resident system through
the C ABI (md_steps).  Metric: atom-steps/s = N x timesteps / device time.
The system (box side 6, N = 32768, diameters U[0.8, 1.2], T = 1e-3) is
synthetic, drawn with a fixed seed.  Its working set (~40 MB) fits in the
129 MB L2, so L2 is flushed (a 512 MB buffer written) before each timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--gpus N > 1 runs under torchrun as N independent replicas (one per GPU; the
method has no cross-replica exchange): weak scaling, value = all ranks'
atom-steps / the slowest rank's time.  --impl reference times the FP64 CPU
oracle on the host instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2112_12271_gb300 import workloads as W  # noqa: E402

MD_PER_STEP = 1000
DT = 0.005
METRIC = "atom-steps/s at d=6 N=32768 (mixed FP32-pair/FP64 VV)"
UNIT = "atom-steps/s"
WORKLOAD = "d6_N32768_polydisperse_harmonic_L6_NVE_dt0.005_skin0.3"
# c1: the benchmark system; c1l: the same density with N = 2^21 (L = 12), whose
# working set exceeds L2 (the HBM-bound case used for ncu captures)
WORKLOADS = {"c1": 32768, "c1l": 2 ** 21, "batch": 0, "serve": 0, "sweep": 0, "paper": 0}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def l2_bytes():
    """The device's L2 size in bytes; None where this PyTorch does not expose
    it or there is no device."""
    try:
        import torch
        return int(torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size)
    except Exception:
        return None


def footprint_bytes(s):
    """Device bytes of the system as the library allocates them (lists at
    their initial capacity): set against the L2 size it says whether the
    timed kernel streams from HBM or runs out of L2."""
    try:
        from paper_2112_12271_gb300 import hdmd
        return int(hdmd.system_footprint(s.d, s.N, s.L, s.sigma))
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarize(lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the maximum clock and every throttle reason seen
        Active, from nvidia-smi CSV rows in the order of FIELDS (no header,
        no units); None without a readable row."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                clk, top = float(p[1]), float(p[2])
            except ValueError:
                continue
            sm.append(clk)
            mx = top
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- CPU arms
def oracle_md_sample(sysd, nsteps, openmp=False):
    """Time the FP64 oracle on nsteps of the workload (the list build at the
    start of the call included); openmp=True runs its threaded build."""
    import oracle
    oracle.build(openmp=openmp)
    t0 = time.perf_counter()
    out = oracle.md_steps(sysd.x, sysd.v, sysd.sigma, sysd.L, nsteps, DT, openmp=openmp)
    dt = time.perf_counter() - t0
    return dt, out


def host_cpu():
    """CPU model and logical core count of this host (for the baseline record)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    model = "%s (%s)" % (line.split(":", 1)[1].strip(), platform.machine())
                    break
    except OSError:
        pass
    return {"cpu": model, "nproc": os.cpu_count()}


def oracle_threads():
    """Set the OpenMP oracle to every host core; returns the count it uses."""
    import oracle
    oracle.build(openmp=True)
    return oracle.set_threads(os.cpu_count() or 1)


def cpu_baselines(sysd, n_serial=100, n_omp=200):
    """The oracle timed on the host: serially on one core (n_serial steps),
    and its OpenMP build on every core (n_omp steps, per-atom force and
    integration loops and the per-subcell list build run in parallel, as in
    the paper's scheme).  Each call builds the list once at its start, then
    whenever the trigger fires."""
    dt1, o1 = oracle_md_sample(sysd, n_serial)
    serial = {"value": sysd.N * n_serial / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
              **host_cpu(),
              "sample": "%d VV timesteps of the same d=6 N=32768 system (%d list builds), "
                        "serial FP64 C, %.1f s" % (n_serial, o1["builds"], dt1)}
    nt = oracle_threads()
    dtn, on = oracle_md_sample(sysd, n_omp, openmp=True)
    allc = {"value": sysd.N * n_omp / dtn, "unit": UNIT, "cores": nt, "kind": "oracle",
            **host_cpu(),
            "sample": "%d VV timesteps of the same d=6 N=32768 system (%d list builds), "
                      "FP64 C, OpenMP on %d threads, %.1f s" % (n_omp, on["builds"], nt, dtn)}
    return allc, serial


REF_PER_STEP = 200   # oracle timesteps per bench step of the reference arm


def run_reference(args):
    """The oracle on every host core, on the workload of the GPU arm: each
    bench step continues the trajectory for REF_PER_STEP timesteps (lists
    rebuilt when the trigger fires, plus once at the start of each call)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    s = W.c1_poly_d6()
    nt = oracle_threads()
    x, v, img = s.x, s.v, None
    for _ in range(args.warmup):
        oracle_md_sample(s, 5, openmp=True)
    t, builds = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = oracle.md_steps(x, v, s.sigma, s.L, REF_PER_STEP, DT, img=img, openmp=True)
        t += time.perf_counter() - t0
        x, v, img = out["x"], out["v"], out["img"]
        builds += out["builds"]
    value = s.N * REF_PER_STEP * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": s.N, "d": 6, "dt": DT, "skin": 0.3,
                       "timesteps_per_step": REF_PER_STEP, "l2": "cpu",
                       "list_builds": builds},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             **host_cpu(),
                             "sample": "%d VV timesteps per bench step continuing one "
                                       "trajectory, FP64 C oracle with OpenMP on %d threads "
                                       "(%d list builds in all)" % (REF_PER_STEP, nt, builds)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- roofline
def alg_bytes_per_atom_step(d, Z, b_F):
    """Algorithmic bytes of one atom-step of the fused force + velocity-Verlet
    kernel: the list once (4 Z), its length (4), the diameter (4), x read
    and written (16 d), v read and written (16 d), F written and read
    (2 b_F d, b_F = 4 in mixed precision, 8 in FP64); neighbour coordinates
    are taken as cache-resident (atoms are in subcell order)."""
    return 4.0 * Z + 4 + 4 + 16 * d + 16 * d + 2 * b_F * d


def design_bytes_per_atom_step(d, Z):
    """What the mixed kernel of this design moves per atom-step: 8-byte list
    entries (index + subcell-offset code), the length, v and dlt read and
    written in FP64, and three FP32 rows (own, build-time, new)."""
    RF = (d + 1 + 3) & ~3
    return 8.0 * Z + 4 + 16 * d + 16 * d + 3 * 4 * RF


# DRAM bytes per step of the kernel the roofline names, dram__bytes_read.sum
# + dram__bytes_write.sum from one ncu capture of the current kernel (the
# commands are in profiles/); None where no capture of the current kernel
# exists.  c1_resident: 9.98 MB for one resident launch (ncu replays it with
# cold caches, so this is the launch's load of the block state), which ran
# ~36 steps (11 launches over 392 steps in the captured run): ~0.28 MB per
# step.  c1l: the per-step kernel at N = 2^20 moved 417.6 MB per launch
# (398 B per atom), scaled to N = 2^21 by the atom count.
TRAFFIC = {"c1": None, "c1_resident": 9.980e6 / 36.0, "c1l": 417.61e6 * 2.0}


def list_build_kernels(d, N, n_cell, n_cells):
    """Kernels one list build launches: five of binning, the list kernel, and
    the sort of the lists where the half-stencil form applies (n_cell >= 3
    and at least 1500 candidates per atom, 3^d times the atoms per subcell:
    the library's rule)."""
    return 6 + (1 if n_cell >= 3 and 3 ** d * N >= 1500 * n_cells else 0)


def roofline_record(s, info, step_ms, workload, b_F=4, kernel=None):
    """Roofline of the kernel that advances the system one step: algorithmic
    bytes of a step over its device time per step (for the resident kernel,
    one launch's duration over the steps it ran)."""
    d = s.d
    Z = info["total_list_entries"] / s.N
    bpa = alg_bytes_per_atom_step(d, Z, b_F)
    achieved = bpa * s.N / (step_ms * 1e-3) / 1e9 if step_ms else None
    peak, peak_kind = peaks()
    name = kernel or "k_step<%d,%s> (pair forces + kicks + drift + trigger, one launch per step)" % (
        d, "mixed" if b_F == 4 else "fp64")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": TRAFFIC.get(workload + ("_resident" if kernel else "")),
            "kernel": name, "ms_per_step": step_ms,
            "bytes_per_atom_step": bpa, "N": s.N, "mean_list_length": Z,
            "design_bytes_per_atom_step": design_bytes_per_atom_step(d, Z),
            "peak_kind": peak_kind, "l2_bytes": l2_bytes(),
            "footprint_bytes": footprint_bytes(s)}


# --------------------------------------------------------------------- GPU arm
def c1l_record(hdmd, stream, flush, steps=100):
    """The same density with N = 2^21 (L = 12): the system (3.5 GB) does not
    fit in L2, so the step kernel streams from HBM.  Average duration of the
    fused step kernel (CUDA events, 20 launches) and the MD rate of one
    100-step run after an L2 flush."""
    import torch
    s = W.c1_poly_d6(N=2 ** 21)
    with hdmd.System(s.d, s.L, s.sigma, s.x, s.v, precision=hdmd.HDMD_MIXED,
                     stream=stream.cuda_stream) as g:
        g.md_steps(20, DT)
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t = g.md_steps(steps, DT)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        info = g.info()
        prof = g.profile(reps=20, dt=DT)
    return {"workload": "d6_N2097152_polydisperse_harmonic_L12_NVE_dt0.005_skin0.3",
            "value": s.N * steps / (ms / 1000.0), "unit": UNIT, "timesteps": steps,
            "rebuilds": t["rebuilds"], "kernel_ms": prof,
            "roofline": roofline_record(s, info, prof["step_ms"], "c1l")}


def batch_pool_bytes(specs):
    return sum(2500 * sp["N"] * sp["d"] for sp in specs) + (256 << 20)


def batch_pass(hdmd, stream, systems, precision, max_iter, autotune=True):
    """One launch of the batched engine over every job (to the end); returns
    (device ms, results, lanes by d)."""
    import torch
    specs = [dict(N=s.N, d=s.d) for s in systems]
    b = hdmd.Batch(pool_bytes=batch_pool_bytes(specs), max_jobs=len(systems) + 8,
                   precision=precision, stream=stream.cuda_stream)
    try:
        ids = [b.add(hdmd.JOB_FIRE, s.d, s.L, s.sigma, s.x, max_iter=max_iter) for s in systems]
        assert all(i is not None for i in ids)
        if autotune:
            b.autotune(reps=2)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.run(0)
        c.record(stream)
        c.synchronize()
        res = [b.result(i) for i in ids]
        lanes = b.info()["lanes"]
    finally:
        b.close()
    return a.elapsed_time(c), res, lanes


def c3_record(hdmd, stream, jobs=512, max_iter=20000):
    """512 FIRE minimisations (d 3-6, N 256-8192) to max|F_i| < 1e-10 in one
    persistent launch: mixed precision with the FP64 polish against the plain
    FP64 form of the same engine on the same jobs."""
    specs = W.c3_batch_specs(jobs, seed=0)
    systems = [W.c3_job(sp) for sp in specs]
    batch_pass(hdmd, stream, systems[:32], hdmd.HDMD_MIXED, max_iter)   # warm-up
    out = {"workload": "batch_fire_%d_d3-6_N256-8192_bidisperse" % jobs, "jobs": jobs,
           "atoms": sum(s.N for s in systems), "max_iter": max_iter, "unit": "jobs/s"}
    for name, prec in (("mixed", hdmd.HDMD_MIXED), ("fp64", hdmd.HDMD_FP64)):
        ms, res, lanes = batch_pass(hdmd, stream, systems, prec, max_iter)
        conv = sum(1 for r in res if r["converged"])
        out[name] = {"value": conv / (ms / 1000.0), "converged": conv, "seconds": ms / 1000.0,
                     "max_fmax_converged": max((r["fmax"] for r in res if r["converged"]),
                                               default=None),
                     "fire_iterations": sum(r["iterations"] for r in res),
                     "lanes_by_d": lanes[3:7]}
    out["value"] = out["mixed"]["value"]
    out["speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def c4_record(serve_seconds=2.0, slots=16, small_n=1024, budget=256, pool_gb=2, policy="sjf",
              seq_sample=24, time_limit=300.0, batch_work=None, resident=False, compare=True,
              rate=200.0):
    """A fixed slice of the serving stream (the first serve_seconds of the
    Poisson arrivals at 200 requests/s): jobs/s and p50/p99 latency through
    the continuous-batching server, beside the first seq_sample requests
    served one after another as plain FP64 systems and by the server."""
    from paper_2112_12271_gb300 import serve
    from paper_2112_12271_gb300 import hdmd
    reqs = W.c4_requests(duration=serve_seconds, rate=rate, seed=0)
    systems = [W.c4_system(r) for r in reqs]
    warm = W.c4_requests(duration=0.05, rate=200.0, seed=1)
    kw = dict(precision=hdmd.HDMD_MIXED, slots=slots, small_N=small_n,
              batch_pool_bytes=pool_gb << 30, budget=budget, policy=policy,
              batch_work=batch_work, resident=resident)
    srv = serve.Server(**kw)
    srv.run(warm, [W.c4_system(r) for r in warm])
    summ = serve.summarize(srv.run(reqs, systems, time_limit=time_limit))
    srv.close()
    k = min(seq_sample, len(reqs))
    seq = sub = None
    if compare:
        seq = serve.summarize(serve.sequential_fp64(reqs[:k], systems[:k]))
        srv2 = serve.Server(**kw)
        sub = serve.summarize(srv2.run(reqs[:k], systems[:k]))
        srv2.close()
    return {"workload": "serve_poisson200_md_fire_d3-8_N256-131072",
            "routing": {"small_N": small_n, "batch_work": batch_work, "slots": slots,
                        "budget": budget, "system_jobs_resident": resident},
            "slice": "first %.1f s of arrivals at %.0f requests/s (%d requests)"
                     % (serve_seconds, rate, len(reqs)),
            "value": summ["jobs_per_s"], "unit": "jobs/s", "latency_p50_s": summ["p50_s"],
            "latency_p99_s": summ["p99_s"], "summary": summ, "policy": policy,
            "first_%d_requests" % k: {"server": sub, "sequential_fp64": seq}}


def run_gpu(args):
    import torch
    from paper_2112_12271_gb300 import build as B
    from paper_2112_12271_gb300 import hdmd

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
        B.build()

    from paper_2112_12271_gb300 import replicas
    s = W.c1_poly_d6(seed=replicas.replica_seed(rank), N=args.atoms or WORKLOADS[args.workload])
    md_per_step = args.md_per_step
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_md(g, K, W_):
        for _ in range(W_):
            g.md_steps(md_per_step, DT)
        ms, rebuilds = [], 0
        for _ in range(K):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t = g.md_steps(md_per_step, DT)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            rebuilds += t["rebuilds"]
        return ms, rebuilds, t

    g = hdmd.System(s.d, s.L, s.sigma, s.x, s.v, precision=hdmd.HDMD_MIXED,
                    stream=stream.cuda_stream)
    if args.eager:
        g.tune(use_graphs=0)   # profilers cannot see kernels inside conditional graphs
    if args.lanes:
        g.tune(lanes_per_atom=args.lanes)
    info = g.info()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    ms, rebuilds, last = timed_md(g, args.steps, args.warmup)
    torch.cuda.synchronize()
    clocks = clk.stop()
    value, total_ms = replicas.aggregate(s.N * md_per_step * args.steps, sum(ms), device=dev)
    info = g.info()
    prof = g.profile(reps=50, dt=DT) if not args.no_profile else None

    # end to end through the public API: host state in (pinned), md_steps,
    # positions and velocities back out (pinned), per step
    nd = s.N * s.d
    xh = torch.from_numpy(np.ascontiguousarray(s.x)).pin_memory().numpy()
    vh = torch.from_numpy(np.ascontiguousarray(s.v)).pin_memory().numpy()
    xo = torch.empty((s.N, s.d), dtype=torch.float64).pin_memory().numpy()
    vo = torch.empty((s.N, s.d), dtype=torch.float64).pin_memory().numpy()
    e2e_ms = []
    for k in range(0 if args.no_e2e else args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_state(xh, vh)
        g.md_steps(md_per_step, DT)
        g.state_into(xo, vo)
        if k >= args.warmup:
            e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_value = (ws * s.N * md_per_step * args.steps / (sum(e2e_ms) / 1000.0)) if e2e_ms else None
    g.close()

    # FP64 plain form of the same workload
    fp64 = None
    if not args.no_fp64:
        g64 = hdmd.System(s.d, s.L, s.sigma, s.x, s.v, precision=hdmd.HDMD_FP64,
                          stream=stream.cuda_stream)
        k64 = max(1, min(args.steps, 10))
        ms64, _, _ = timed_md(g64, k64, 1)
        info64 = g64.info()
        prof64 = g64.profile(reps=20, dt=DT) if not args.no_profile else None
        g64.close()
        fp64 = {"value": s.N * md_per_step * k64 / (sum(ms64) / 1000.0), "unit": UNIT,
                "ms_per_step": sum(ms64) / k64, "steps": k64, "kernel_ms": prof64,
                "roofline": roofline_record(s, info64, prof64["step_ms"] if prof64 else None,
                                            "none", b_F=8)}

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    d = s.d
    Z = info["total_list_entries"] / s.N
    per_build = list_build_kernels(d, s.N, info["n_cell"], info["n_cells"])
    if info.get("resident"):
        # per bench step: first kick-drift, step budget, final force + kick;
        # one resident launch per list, and the list builds
        n_launch = args.steps * 3 + (rebuilds + args.steps) + per_build * rebuilds
    else:
        n_launch = args.steps * (md_per_step + 1) + per_build * rebuilds
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-pair/f64-accumulate",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "c1" else
                   "d6_N%d_polydisperse_harmonic_L%.0f_NVE_dt0.005_skin0.3" % (s.N, s.L),
                   "N": s.N, "d": d, "L": s.L,
                   "timesteps_per_step": md_per_step, "dt": DT, "skin": 0.3,
                   "l2": "flushed (512 MB write) before each timed step",
                   "n_cell": info["n_cell"], "mean_list_length": Z,
                   "lanes_per_atom": info["lanes_per_atom"], "graphs": info["graphs"],
                   "resident_blocks": info.get("resident", 0),
                   "rebuilds_per_step": rebuilds / args.steps},
        "fp64": fp64,
        "kernel_ms": prof,
        "roofline": (roofline_record(s, info, prof["resident_step_ms"], args.workload,
                                     kernel="k_md_resident<%d> (resident MD: pair forces + kicks "
                                            "+ drift + trigger, many steps per launch)" % d)
                     if prof and prof.get("resident_step_ms") else
                     roofline_record(s, info, prof["step_ms"] if prof else None, args.workload)),
        "roofline_per_step_kernel": roofline_record(s, info, prof["step_ms"] if prof else None,
                                                    args.workload) if prof else None,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 2 * nd * 8,
                "d2h_bytes_per_step": 2 * nd * 8 + 7 * 8},
        "gpu_launches": n_launch,
        "clocks": clocks,
    }
    if ws == 1 and args.workload == "c1" and not args.no_sub:
        # the other figures the benchmark metric names, each measured here
        line["c1l"] = c1l_record(hdmd, stream, flush)
        del flush
        line["c3_batched_fire"] = c3_record(hdmd, stream, max_iter=args.max_iter)
        line["c4_serving"] = c4_record(policy=args.policy, slots=args.slots,
                                       small_n=args.small_n, budget=args.budget,
                                       pool_gb=args.pool_gb)
        # the same request mix offered below the server's capacity (~15
        # jobs/s): latency of service rather than of the queue
        line["c4_serving_below_capacity"] = c4_record(
            serve_seconds=10.0, rate=10.0, policy=args.policy, slots=args.slots,
            small_n=args.small_n, budget=args.budget, pool_gb=args.pool_gb, compare=False)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"], line["cpu_baseline_serial"] = cpu_baselines(s)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


# --------------------------------------------------------------------- batched FIRE
def run_batch(args):
    """512 independent FIRE minimisations (to max|F_i| < 1e-10) in the batched
    engine, mixed precision with FP64 polish, against the plain FP64 form of
    the same engine on the same 512 jobs (one pass each)."""
    import torch
    from paper_2112_12271_gb300 import build as B
    from paper_2112_12271_gb300 import hdmd
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    rec = c3_record(hdmd, stream, jobs=args.jobs, max_iter=args.max_iter)
    line = {"metric": "batched FIRE jobs/s converged to |F|max<1e-10 (%d jobs, d 3-6, N 256-8192)"
                      % args.jobs,
            "value": rec["value"], "unit": "jobs/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1000.0 * rec["mixed"]["seconds"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-accumulate+f64-polish", "data": "synthetic",
            "config": {"workload": rec["workload"], "jobs": rec["jobs"], "atoms": rec["atoms"],
                       "max_iter": rec["max_iter"]},
            "mixed": rec["mixed"], "fp64": rec["fp64"], "speedup_vs_fp64": rec["speedup_vs_fp64"]}
    print(json.dumps(line), flush=True)
    return 0

# -------------------------------------------------------- the paper's own model
PAPER_TAU_T = 0.5   # Berendsen damping time (the paper names tau_temp, no value)
def run_paper(args):
    """The paper's benchmark protocol (Sec. III) at d = 3..6: its Morse law
    (a = 30) with volume-scaled prefactors and masses, diameters of Eq. (3)
    with R = d, phi*_d of Table III, T = 0.25, dt = 0.0016, skin 0.25.  Each
    system is pushed off as the paper does (FIRE until E_pair/N < eps, each
    move capped at 0.01), given velocities at T, then run for
    args.paper_tau time units of NVT MD (Berendsen, tau_T = 0.5)
    (625 steps each) with one SWAP pass (p = 0.1) per time unit.  Reports
    atom-steps/s per d, the device time per list entry and step, and the
    split of the device time over leapfrog, list builds, minimisation (one
    FIRE per 10 time units, counted pro rata) and SWAP, as in Table IV."""
    import torch
    from paper_2112_12271_gb300 import build as B
    from paper_2112_12271_gb300 import hdmd
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    steps_per_tau = int(round(1.0 / W.PAPER_DT))
    rows, total_atom_steps, total_s = [], 0, 0.0
    for d in range(3, 7):
        s = W.paper_model(d, args.paper_n, seed=d)
        law = dict(skin=0.25, stream=stream.cuda_stream, law="morse", a=W.MORSE_A, eps_scale=True)
        # the paper's pushoff: FIRE until the average pair energy is below
        # eps, each move capped (Sec. II.A, Table II); in FP64, whose range
        # holds the Morse forces of nearly coincident random atoms
        with hdmd.System(d, s.L, s.sigma, s.x, None, s.mass, precision=hdmd.HDMD_FP64, **law) as g:
            push = g.fire(e_thres=1.0, dx_max=0.01, dt0=W.PAPER_DT, dt_max=10 * W.PAPER_DT,
                          dt_min=0.02 * W.PAPER_DT, max_iter=100000, n_neg_max=10 ** 9)
            x0 = g.state(v=False, img=False)["x"]
        with hdmd.System(d, s.L, s.sigma, x0, s.v, s.mass, precision=hdmd.HDMD_MIXED, **law) as g:
            g.thermostat(W.PAPER_T, PAPER_TAU_T)             # the paper's runs are NVT
            g.md_steps(steps_per_tau, W.PAPER_DT)          # warm-up: graphs, first builds
            g.set_reference()                                # r_i(0) of the observables
            a = torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            acc = reb = 0
            swap_ms = 0.0
            for tau in range(args.paper_tau):
                t = g.md_steps(steps_per_tau, W.PAPER_DT)
                reb += t["rebuilds"]
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                acc += g.swap(W.PAPER_T, p=0.1, nsweeps=1, seed=1000 * d + tau)[0]
                e1.record(stream)
                e1.synchronize()
                swap_ms += e0.elapsed_time(e1)
            c.record(stream)
            c.synchronize()
            sec = a.elapsed_time(c) / 1000.0
            info = g.info()
            prof = g.profile(reps=20, dt=W.PAPER_DT)
            t0 = time.perf_counter()
            obs = g.observables(nbins=100, r_max=2.0)
            obs_ms = 1000.0 * (time.perf_counter() - t0)
            st = g.state(v=False, img=False, sigma=True)   # SWAP moved the diameters
        # one energy minimisation of the current configuration per 10 time
        # units, as in the paper's runs (FIRE to E_pair/N < 1e-25), on a copy
        with hdmd.System(d, s.L, st["sigma"], st["x"], None, st["sigma"] ** d,
                         precision=hdmd.HDMD_MIXED, **law) as gm:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mres = gm.fire(e_thres=1e-25, dt0=W.PAPER_DT, dt_max=10 * W.PAPER_DT,
                           dt_min=0.02 * W.PAPER_DT, max_iter=200000)
            e1.record(stream)
            e1.synchronize()
            min_ms = e0.elapsed_time(e1) * args.paper_tau / 10.0
        vl_ms = reb * prof["rebuild_ms"]
        md_ms = 1000.0 * sec - swap_ms
        whole = 1000.0 * sec + min_ms
        shares = {"leapfrog": (md_ms - vl_ms) / whole, "vl_build": vl_ms / whole,
                  "minimisation": min_ms / whole, "swap": swap_ms / whole}
        n_steps = steps_per_tau * args.paper_tau
        z = info["total_list_entries"] / s.N
        rows.append({"d": d, "N": s.N, "phi_star": W.PHI_STAR[d], "L": s.L, "n_cell": info["n_cell"],
                     "pushoff_iterations": push["iterations"],
                     "seconds": sec, "atom_steps_per_s": s.N * n_steps / sec,
                     "ns_per_list_entry_step": 1e9 * sec / (n_steps * s.N * z),
                     "mean_list_length": z, "rebuilds": reb, "swap_accepted": acc,
                     "T_end": t["T"], "E_pair_per_atom": t["E_pair"] / s.N,
                     "msd": obs["msd"], "alpha2": obs["alpha2"], "f_ov": obs["f_ov"],
                     "Z": obs["Z"], "observables_ms": obs_ms,
                     "minimisation": {"iterations": mres["iterations"], "ms": min_ms * 10.0 / args.paper_tau,
                                      "E_pair_per_atom": mres["E_pair"] / s.N},
                     "runtime_share": shares})
        total_atom_steps += s.N * n_steps
        total_s += sec
        print(json.dumps({"paper_row": rows[-1]}), file=sys.stderr, flush=True)
    line = {"metric": "paper model: atom-steps/s, Morse a=30, phi*_d, T=0.25, d 3-6 (MD + SWAP per tau)",
            "value": total_atom_steps / total_s, "unit": "atom-steps/s", "n_gpus": 1,
            "steps": args.paper_tau, "warmup": 1, "ms_per_step": 1000.0 * total_s / (4 * args.paper_tau),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-accumulate", "data": "synthetic",
            "config": {"workload": "paper_model_morse_d3-6_N%d" % args.paper_n, "N": args.paper_n,
                       "tau": args.paper_tau, "steps_per_tau": steps_per_tau, "dt": W.PAPER_DT,
                       "skin": 0.25, "T": W.PAPER_T, "swap_p": 0.1},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0

# ------------------------------------------------------------- dimension sweep
def run_sweep(args):
    """Dimension sweep d = 4..8 at N = 65536: FIRE to max|F_i| < 1e-10 (mixed
    precision with the FP64 polish, and the plain FP64 form beside it), then
    100 SWAP sweeps (p = 0.1, T = 1e-3) of the minimised packing."""
    import torch
    from paper_2112_12271_gb300 import build as B
    from paper_2112_12271_gb300 import hdmd
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        c = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        c.record(stream)
        c.synchronize()
        return a.elapsed_time(c) / 1000.0, out

    rows, total = [], 0.0
    for d in range(4, 9):
        s = W.c2_sweep(d, seed=0, N=args.sweep_n)
        row = {"d": d, "N": s.N, "L": s.L}
        with hdmd.System(s.d, s.L, s.sigma, s.x, precision=hdmd.HDMD_MIXED,
                         stream=stream.cuda_stream) as g:
            row["n_cell"] = g.info()["n_cell"]
            t_fire, r = timed(lambda: g.fire(max_iter=args.sweep_max_iter))
            t_swap, (acc, _) = timed(lambda: g.swap(1e-3, p=0.1, nsweeps=args.swap_sweeps, seed=d))
            row.update(fire_s=t_fire, fire_iterations=r["iterations"],
                       polish_iterations=r["polish_iterations"], converged=bool(r["converged"]),
                       fmax=r["fmax"], E_pair=r["E_pair"], swap_s=t_swap,
                       swap_ms_per_sweep=1000.0 * t_swap / args.swap_sweeps,
                       swap_accepted=acc, swap_candidates=args.swap_sweeps * int(round(0.1 * s.N)))
        total += t_fire + t_swap
        if not args.no_fp64:
            with hdmd.System(s.d, s.L, s.sigma, s.x, precision=hdmd.HDMD_FP64,
                             stream=stream.cuda_stream) as g:
                t64, r64 = timed(lambda: g.fire(max_iter=args.sweep_max_iter))
            row.update(fp64_fire_s=t64, fp64_fire_iterations=r64["iterations"],
                       fp64_converged=bool(r64["converged"]))
        rows.append(row)
        print(json.dumps({"sweep_row": row}), file=sys.stderr, flush=True)
    line = {"metric": "dimension sweep: FIRE to |F|max<1e-10 + %d SWAP sweeps, d 4-8" % args.swap_sweeps,
            "value": total, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1000.0 * total, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-pair/f64-accumulate+f64-polish", "data": "synthetic",
            "config": {"workload": "sweep_d4-8_N%d_poly_fire_swap" % args.sweep_n,
                       "N": args.sweep_n, "swap_sweeps": args.swap_sweeps, "p": 0.1, "T": 1e-3,
                       "max_iter": args.sweep_max_iter},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0

# --------------------------------------------------------------------- serving
def run_serve(args):
    """Poisson stream (200 requests/s) of MD and FIRE requests through the
    continuous-batching server; p50/p99 latency and jobs/s, beside the same
    first requests served one after another as plain FP64 systems."""
    from paper_2112_12271_gb300 import serve   # sets the stream work-queue count first
    from paper_2112_12271_gb300 import build as B
    from paper_2112_12271_gb300 import hdmd
    import torch
    torch.cuda.set_device(0)
    B.build()
    reqs = W.c4_requests(duration=args.serve_seconds, rate=200.0, seed=0)
    systems = [W.c4_system(r) for r in reqs]
    warm = W.c4_requests(duration=0.05, rate=200.0, seed=1)
    warm_sys = [W.c4_system(r) for r in warm]
    srv = serve.Server(precision=hdmd.HDMD_MIXED, slots=args.slots, small_N=args.small_n,
                       batch_pool_bytes=args.pool_gb << 30, budget=args.budget,
                       policy=args.policy)
    srv.run(warm, warm_sys)            # warm-up: builds, graphs, allocator
    recs = srv.run(reqs, systems, time_limit=args.serve_time_limit)
    srv.close()
    summ = serve.summarize(recs)
    k = min(args.seq_sample, len(reqs))
    seq = serve.summarize(serve.sequential_fp64(reqs[:k], systems[:k]))
    srv2 = serve.Server(precision=hdmd.HDMD_MIXED, slots=args.slots, small_N=args.small_n,
                        batch_pool_bytes=args.pool_gb << 30, budget=args.budget,
                        policy=args.policy)
    sub = serve.summarize(srv2.run(reqs[:k], systems[:k]))
    srv2.close()
    md_work = sum(r["N"] * r["nsteps"] for r in reqs if r["kind"] == 0)
    line = {"metric": "serving: jobs/s and p50/p99 latency, Poisson 200 req/s of MD + FIRE",
            "value": summ["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1000.0 * summ["makespan_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-pair/f64-accumulate", "data": "synthetic",
            "config": {"workload": "serve_poisson200_md_fire_d3-8_N256-131072",
                       "requests": len(reqs), "arrival_seconds": args.serve_seconds,
                       "md_atom_steps": md_work, "budget_per_launch": args.budget,
                       "slots": args.slots, "small_N": args.small_n, "policy": args.policy},
            "latency_p50_s": summ["p50_s"], "latency_p99_s": summ["p99_s"], "summary": summ,
            "first_%d_requests" % k: {"server": sub, "sequential_fp64": seq}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS))
    ap.add_argument("--md-per-step", type=int, default=MD_PER_STEP)
    ap.add_argument("--atoms", type=int, default=0,
                    help="c1/c1l workloads: atoms at the same density (0: the workload's N)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per atom (0: library default)")
    ap.add_argument("--jobs", type=int, default=512, help="batched workload: number of jobs")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="serving workload: seconds of Poisson arrivals")
    ap.add_argument("--serve-time-limit", type=float, default=300.0,
                    help="serving workload: stop serving after this many seconds")
    ap.add_argument("--budget", type=int, default=256,
                    help="serving workload: steps / FIRE iterations per job per launch")
    ap.add_argument("--pool-gb", type=int, default=2,
                    help="serving workload: batched-engine device pool (GiB)")
    ap.add_argument("--policy", default="sjf", choices=["fifo", "sjf"],
                    help="serving workload: admission order of waiting systems")
    ap.add_argument("--slots", type=int, default=16,
                    help="serving workload: concurrent system jobs")
    ap.add_argument("--small-n", type=int, default=1024,
                    help="serving workload: largest N served by the batched engine")
    ap.add_argument("--seq-sample", type=int, default=24,
                    help="serving workload: requests of the sequential FP64 comparison")
    ap.add_argument("--max-iter", type=int, default=20000,
                    help="batched and sweep workloads: FIRE iteration limit per job")
    ap.add_argument("--sweep-n", type=int, default=65536, help="sweep workload: atoms per system")
    ap.add_argument("--paper-n", type=int, default=100000, help="paper workload: atoms per system")
    ap.add_argument("--paper-tau", type=int, default=10, help="paper workload: time units of MD")
    ap.add_argument("--swap-sweeps", type=int, default=100, help="sweep workload: SWAP sweeps")
    ap.add_argument("--sweep-max-iter", type=int, default=200000,
                    help="sweep workload: FIRE iteration limit")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: skip the C1-L, batched and serving sub-records")
    ap.add_argument("--eager", action="store_true",
                    help="launch kernels one by one instead of CUDA graphs (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "paper":
        return run_paper(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
