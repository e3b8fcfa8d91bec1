"""Continuous-batching job server for MD and FIRE requests.

Requests (an MD run of n steps or a FIRE minimisation, each with its own N,
d, box and diameters) arrive over time.  Every admitted job keeps its state
resident on the GPU until it finishes, and jobs that arrive while others run
are admitted as soon as a slot and device memory free up, so their work
overlaps on the device:

* jobs are routed by estimated work (``work``: atom-steps, FIRE counted at
  a typical iteration count): a job of at most ``batch_work`` atom-steps and
  at most ``small_N`` atoms joins the batched engine, every other job runs
  as its own system;
* a system job runs as its own system (``hdmd.System``, the
  grid-wide kernels and CUDA graphs) on its own CUDA stream, in one of
  ``slots`` worker threads.  It is admitted (first come first served, or
  with policy "sjf" smallest estimated work first) when a slot is free and
  its device footprint (``hdmd.system_footprint``, with
  head-room for list growth) fits in what the running systems leave of the
  device-memory budget (by default 85 % of the free HBM at start, less the
  batch pool);
* a batched job joins the batched engine (``hdmd.Batch``, one
  thread block per job): a batch thread admits it when the engine's device
  pool has room for its arrays and launches the persistent kernels, each
  launch advancing every resident job by at most ``budget`` steps or FIRE
  iterations; finished jobs are retired and their memory goes to the next.

A job's result does not depend on what else is running: a system's kernels
and a batched job's block use fixed-order reductions, so each result is the
same alone and in the mix.
"""
from __future__ import annotations

import collections
import os
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import hdmd

# Every system and the batched engine launch on streams of their own; with
# the CUDA default of 8 hardware work queues, streams share queues and one
# job's long graph launch would hold up unrelated jobs behind it.  Takes
# effect only when the process has not created its CUDA context yet.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")


class Record:
    """Timeline and result of one request (times in seconds from the start)."""
    __slots__ = ("idx", "req", "arrival", "admitted", "done", "status", "result", "path",
                 "reserved")

    def __init__(self, idx, req):
        self.idx, self.req = idx, req
        self.arrival = self.admitted = self.done = None
        self.status = None
        self.result = None
        self.path = None
        self.reserved = 0

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def work(req, fire_iterations=500):
    """Estimated work of a request in atom-steps (FIRE: a typical iteration
    count), the key of the shortest-job-first policy."""
    steps = req.get("nsteps", 0) if req["kind"] == hdmd.JOB_MD else fire_iterations
    return req["N"] * steps


class Server:
    def __init__(self, precision=hdmd.HDMD_MIXED, slots=16, small_N=1024,
                 batch_pool_bytes=2 << 30, max_batch_jobs=2048, mem_bytes=None,
                 budget=256, dt=0.005, max_iter=20000, keep_positions=False,
                 headroom=1.5, log=None, policy="fifo", batch_work=None, resident=False):
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        # no work limit given: route by size alone
        self.batch_work = float("inf") if batch_work is None else float(batch_work)
        # system jobs share the GPU: the resident MD kernel holds whole SMs
        # for a list's lifetime, which the other jobs would wait behind
        self.resident = resident
        import torch
        self.torch = torch
        self.precision = precision
        self.slots = slots
        self.small_N = small_N
        self.budget = budget
        self.dt = dt
        self.max_iter = max_iter
        self.keep_positions = keep_positions
        self.headroom = headroom
        self.log = log
        self.batch_stream = torch.cuda.Stream()
        self.batch = hdmd.Batch(pool_bytes=batch_pool_bytes, max_jobs=max_batch_jobs,
                                precision=precision, stream=self.batch_stream.cuda_stream)
        if mem_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            mem_bytes = int(0.85 * free)
        self.mem_bytes = int(mem_bytes)
        self._local = threading.local()
        self._lock = threading.Lock()

    def to_batch(self, req):
        """True when the request goes to the batched engine."""
        return req["N"] <= self.small_N and work(req) <= self.batch_work

    # ------------------------------------------------------------ system jobs
    def _system_job(self, rec, system):
        torch = self.torch
        if not hasattr(self._local, "stream"):
            self._local.stream = torch.cuda.Stream()
        s = self._local.stream
        req = rec.req
        with hdmd.System(system.d, system.L, system.sigma, system.x, system.v,
                         precision=self.precision, stream=s.cuda_stream) as g:
            g.resident(self.resident)
            if req["kind"] == hdmd.JOB_MD:
                t = g.md_steps(req["nsteps"], self.dt)
                res = dict(status=hdmd.JOB_DONE, E_pair=t["E_pair"], K=t["K"],
                           iterations=req["nsteps"], converged=0)
            else:
                r = g.fire(max_iter=self.max_iter)
                res = dict(status=hdmd.JOB_DONE if r["converged"] else hdmd.JOB_NOT_CONVERGED,
                           E_pair=r["E_pair"], K=0.0, iterations=r["iterations"],
                           converged=r["converged"], fmax=r["fmax"])
            if self.keep_positions:
                res["x"] = g.state(v=False, img=False)["x"]
        rec.result = res
        rec.status = res["status"]
        rec.done = time.perf_counter() - self._t0
        return rec

    # ------------------------------------------------------------ batch thread
    def _batch_loop(self, queue, systems, stop):
        running = {}
        while True:
            while queue:
                rec = queue[0]
                s, req = systems[rec.idx], rec.req
                jid = self.batch.add(req["kind"], s.d, s.L, s.sigma, s.x,
                                     s.v if req["kind"] == hdmd.JOB_MD else None,
                                     dt=self.dt, nsteps=req.get("nsteps", 0),
                                     max_iter=self.max_iter)
                if jid is None:
                    break          # no room in the pool: wait for retirements
                rec.path = "batch"
                rec.admitted = time.perf_counter() - self._t0
                running[jid] = rec
                queue.popleft()
            if running:
                self.batch.run(self.budget)
                for jid in list(running):
                    r = self.batch.result(jid, positions=self.keep_positions)
                    if r["status"] != hdmd.JOB_RUNNING:
                        rec = running.pop(jid)
                        rec.done = time.perf_counter() - self._t0
                        rec.status = r["status"]
                        rec.result = r
                        self.batch.remove(jid)
            elif stop.is_set() and not queue:
                return
            else:
                time.sleep(0.0005)

    # ------------------------------------------------------------ main loop
    def run(self, requests, systems, time_limit=None):
        """Serve requests (dicts with arrival time t [s], kind, d, N, nsteps)
        whose inputs are systems[i]; returns one Record per request."""
        recs = [Record(i, r) for i, r in enumerate(requests)]
        pending = collections.deque(sorted(range(len(recs)), key=lambda i: requests[i]["t"]))
        small_q, big_q = collections.deque(), collections.deque()
        stop = threading.Event()
        futures = []
        reserved = 0
        in_flight = []
        pool = ThreadPoolExecutor(max_workers=self.slots)
        self._t0 = t0 = time.perf_counter()
        bt = threading.Thread(target=self._batch_loop, args=(small_q, systems, stop), daemon=True)
        bt.start()
        last_log = 0.0
        try:
            while True:
                now = time.perf_counter() - t0
                while pending and requests[pending[0]]["t"] <= now:
                    rec = recs[pending.popleft()]
                    rec.arrival = rec.req["t"]
                    if self.to_batch(rec.req):
                        small_q.append(rec)
                    elif self.policy == "sjf":   # keep the waiting systems by estimated work
                        big_q.append(rec)
                        big_q = collections.deque(sorted(big_q, key=lambda r: (work(r.req), r.idx)))
                    else:
                        big_q.append(rec)
                # retire finished systems, returning their memory reservation
                still = []
                for rec, f in in_flight:
                    if f.done():
                        f.result()
                        reserved -= rec.reserved
                    else:
                        still.append((rec, f))
                in_flight = still
                # admit systems first come first served: a free slot and memory
                while big_q and len(in_flight) < self.slots:
                    rec = big_q[0]
                    s = systems[rec.idx]
                    need = int(self.headroom * hdmd.system_footprint(
                        s.d, s.N, s.L, s.sigma, precision=self.precision))
                    if in_flight and reserved + need > self.mem_bytes:
                        break
                    big_q.popleft()
                    rec.reserved = need
                    reserved += need
                    rec.path = "system"
                    rec.admitted = time.perf_counter() - t0
                    f = pool.submit(self._system_job, rec, s)
                    in_flight.append((rec, f))
                    futures.append(f)
                if self.log and now - last_log >= 1.0:
                    last_log = now
                    self.log("t=%.1f s: arrived %d, queued %d+%d, systems %d (%.2f GB), done %d"
                             % (now, len(recs) - len(pending), len(small_q), len(big_q),
                                len(in_flight), reserved / 1e9,
                                sum(1 for r in recs if r.done is not None)))
                if not pending and not big_q and not in_flight:
                    break
                if time_limit is not None and now > time_limit:
                    break
                time.sleep(0.0005)
            stop.set()
            bt.join()
            for f in futures:
                f.result()
        finally:
            stop.set()
            pool.shutdown(wait=True)
        return recs

    def close(self):
        self.batch.close()


def summarize(recs):
    """Completed jobs, jobs/s over the span from the first arrival to the last
    completion, and latency (completion - arrival) percentiles."""
    done = [r for r in recs if r.done is not None]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    first = min(r.arrival for r in recs if r.arrival is not None) if done else 0.0
    last = max(r.done for r in done) if done else 1.0
    return dict(jobs=len(recs), completed=len(done),
                converged_fire=sum(1 for r in done if r.req["kind"] == 1 and r.status == hdmd.JOB_DONE),
                jobs_per_s=len(done) / max(last - first, 1e-9),
                p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                makespan_s=last - first,
                batch_jobs=sum(1 for r in done if r.path == "batch"),
                system_jobs=sum(1 for r in done if r.path == "system"))


def sequential_fp64(requests, systems, dt=0.005, max_iter=20000):
    """The same requests served one after another, each as its own FP64 system
    (no batching, no overlap): latency = completion - arrival."""
    import torch
    stream = torch.cuda.current_stream()
    recs = [Record(i, r) for i, r in enumerate(requests)]
    t0 = time.perf_counter()
    for i in sorted(range(len(recs)), key=lambda k: requests[k]["t"]):
        req, s, rec = requests[i], systems[i], recs[i]
        now = time.perf_counter() - t0
        if req["t"] > now:
            time.sleep(req["t"] - now)
        rec.arrival = req["t"]
        with hdmd.System(s.d, s.L, s.sigma, s.x, s.v, precision=hdmd.HDMD_FP64,
                         stream=stream.cuda_stream) as g:
            if req["kind"] == hdmd.JOB_MD:
                g.md_steps(req["nsteps"], dt)
                rec.status = hdmd.JOB_DONE
            else:
                r = g.fire(max_iter=max_iter)
                rec.status = hdmd.JOB_DONE if r["converged"] else hdmd.JOB_NOT_CONVERGED
        rec.done = time.perf_counter() - t0
        rec.path = "sequential"
    return recs
