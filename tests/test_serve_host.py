"""Host logic of the job server, on the CPU.

``serve.Server`` is driven with stand-ins for its GPU objects (the per-job
systems, the batched engine and the CUDA streams), so its scheduler runs
unchanged without a device: the split between the batched engine and
dedicated systems, admission by device-memory footprint, the slot limit,
first-come-first-served and shortest-job-first order, the batched engine's
back-pressure when its pool is full, and the summary statistics."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2112_12271_gb300 import hdmd, serve

torch = pytest.importorskip("torch")

FOOT = 1000          # stand-in footprint: bytes per atom
JOB_S = 0.03         # how long a stand-in system job runs


class Tracker:
    """What the stand-ins saw: start order and peak concurrency."""

    def __init__(self):
        self.lock = threading.Lock()
        self.running = 0
        self.peak = 0
        self.started = []        # N of each system job, in start order
        self.start_time = {}     # N -> perf_counter at start
        self.running_at_start = []
        self.batch_added = []    # N of each batched job, in admission order
        self.batch_peak = 0
        self.resident = []       # resident-kernel switch of each system job


class FakeStream:
    cuda_stream = 0


def fakes(tracker, batch_capacity=64):
    class FakeSystem:
        def __init__(self, d, L, sigma, x, v, precision=None, stream=None, **kw):
            self.N = len(sigma)
            self.x = x

        def __enter__(self):
            with tracker.lock:
                tracker.running += 1
                tracker.peak = max(tracker.peak, tracker.running)
                tracker.started.append(self.N)
                tracker.start_time[self.N] = time.perf_counter()
                tracker.running_at_start.append(tracker.running)
            return self

        def __exit__(self, *exc):
            with tracker.lock:
                tracker.running -= 1
            return False

        def resident(self, on=True):
            tracker.resident.append(bool(on))

        def md_steps(self, n, dt):
            time.sleep(JOB_S)
            return dict(E_pair=float(self.N), K=1.0)

        def fire(self, max_iter=20000):
            time.sleep(JOB_S)
            return dict(converged=1, E_pair=0.0, iterations=7, fmax=1e-11)

        def state(self, v=True, img=True):
            return dict(x=np.array(self.x))

    class FakeBatch:
        def __init__(self, pool_bytes=0, max_jobs=0, precision=None, stream=None):
            self.jobs = {}
            self.next = 0

        def add(self, kind, d, L, sigma, x, v, dt=0.005, nsteps=0, max_iter=20000):
            if len(self.jobs) >= batch_capacity:
                return None
            jid = self.next
            self.next += 1
            self.jobs[jid] = dict(kind=kind, left=nsteps if kind == hdmd.JOB_MD else 1,
                                  N=len(sigma))
            tracker.batch_added.append(len(sigma))
            tracker.batch_peak = max(tracker.batch_peak, len(self.jobs))
            return jid

        def run(self, budget):
            time.sleep(0.002)
            for j in self.jobs.values():
                j["left"] -= budget if j["kind"] == hdmd.JOB_MD else 1

        def result(self, jid, positions=False):
            j = self.jobs[jid]
            return dict(status=hdmd.JOB_RUNNING if j["left"] > 0 else hdmd.JOB_DONE,
                        E_pair=float(j["N"]))

        def remove(self, jid):
            del self.jobs[jid]

        def close(self):
            pass

    return FakeSystem, FakeBatch


@pytest.fixture
def patched(monkeypatch):
    tr = Tracker()

    def install(batch_capacity=64):
        FakeSystem, FakeBatch = fakes(tr, batch_capacity)
        monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
        monkeypatch.setattr(serve.hdmd, "System", FakeSystem)
        monkeypatch.setattr(serve.hdmd, "Batch", FakeBatch)
        monkeypatch.setattr(serve.hdmd, "system_footprint",
                            lambda d, N, L, sigma, precision=None, **kw: FOOT * N)
        return tr

    return install


def jobs(Ns, kinds=None, nsteps=None, t=None):
    """Requests and their inputs; every N differs so the stand-ins can tell
    the jobs apart."""
    reqs, systems = [], []
    for k, N in enumerate(Ns):
        kind = hdmd.JOB_MD if kinds is None else kinds[k]
        reqs.append(dict(t=0.0 if t is None else t[k], kind=kind, d=3, N=N,
                         nsteps=100 if nsteps is None else nsteps[k]))
        systems.append(SimpleNamespace(d=3, N=N, L=10.0, sigma=np.ones(N),
                                       x=np.zeros((N, 3)), v=np.zeros((N, 3))))
    return reqs, systems


def server(**kw):
    base = dict(slots=4, small_N=100, mem_bytes=1 << 40, budget=50, headroom=1.0)
    base.update(kw)
    return serve.Server(**base)


def test_small_jobs_batched_big_jobs_on_systems(patched):
    tr = patched()
    Ns = [50, 2000, 60, 3000, 100, 4000, 101]          # 100 = small_N joins the batch
    reqs, systems = jobs(Ns, kinds=[0, 1, 1, 0, 0, 1, 0])
    srv = server()
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert all(r.done is not None for r in recs)
    for r in recs:
        assert r.path == ("batch" if r.req["N"] <= 100 else "system")
        assert r.status == hdmd.JOB_DONE
        assert r.admitted >= r.arrival - 1e-9 and r.done >= r.admitted
    assert sorted(tr.started) == [101, 2000, 3000, 4000]
    assert sorted(tr.batch_added) == [50, 60, 100]
    # MD results carry the stand-in energy of their own job
    for r in recs:
        if r.path == "system" and r.req["kind"] == hdmd.JOB_MD:
            assert r.result["E_pair"] == float(r.req["N"])


def test_device_memory_bounds_concurrent_systems(patched):
    tr = patched()
    Ns = [1000 + k for k in range(6)]
    reqs, systems = jobs(Ns)
    # room for two of these footprints at once, not three
    srv = server(slots=8, mem_bytes=int(2.5 * FOOT * 1000))
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert all(r.done is not None for r in recs)
    assert tr.peak == 2
    # finished jobs return their reservation: later jobs run in pairs again
    assert tr.running_at_start.count(2) >= 2, tr.running_at_start


def test_job_larger_than_memory_runs_alone(patched):
    tr = patched()
    reqs, systems = jobs([5000, 1001, 1002])
    srv = server(slots=8, mem_bytes=FOOT * 3000)   # the first job alone exceeds it
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert all(r.done is not None for r in recs)
    assert tr.started[0] == 5000
    big = recs[0]
    # nothing was admitted beside it while it ran
    assert all(r.admitted >= big.done - 1e-3 for r in recs[1:])


def test_slot_limit(patched):
    tr = patched()
    reqs, systems = jobs([1000 + k for k in range(9)])
    srv = server(slots=3)
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert all(r.done is not None for r in recs)
    assert tr.peak == 3
    # no job is admitted beyond the slots to wait for a worker
    for r in recs:
        assert tr.start_time[r.req["N"]] - (srv._t0 + r.admitted) < 0.5 * JOB_S


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_admission_order(patched, policy):
    tr = patched()
    Ns = [4000, 1500, 3000, 1200, 2500]
    nsteps = [100, 400, 50, 100, 100]          # work N * nsteps: 4e5 6e5 1.5e5 1.2e5 2.5e5
    reqs, systems = jobs(Ns, nsteps=nsteps)
    srv = server(slots=1, policy=policy)
    srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    if policy == "fifo":
        assert tr.started == Ns
    else:
        assert tr.started == [N for _, N in sorted(zip((n * s for n, s in zip(Ns, nsteps)), Ns))]


def test_fifo_keeps_arrival_order_over_time(patched):
    tr = patched()
    Ns = [1500, 1200, 1800, 1100]
    reqs, systems = jobs(Ns, t=[0.03, 0.0, 0.02, 0.01])
    srv = server(slots=1)
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert tr.started == [1200, 1100, 1800, 1500]
    for r in recs:
        assert r.arrival == r.req["t"]


def test_full_batch_pool_holds_jobs_back(patched):
    tr = patched(batch_capacity=2)
    Ns = [10 + k for k in range(7)]
    reqs, systems = jobs(Ns, nsteps=[200] * 7)
    srv = server(budget=50)
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert all(r.done is not None and r.path == "batch" for r in recs)
    assert tr.batch_peak == 2
    assert tr.batch_added == Ns                   # first come first served


def test_unknown_policy_is_rejected(patched):
    patched()
    with pytest.raises(ValueError):
        server(policy="lifo")


def test_work_estimate():
    assert serve.work(dict(kind=hdmd.JOB_MD, N=1000, nsteps=300)) == 300000
    assert serve.work(dict(kind=hdmd.JOB_FIRE, N=1000)) == 500000
    assert serve.work(dict(kind=hdmd.JOB_FIRE, N=1000), fire_iterations=20) == 20000


def test_summarize():
    recs = []
    for k, (arr, done, kind, status, path) in enumerate([
            (0.0, 1.0, 0, hdmd.JOB_DONE, "batch"),
            (0.5, 2.5, 1, hdmd.JOB_DONE, "system"),
            (1.0, 2.0, 1, hdmd.JOB_NOT_CONVERGED, "system"),
            (1.5, None, 0, None, None)]):
        r = serve.Record(k, dict(kind=kind))
        r.arrival, r.done, r.status, r.path = arr, done, status, path
        recs.append(r)
    s = serve.summarize(recs)
    assert s["jobs"] == 4 and s["completed"] == 3
    assert s["converged_fire"] == 1
    assert s["makespan_s"] == pytest.approx(2.5)
    assert s["jobs_per_s"] == pytest.approx(3 / 2.5)
    lat = [1.0, 2.0, 1.0]
    assert s["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["p99_s"] == pytest.approx(np.percentile(lat, 99))
    assert s["batch_jobs"] == 1 and s["system_jobs"] == 2


def test_routing_by_estimated_work(patched):
    """A job joins the batched engine when it has at most small_N atoms and
    at most batch_work estimated atom-steps (FIRE at its typical iteration
    count, 500); every other job runs as a system, with the resident MD
    kernel off (system jobs share the GPU)."""
    tr = patched()
    Ns = [1000, 1001, 3000, 6000]
    reqs, systems = jobs(Ns, kinds=[0, 0, 1, 1], nsteps=[1000, 5000, 0, 0])
    # work: 1e6 (batch), 5.005e6 (system), 1.5e6 (batch), N > small_N (system)
    srv = server(small_N=5000, batch_work=2e6)
    assert [srv.to_batch(r) for r in reqs] == [True, False, True, False]
    recs = srv.run(reqs, systems, time_limit=20.0)
    srv.close()
    assert [r.path for r in recs] == ["batch", "system", "batch", "system"]
    assert sorted(tr.batch_added) == [1000, 3000]
    assert tr.resident == [False, False]
