"""GPU test of the continuous-batching server: requests arriving over time
are admitted while others run, both job paths (batched engine and dedicated
systems) are exercised, and every result equals the result of the same
request run alone."""
import numpy as np
import pytest

from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd, serve
    build.build()
    return hdmd, serve


def small_stream():
    reqs = W.c4_requests(duration=0.06, rate=200.0, seed=8)
    for r in reqs:                       # keep the test short
        r["N"] = int(min(r["N"], 2500 if r["d"] < 8 else 3200))
        r["nsteps"] = 300
    return reqs


def test_served_results_equal_alone(env):
    hdmd, serve = env
    reqs = small_stream()
    assert len(reqs) >= 6
    systems = [W.c4_system(r) for r in reqs]
    srv = serve.Server(precision=hdmd.HDMD_MIXED, slots=4, small_N=1800,
                       batch_pool_bytes=1 << 30, max_batch_jobs=256, budget=64,
                       keep_positions=True)
    recs = srv.run(reqs, systems)
    srv.close()
    s = serve.summarize(recs)
    assert s["completed"] == len(reqs)
    assert s["batch_jobs"] >= 2 and s["system_jobs"] >= 1
    # continuous batching: jobs were admitted while others were running, on
    # both paths
    for path in ("batch", "system"):
        rs = [r for r in recs if r.path == path]
        assert any(a.admitted < b.admitted < a.done for a in rs for b in rs if a is not b), path
    for rec, sysd in zip(recs, systems):
        req = rec.req
        if rec.path == "batch":
            with hdmd.Batch(pool_bytes=256 << 20, max_jobs=4, precision=hdmd.HDMD_MIXED) as b:
                jid = b.add(req["kind"], sysd.d, sysd.L, sysd.sigma, sysd.x,
                            sysd.v if req["kind"] == 0 else None, dt=0.005,
                            nsteps=req["nsteps"], max_iter=20000)
                b.run(0)
                alone = b.result(jid, positions=True)
        else:
            with hdmd.System(sysd.d, sysd.L, sysd.sigma, sysd.x, sysd.v,
                             precision=hdmd.HDMD_MIXED) as g:
                if req["kind"] == 0:
                    t = g.md_steps(req["nsteps"], 0.005)
                    alone = dict(E_pair=t["E_pair"])
                else:
                    alone = dict(E_pair=g.fire(max_iter=20000)["E_pair"])
                alone["x"] = g.state(v=False, img=False)["x"]
        assert rec.result["E_pair"] == alone["E_pair"], (rec.path, req)
        assert np.array_equal(rec.result["x"], alone["x"]), (rec.path, req)


def test_footprint_matches_allocation(env):
    hdmd, _ = env
    for d, N, phi in ((3, 700, 0.5), (6, 5000, 0.14), (8, 3000, 0.047), (4, 20000, 0.37)):
        s = W.make_system(d, N, phi=phi, dist="poly", T=1e-3, seed=d)
        for prec in (hdmd.HDMD_FP64, hdmd.HDMD_MIXED):
            fp = hdmd.system_footprint(d, N, s.L, s.sigma, precision=prec)
            with hdmd.System(d, s.L, s.sigma, precision=prec) as g:
                assert g.info()["device_bytes"] == fp, (d, N, prec)
