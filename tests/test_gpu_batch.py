"""GPU tests of the batched engine (batch_* ABI): each job gives the answer the
oracle gives, the same bits alone and in a mix, the same bits whether it runs
to the end in one launch or in budgeted pieces, and admission respects the
device pool."""
import numpy as np
import pytest

import oracle
from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    build.build()
    oracle.build()
    return hdmd


def jobs_mix(seed=0):
    out = []
    for k, (d, N, phi) in enumerate([(3, 300, 0.4), (4, 500, 0.3), (3, 700, 0.85), (5, 400, 0.2),
                                     (6, 600, 0.12), (4, 250, 0.55)]):
        out.append((d, W.make_system(d, N, phi=phi, dist="bi", T=0.0, seed=seed + k)))
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_fire_jobs_converge_checked_by_oracle(H, prec):
    p = H.HDMD_MIXED if prec == "mixed" else H.HDMD_FP64
    mix = jobs_mix()
    with H.Batch(pool_bytes=256 << 20, max_jobs=64, precision=p) as b:
        ids = [b.add(H.JOB_FIRE, d, s.L, s.sigma, s.x) for d, s in mix]
        assert b.run(0) == 0
        for (d, s), jid in zip(mix, ids):
            r = b.result(jid, positions=True)
            assert r["status"] == H.JOB_DONE and r["converged"], r
            Fo, Eo, _ = oracle.forces(r["x"], s.sigma, s.L)
            assert np.linalg.norm(Fo, axis=1).max() < 1e-10
            assert r["E_pair"] == pytest.approx(Eo, rel=1e-6, abs=1e-20)


def test_batch_job_same_alone_and_in_mix_and_in_pieces(H):
    mix = jobs_mix(seed=10)
    d0, s0 = mix[2]
    res = []
    for mode in ("alone", "mix", "pieces"):
        with H.Batch(pool_bytes=256 << 20, max_jobs=64, precision=H.HDMD_MIXED) as b:
            for d in (3, 4, 5, 6):
                b.set_lanes(d, 4)
            if mode == "alone":
                jid = b.add(H.JOB_FIRE, d0, s0.L, s0.sigma, s0.x)
            else:
                ids = [b.add(H.JOB_FIRE, d, s.L, s.sigma, s.x) for d, s in mix]
                jid = ids[2]
            if mode == "pieces":
                while b.run(37):
                    pass
            else:
                b.run(0)
            res.append(b.result(jid, positions=True))
    for r in res[1:]:
        assert r["iterations"] == res[0]["iterations"]
        assert r["E_pair"] == res[0]["E_pair"]
        assert np.array_equal(r["x"], res[0]["x"])


def test_batch_md_matches_oracle_and_system(H):
    s = W.c0_bidisperse_d3()
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005)
    with H.Batch(pool_bytes=64 << 20, max_jobs=4, precision=H.HDMD_FP64) as b:
        jid = b.add(H.JOB_MD, 3, s.L, s.sigma, s.x, s.v, dt=0.005, nsteps=100)
        b.run(0)
        r = b.result(jid, positions=True)
    assert r["status"] == H.JOB_DONE and r["iterations"] == 100
    dx = r["x"] - ref["x"]
    dx -= s.L * np.round(dx / s.L)
    assert np.abs(dx).max() < 1e-9
    assert r["E_pair"] == pytest.approx(ref["E"], rel=1e-10)
    assert r["K"] == pytest.approx(ref["K"], rel=1e-10)


@pytest.mark.parametrize("d,N,kw", [(3, 1000, dict(phi=0.6)), (6, 3000, dict(L=5.0))])
def test_batch_mixed_md_matches_oracle(H, d, N, kw):
    """The mixed-precision batched MD that the serving loop runs (FP32 pair
    forces, FP64 kick and drift): 100 steps against the FP64 oracle within
    the mixed trajectory tolerance of the single-system tests (1e-5 of the
    positions, E and K relative), beside a different job in the same batch."""
    s = W.make_system(d, N, dist="poly", T=1e-3, seed=40 + d, **kw)
    other = W.make_system(4, 500, phi=0.3, dist="bi", T=1e-3, seed=9)
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005)
    assert ref["builds"] >= 1
    with H.Batch(pool_bytes=128 << 20, max_jobs=4, precision=H.HDMD_MIXED) as b:
        jid = b.add(H.JOB_MD, d, s.L, s.sigma, s.x, s.v, dt=0.005, nsteps=100)
        b.add(H.JOB_MD, 4, other.L, other.sigma, other.x, other.v, dt=0.005, nsteps=60)
        b.run(0)
        r = b.result(jid, positions=True)
    assert r["status"] == H.JOB_DONE and r["iterations"] == 100
    dx = r["x"] - ref["x"]
    dx -= s.L * np.round(dx / s.L)
    assert np.abs(dx).max() < 1e-5
    assert r["E_pair"] == pytest.approx(ref["E"], rel=1e-5)
    assert r["K"] == pytest.approx(ref["K"], rel=1e-5)


def test_batch_admission_by_pool_memory(H):
    s = W.make_system(4, 2000, phi=0.3, dist="bi", T=0.0, seed=3)
    with H.Batch(pool_bytes=8 << 20, max_jobs=32, precision=H.HDMD_MIXED) as b:
        ids = []
        while True:
            jid = b.add(H.JOB_FIRE, 4, s.L, s.sigma, s.x)
            if jid is None:
                break
            ids.append(jid)
            assert len(ids) < 32
        assert len(ids) >= 1
        free0 = b.info()["free_bytes"]
        b.remove(ids[0])
        assert b.info()["free_bytes"] > free0
        assert b.add(H.JOB_FIRE, 4, s.L, s.sigma, s.x) is not None


def test_batch_autotune_picks_lanes(H):
    mix = jobs_mix(seed=20)
    with H.Batch(pool_bytes=256 << 20, max_jobs=64, precision=H.HDMD_MIXED) as b:
        for d, s in mix:
            b.add(H.JOB_FIRE, d, s.L, s.sigma, s.x)
        b.autotune(reps=2)
        lanes = b.info()["lanes"]
        for d in (3, 4, 5, 6):
            assert lanes[d] in (1, 2, 4, 8, 16)
        assert b.run(0) == 0
