"""The seeded input generators on the CPU: each produces the sizes and
distributions its docstring states (the input recipe of the benchmarks),
independently of the code under test."""
import math

import numpy as np
import pytest

from paper_2112_12271_gb300 import workloads as W


def test_sphere_volume_closed_forms():
    s = np.array([0.8, 1.0, 1.4])
    assert np.allclose(W.sphere_volume(1, s), s)                       # a segment
    assert np.allclose(W.sphere_volume(2, s), math.pi * s ** 2 / 4)    # a disc
    assert np.allclose(W.sphere_volume(3, s), math.pi * s ** 3 / 6)    # a ball
    assert np.allclose(W.sphere_volume(4, s), math.pi ** 2 * s ** 4 / 32)


@pytest.mark.parametrize("d", [2, 3, 6, 9])
def test_box_side_gives_the_packing_fraction(d):
    rng = np.random.default_rng(d)
    sigma = W.polydisperse(rng, 500)
    phi = 0.3
    L = W.box_side(d, sigma, phi)
    assert W.sphere_volume(d, sigma).sum() / L ** d == pytest.approx(phi, rel=1e-12)


def test_positions_lie_in_the_box_and_velocities_are_thermal():
    rng = np.random.default_rng(0)
    x = W.uniform_positions(rng, 20000, 4, 3.0)
    assert x.min() >= -1.5 and x.max() < 1.5
    v = W.thermal_velocities(rng, 20000, 4, 0.25)
    assert np.abs(v.mean(axis=0)).max() < 1e-12            # no drift
    # K = d (N - 1) T / 2: the centre of mass carries no kinetic energy
    assert 0.5 * (v ** 2).sum() == pytest.approx(0.5 * 4 * 19999 * 0.25, rel=1e-12)


def test_batch_specs():
    specs = W.c3_batch_specs()
    assert len(specs) == 512
    N = np.array([s["N"] for s in specs])
    d = np.array([s["d"] for s in specs])
    assert N.min() >= 256 and N.max() <= 8192
    # log-uniform: log N spread evenly over [log 256, log 8192]
    u = (np.log(N) - math.log(256)) / (math.log(8192) - math.log(256))
    assert abs(u.mean() - 0.5) < 0.05 and abs(u.var() - 1 / 12) < 0.015
    assert set(d) == {3, 4, 5, 6}
    ratio = np.array([s["phi"] / W.jamming_estimate(s["d"]) for s in specs])
    assert ratio.min() >= 0.6 and ratio.max() <= 1.2
    assert len({s["seed"] for s in specs}) == 512
    job = W.c3_job(specs[0])
    assert sorted(set(np.round(job.sigma, 12))) == [1.0, 1.4]           # bidisperse
    assert W.sphere_volume(job.d, job.sigma).sum() / job.L ** job.d == pytest.approx(specs[0]["phi"])


def test_request_stream():
    reqs = W.c4_requests(duration=10.0, rate=200.0, seed=3)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 10.0
    assert abs(len(reqs) - 2000) < 4 * math.sqrt(2000)                 # Poisson count
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 200, rel=0.1)
    assert gaps.std() == pytest.approx(1 / 200, rel=0.15)              # exponential: sd = mean
    kinds = np.array([r["kind"] for r in reqs])
    assert 0.4 < kinds.mean() < 0.6
    steps = np.array([r["nsteps"] for r in reqs])
    assert steps.min() >= 1000 and steps.max() <= 10000
    assert {r["d"] for r in reqs} == set(range(3, 9))
    N = np.array([r["N"] for r in reqs])
    assert N.min() >= 256 and N.max() <= 131072
    low_d = np.array([r["N"] for r in reqs if r["d"] <= 5])            # where the floor is 256
    assert np.median(low_d) == pytest.approx(4096, rel=0.15)
    for r in reqs:
        assert r["N"] >= W.min_valid_N(r["d"], r["phi"])
        assert r["phi"] == W.jamming_estimate(r["d"])


def test_request_boxes_hold_one_image():
    """Every served system's box exceeds twice its largest diameter, so only
    the nearest image of a pair can interact."""
    for r in W.c4_requests(duration=0.25, rate=200.0, seed=5):
        s = W.c4_system(r)
        assert s.N == r["N"] and s.d == r["d"]
        assert s.L > 2 * s.sigma.max(), r
