"""GPU parity for the paper's own model (Sec. II.A): the truncated and shifted
Morse law of Eq. (1) with a = 30, volume-scaled prefactors eps_i = sigma_i^d
mixed as sqrt(eps_i eps_j), masses m_i = sigma_i^d, diameters from Eq. (3)
with R = d, packing fractions phi*_d of Table III, skin 0.25, dt = 0.0016.

The oracle runs under the same law (oracle.law).  Tolerances as in
test_gpu_parity: forces max|dF| <= tol max|F| (1e-12 FP64, 1e-5 mixed),
energy and virial relative tol; 100-step trajectories within 1e-9 (FP64)
and 1e-5 (mixed); FIRE minima checked by the oracle's forces (< 1e-10);
SWAP decisions, diameters and rescaled velocities equal to the serial oracle.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A = W.MORSE_A
SKIN = 0.25
LAW = dict(law="morse", a=A, eps_scale=True)


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    build.build()
    oracle.build()
    return hdmd


def _start(d, N, seed, jitter):
    """The paper relaxes its random initial positions (whose Morse energies
    reach 1e27 at phi*_d) by a FIRE pushoff before MD.  Here the oracle's
    FIRE with the bounded harmonic law removes every overlap (phi*_d is
    below jamming), and a Gaussian jitter of the given width then brings
    back overlaps of moderate depth, so the Morse forces are exercised."""
    s = W.paper_model(d, N, seed=seed)
    r = oracle.fire(s.x, s.sigma, s.L, max_iter=20000)
    x = r["x"] + np.random.default_rng(seed).normal(0.0, jitter, r["x"].shape)
    x = (x + 0.5 * s.L) % s.L - 0.5 * s.L
    return s, x


@pytest.mark.parametrize("d,N", [(3, 700), (4, 900), (6, 1500)])
def test_forces_energy_virial(H, d, N):
    s, xj = _start(d, N, d, 0.02)
    for x in (xj, s.x):          # moderate overlaps; the raw random state
        with oracle.law("morse", A, eps_scale=True):
            Fo, Eo, Wo = oracle.forces(x, s.sigma, s.L)
        assert Eo > 0
        for prec, tol in ((H.HDMD_FP64, 1e-12), (H.HDMD_MIXED, 1e-5)):
            with H.System(d, s.L, s.sigma, x, s.v, s.mass, skin=SKIN, precision=prec, **LAW) as g:
                F, E, Wv = g.forces()
            assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max(), prec
            assert np.isfinite(F).all()
            assert E == pytest.approx(Eo, rel=tol)
            assert Wv == pytest.approx(Wo, rel=tol)


def test_harmonic_law_with_scaled_prefactors(H):
    s = W.paper_model(5, 800, phi=0.5 * W.PHI_STAR[5], seed=2)
    with oracle.law("harmonic", eps_scale=True):
        Fo, Eo, Wo = oracle.forces(s.x, s.sigma, s.L)
    with H.System(5, s.L, s.sigma, s.x, precision=H.HDMD_FP64, law="harmonic", eps_scale=True) as g:
        F, E, Wv = g.forces()
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert E == pytest.approx(Eo, rel=1e-12)


def test_100_steps_with_masses_match_oracle(H):
    s, x0 = _start(3, 800, 5, 0.005)
    with oracle.law("morse", A, eps_scale=True):
        ref = oracle.md_steps(x0, s.v, s.sigma, s.L, 100, W.PAPER_DT, skin=SKIN, mass=s.mass)
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(3, s.L, s.sigma, x0, s.v, s.mass, skin=SKIN, precision=prec, **LAW) as g:
            t = g.md_steps(100, W.PAPER_DT)
            st = g.state()
        dx = st["x"] - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < tol, (prec, np.abs(dx).max())
        assert np.abs(st["v"] - ref["v"]).max() < 10 * tol
        assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))
        assert t["K"] == pytest.approx(ref["K"], rel=max(tol, 1e-11))


@pytest.mark.parametrize("d,N", [(3, 500), (5, 700)])
def test_fire_minimum_checked_by_oracle(H, d, N):
    s, x0 = _start(d, N, 20 + d, 0.005)
    for prec in (H.HDMD_MIXED, H.HDMD_FP64):
        with H.System(d, s.L, s.sigma, x0, None, s.mass, skin=SKIN, precision=prec, **LAW) as g:
            r = g.fire(max_iter=200000)
            xs = g.state()["x"]
        assert r["converged"], r
        with oracle.law("morse", A, eps_scale=True):
            Fo, Eo, _ = oracle.forces(xs, s.sigma, s.L)
        assert np.linalg.norm(Fo, axis=1).max() < 1e-10
        # with every pair force below 1e-10 and the Morse stiffness 2 a^2 at
        # contact, a residual overlap holds at most 1e-20 / (4 a^2) of energy;
        # over all pairs that bounds what rounding of x may add or remove
        assert r["E_pair"] == pytest.approx(Eo, rel=1e-6, abs=1e-18)


def test_swap_with_masses_matches_serial_oracle(H):
    s, x0 = _start(3, 600, 8, 0.005)
    rng = np.random.default_rng(8)
    pairs, u = W.swap_pairs(rng, s.N, s.N // 3)
    T = W.PAPER_T
    with oracle.law("morse", A, eps_scale=True):
        ref = oracle.swap(x0, s.sigma, s.L, T, pairs, u, mass=s.mass, v=s.v)
    assert 0 < ref["naccepted"] < len(pairs)
    for prec in (H.HDMD_FP64, H.HDMD_MIXED):
        with H.System(3, s.L, s.sigma, x0, s.v, s.mass, skin=SKIN, precision=prec, **LAW) as g:
            nacc, flags = g.swap(T, pairs=pairs, uniforms=u)
            st = g.state(sigma=True)
        assert nacc == ref["naccepted"]
        assert (flags == ref["accepted"]).all()
        assert (st["sigma"] == ref["sigma"]).all()
        assert np.abs(st["v"] - ref["v"]).max() <= 1e-14 * np.abs(ref["v"]).max()


@pytest.mark.parametrize("law,masses", [("morse", False), ("harmonic", True), ("morse", True)])
def test_fire_first_iterations_follow_oracle(H, law, masses):
    s, x0 = _start(3, 300, 31, 0.01)
    m = s.mass if masses else None
    for it in (1, 5, 40):
        with oracle.law(law, A, eps_scale=True):
            ref = oracle.fire(x0, s.sigma, s.L, skin=SKIN, mass=m, max_iter=it)
        with H.System(3, s.L, s.sigma, x0, None, m, skin=SKIN, precision=H.HDMD_FP64,
                      law=law, a=A, eps_scale=True) as g:
            r = g.fire(max_iter=it)
            xs = g.state()["x"]
        assert r["iterations"] == ref["iters"] == it
        dx = xs - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < 1e-10, (it, np.abs(dx).max())
        assert r["E_pair"] == pytest.approx(ref["E"], rel=1e-10)


@pytest.mark.parametrize("row", read_golden("paper_list_sizes.txt"))
def test_list_sizes_match_the_paper(H, row):
    """The paper prints the mean list size of its runs at phi*_d (Sec. III).
    After the pushoff and ten time units of MD at T = 0.25, the liquid's
    mean list length (list radius sigma_ij + 0.25) is within 2 % of it (the
    uniform random start, before the liquid forms contacts, is ~15 % lower,
    and after one time unit still ~4 %)."""
    d, nvl = int(row[0]), float(row[1])
    s = W.paper_model(d, 20000, seed=40 + d)
    with H.System(d, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        g.fire(max_iter=20000)
        x0 = g.state(v=False, img=False)["x"]
    with H.System(d, s.L, s.sigma, x0, s.v, s.mass, skin=SKIN, precision=H.HDMD_MIXED, **LAW) as g:
        g.md_steps(10 * int(round(1.0 / W.PAPER_DT)), W.PAPER_DT)
        g.build_neighbors(force=True)
        z = g.info()["total_list_entries"] / s.N
    assert z == pytest.approx(nvl, rel=0.02), z
