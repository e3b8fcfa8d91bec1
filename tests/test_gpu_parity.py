"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (stated once, used below):
  neighbour lists  identical sets, except pairs whose oracle FP64 distance
                   lies within 1e-6 of sigma_ij + skin (either answer valid);
  forces           max_i |F_gpu - F_oracle| <= tol * max_i |F_oracle| with
                   tol = 1e-12 (FP64) and 1e-5 (mixed: FP32 pair arithmetic);
  energy, virial   relative 1e-12 (FP64), 1e-5 (mixed);
  short MD         100 steps of the d=3 bidisperse system: positions within
                   1e-9 (FP64) and 1e-5 (mixed) of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2112_12271_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIE = 1e-6


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_12271_gb300 import build, hdmd
    build.build()
    oracle.build()
    return hdmd


def tie_pairs(x, sigma, L, skin):
    """Pairs (i, j) whose FP64 distance is within TIE of the list radius."""
    N = len(x)
    out = set()
    for i in range(N):
        dx = x - x[i]
        dx -= L * np.round(dx / L)
        r = np.sqrt((dx * dx).sum(axis=1))
        rc = 0.5 * (sigma + sigma[i]) + skin
        for j in np.nonzero(np.abs(r - rc) <= TIE)[0]:
            if j != i:
                out.add((i, int(j)))
    return out


def compare_lists(gpu, ref, ties):
    gs = oracle.lists_as_sets(*gpu)
    rs = oracle.lists_as_sets(*ref)
    for i, (a, b) in enumerate(zip(gs, rs)):
        for j in a ^ b:
            assert (i, j) in ties, (i, j)


LIST_CASES = [  # d, N, L : covers n_cell = 1 (all pairs), 2, 3 and larger, ragged N
    (2, 700, 22.0), (3, 1000, 11.78), (3, 333, 4.6), (4, 900, 6.3), (5, 777, 4.7),
    (6, 1500, 4.4), (6, 4096, 6.0), (7, 500, 3.3), (8, 600, 3.1), (9, 300, 3.05),
    (10, 250, 3.02), (3, 200, 2.9), (6, 300, 2.6), (10, 120, 2.5),
]


@pytest.mark.parametrize("d,N,L", LIST_CASES)
def test_neighbor_lists_match_oracle(H, d, N, L):
    rng = np.random.default_rng(100 + d)
    x = W.uniform_positions(rng, N, d, L)
    sigma = W.polydisperse(rng, N)
    ref = oracle.neighbors_brute(x, sigma, L, 0.3)
    ties = tie_pairs(x, sigma, L, 0.3)
    for prec in (H.HDMD_FP64, H.HDMD_MIXED):
        with H.System(d, L, sigma, x, precision=prec) as g:
            got = g.neighbors()
            assert got[0].sum() == len(got[1])
            compare_lists(got, ref, ties)


def test_half_stencil_lists_match_oracle_and_repeat(H):
    """A system with many candidates per atom (3^d times the atoms per
    subcell >= 4000: here d = 6, n_cell = 3, ~11 atoms per subcell) takes the
    half-stencil build: each pair tested once and entered in both lists at
    slots taken by atomics, then every list sorted by neighbour index.  The
    sets equal the oracle's brute force, and a forced rebuild gives the same
    lists and order bit for bit."""
    rng = np.random.default_rng(7)
    d, N, L = 6, 8192, 4.6
    x = W.uniform_positions(rng, N, d, L)
    sigma = W.polydisperse(rng, N)
    ref = oracle.neighbors_brute(x, sigma, L, 0.3)
    ties = tie_pairs(x, sigma, L, 0.3)
    with H.System(d, L, sigma, x, precision=H.HDMD_MIXED) as g:
        assert g.info()["n_cell"] == 3
        a = g.neighbors()
        compare_lists(a, ref, ties)
        g.build_neighbors(force=True)
        b = g.neighbors()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("lanes", [1, 2, 8, 32])
def test_lanes_per_atom_layouts(H, lanes):
    s = W.c1_poly_d6(N=2048)
    ref = oracle.neighbors_brute(s.x, s.sigma, s.L, 0.3)
    Fo, Eo, _ = oracle.forces(s.x, s.sigma, s.L)
    with H.System(s.d, s.L, s.sigma, s.x, precision=H.HDMD_FP64) as g:
        g.tune(lanes_per_atom=lanes)
        compare_lists(g.neighbors(), ref, tie_pairs(s.x, s.sigma, s.L, 0.3))
        F, E, _ = g.forces()
        assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
        assert E == pytest.approx(Eo, rel=1e-12)


FORCE_CASES = [(3, 1000, 0.6, "bi"), (4, 800, 0.45, "poly"), (6, 2000, 0.15, "poly"),
               (8, 700, 0.01, "poly"), (2, 500, 0.8, "bi"), (10, 300, 1e-4, "poly")]


@pytest.mark.parametrize("d,N,phi,dist", FORCE_CASES)
def test_forces_energy_virial_match_oracle(H, d, N, phi, dist):
    s = W.make_system(d, N, phi=phi, dist=dist, T=1e-3, seed=d)
    assert s.L > 2 * s.sigma.max()
    Fo, Eo, Wo = oracle.forces(s.x, s.sigma, s.L)
    assert Eo > 0
    for prec, tol in ((H.HDMD_FP64, 1e-12), (H.HDMD_MIXED, 1e-5)):
        with H.System(d, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            F, E, Wv = g.forces()
            assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max(), prec
            assert E == pytest.approx(Eo, rel=tol)
            assert Wv == pytest.approx(Wo, rel=tol)
            assert np.abs(F.sum(axis=0)).max() <= 10 * tol * np.abs(Fo).max() * np.sqrt(N)


def test_short_trajectory_matches_oracle(H):
    s = W.c0_bidisperse_d3()
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005)
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            t = g.md_steps(100, 0.005)
            st = g.state(f=True)
            dx = st["x"] - ref["x"]
            dx -= s.L * np.round(dx / s.L)
            assert np.abs(dx).max() < tol, (prec, np.abs(dx).max())
            assert np.abs(st["v"] - ref["v"]).max() < 10 * tol
            # unwrapped positions agree too (image counts)
            ux = st["x"] + s.L * st["img"]
            rx = ref["x"] + s.L * ref["img"]
            assert np.abs(ux - rx).max() < tol + 1e-9 * s.L
            assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))
            assert t["K"] == pytest.approx(ref["K"], rel=max(tol, 1e-11))
            assert t["rebuilds"] >= 1


def test_md_in_pieces_equals_one_call_and_is_deterministic(H):
    s = W.make_system(4, 1200, phi=0.4, dist="poly", T=1e-2, seed=3)
    outs = []
    for pieces in ((60,), (13, 47), (60,)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
            for n in pieces:
                g.md_steps(n, 0.005)
            outs.append(g.state())
    assert np.array_equal(outs[0]["x"], outs[2]["x"])      # bitwise repeatable
    assert np.abs(outs[0]["x"] - outs[1]["x"]).max() < 1e-12


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_rebuild_schedule_repeats_bitwise(H, prec):
    """The trigger's |dlt|^2 is summed per atom in axis order (no atomics),
    so the same start gives the same rebuild steps and the same bits: three
    runs of 600 steps of a hot d = 6 system that rebuilds every few steps
    (many trigger evaluations close to the threshold s/2)."""
    s = W.make_system(6, 4000, L=5.6, dist="poly", T=0.5, seed=17)
    p = H.HDMD_MIXED if prec == "mixed" else H.HDMD_FP64
    outs = []
    for _ in range(3):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=p) as g:
            t = g.md_steps(600, 0.005)
            outs.append((g.state(), t))
    assert outs[0][1]["rebuilds"] >= 30
    for st, t in outs[1:]:
        assert t["rebuilds"] == outs[0][1]["rebuilds"]
        assert np.array_equal(st["x"], outs[0][0]["x"])
        assert np.array_equal(st["v"], outs[0][0]["v"])
        assert t["E_pair"] == outs[0][1]["E_pair"]


def test_graphs_and_eager_paths_agree(H):
    s = W.make_system(6, 3000, L=5.2, dist="poly", T=1e-3, seed=11)
    res = []
    for graphs in (1, 0):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
            g.tune(use_graphs=graphs)
            t = g.md_steps(150, 0.005)
            res.append((g.state(), t))
    assert np.array_equal(res[0][0]["x"], res[1][0]["x"])
    assert res[0][1]["E_pair"] == res[1][1]["E_pair"]


def test_energy_conservation_and_drift(H):
    s = W.c0_bidisperse_d3()
    with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=H.HDMD_MIXED) as g:
        t0 = g.md_steps(200, 0.005)
        H0 = t0["E_pair"] + t0["K"]
        hs = []
        for _ in range(20):
            t = g.md_steps(100, 0.005)
            hs.append(t["E_pair"] + t["K"])
    hs = np.array(hs)
    assert np.abs(hs - H0).max() < 1e-3 * abs(H0)


def test_list_overflow_grows_and_redoes(H):
    # all atoms packed in one corner: the density-based first guess is far too small
    rng = np.random.default_rng(5)
    d, N, L = 3, 600, 20.0
    x = rng.uniform(-10, -7.5, size=(N, d))
    sigma = W.polydisperse(rng, N)
    with H.System(d, L, sigma, x, precision=H.HDMD_FP64) as g:
        info = g.info()
        assert info["max_list_length"] <= info["list_capacity"]
        compare_lists(g.neighbors(), oracle.neighbors_brute(x, sigma, L, 0.3),
                      tie_pairs(x, sigma, L, 0.3))
        F, E, _ = g.forces()
        Fo, Eo, _ = oracle.forces(x, sigma, L)
        assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()


def test_lost_atom_is_reported(H):
    s = W.make_system(3, 200, phi=0.3, dist="bi", T=0.0, seed=1)
    v = np.zeros_like(s.x)
    v[5, 0] = 1e4 / 0.005      # one step moves it far beyond L/4
    with H.System(s.d, s.L, s.sigma, s.x, v, precision=H.HDMD_MIXED) as g:
        with pytest.raises(H.HDMDError) as e:
            g.md_steps(3, 0.005)
        assert e.value.status == 4


def test_edge_cases(H):
    # two atoms, overlapping, smallest legal box
    x = np.array([[0.0, 0.0], [0.5, 0.0]])
    sig = np.array([1.0, 1.0])
    L = 2 * (1.0 + 0.3)
    with H.System(2, L, sig, x, precision=H.HDMD_FP64) as g:
        F, E, _ = g.forces()
        assert E == pytest.approx(0.5 * 0.25, rel=1e-14)
        assert F[0, 0] == pytest.approx(-0.5, rel=1e-14)
    # dilute: every list empty
    s = W.make_system(3, 100, phi=0.001, dist="poly", T=0.0, seed=2)
    with H.System(3, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        c, idx = g.neighbors()
        F, E, _ = g.forces()
        ref = oracle.neighbors_brute(s.x, s.sigma, s.L, 0.3)
        assert (c == ref[0]).all()
        assert E == 0.0 or E == pytest.approx(oracle.forces(s.x, s.sigma, s.L)[1], rel=1e-5)
    # bad arguments are rejected with a status, not a fault
    with pytest.raises(H.HDMDError):
        H.System(3, 1.0, np.ones(4), np.zeros((4, 3)))
    with H.System(3, 10.0, np.ones(4), np.zeros((4, 3))) as g:
        with pytest.raises(H.HDMDError):
            g.md_steps(-1, 0.005)
        bad = np.zeros((4, 3)); bad[0, 0] = np.nan
        with pytest.raises(H.HDMDError):
            g.set_state(bad)


# ------------------------------------------------------------------ FIRE
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fire_two_spheres(H, prec):
    x = np.array([[0.0, 0.0, 0.0], [0.7, 0.1, 0.0]])
    sig = np.array([1.0, 1.4])
    p = H.HDMD_FP64 if prec == "fp64" else H.HDMD_MIXED
    with H.System(3, 10.0, sig, x, precision=p) as g:
        r = g.fire()
        assert r["converged"] and r["fmax"] < 1e-10
        xs = g.state()["x"]
    d = np.linalg.norm(xs[1] - xs[0])
    assert d >= 1.2 * (1 - 1e-9)


@pytest.mark.parametrize("d,N,phi,dist", [(3, 500, 0.35, "bi"), (4, 800, 0.3, "poly"),
                                          (6, 1500, 0.12, "poly"), (3, 256, 0.9, "bi")])
def test_fire_reaches_tolerance_checked_by_oracle(H, d, N, phi, dist):
    s = W.make_system(d, N, phi=phi, dist=dist, T=0.0, seed=20 + d)
    for prec in (H.HDMD_MIXED, H.HDMD_FP64):
        with H.System(d, s.L, s.sigma, s.x, precision=prec) as g:
            r = g.fire()
            assert r["converged"], r
            xs = g.state()["x"]
        Fo, Eo, _ = oracle.forces(xs, s.sigma, s.L)
        assert np.linalg.norm(Fo, axis=1).max() < 1e-10
        assert r["E_pair"] == pytest.approx(Eo, rel=1e-6, abs=1e-20)
        if prec == H.HDMD_MIXED and r["fmax"] < 1e-10:
            assert r["polish_iterations"] >= 0


def test_fire_first_iterations_follow_oracle(H):
    s = W.make_system(3, 300, phi=0.5, dist="bi", T=0.0, seed=4)
    for it in (1, 5, 40):
        ref = oracle.fire(s.x, s.sigma, s.L, max_iter=it)
        with H.System(3, s.L, s.sigma, s.x, precision=H.HDMD_FP64) as g:
            r = g.fire(max_iter=it)
            assert r["iterations"] == ref["iters"] == it
            xs = g.state()["x"]
        dx = xs - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < 1e-10, (it, np.abs(dx).max())
        assert r["E_pair"] == pytest.approx(ref["E"], rel=1e-10)


def test_fire_dt_floor_and_mixing_with_masses_follow_oracle(H):
    """FIRE 2.0 as published, where the two readings of its back-off and
    mixing part: masses sigma^3 of unequal size (so the mixing after a
    restart from rest moves v off F/m), and dt_max = 0.0095 below
    dt_min / f_dec = 0.0098, so the P < 0 step at iteration 128 keeps dt
    (a floor at dt_min would set it to 0.0049).  Positions after 1, 127,
    128, 129 and 160 iterations, and the iteration count at convergence,
    against the oracle; the mixed precision path at the end too."""
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.05, 0.0], [1.8, 0.0, 0.0],
                  [-4.0, 0.0, 0.0], [-4.0, 0.9, 0.0]])
    sig = np.array([1.0, 1.0, 1.4, 1.2, 0.9])
    m, L = sig ** 3, 12.0
    kw = dict(dt_min=0.0049, dt_max=0.0095)
    a = oracle.fire(x, sig, L, mass=m, max_iter=128, **kw)
    assert float((a["F"] * a["v"]).sum()) < 0     # the P < 0 step the test is about
    for it in (1, 127, 128, 129, 160, None):
        p = dict(kw) if it is None else dict(kw, max_iter=it)
        ref = oracle.fire(x, sig, L, mass=m, **p)
        for prec in ((H.HDMD_FP64, H.HDMD_MIXED) if it is None else (H.HDMD_FP64,)):
            with H.System(3, L, sig, x, None, m, precision=prec) as g:
                r = g.fire(**p)
                xs = g.state()["x"]
            if it is not None:
                assert r["iterations"] == ref["iters"] == it
            else:
                assert ref["status"] == 0 and r["converged"]
                if prec == H.HDMD_FP64:
                    assert r["iterations"] == ref["iters"]
            dx = xs - ref["x"]
            dx -= L * np.round(dx / L)
            # mixed: FP32 pair forces until the FP64 polish, so the path to
            # the (flat, E = 0) minimum differs by their rounding
            tol = 1e-10 if prec == H.HDMD_FP64 else 1e-4
            assert np.abs(dx).max() < tol, (it, prec, np.abs(dx).max())


# ------------------------------------------------------------------ SWAP
@pytest.mark.parametrize("d,N,phi", [(3, 400, 0.6), (5, 600, 0.2), (8, 400, 0.008)])
def test_swap_matches_serial_oracle(H, d, N, phi):
    s = W.make_system(d, N, phi=phi, dist="bi", T=0.0, seed=30 + d)
    assert s.L > 2 * s.sigma.max()
    rng = np.random.default_rng(d)
    pairs, u = W.swap_pairs(rng, N, N // 3)
    T = 0.02
    ref = oracle.swap(s.x, s.sigma, s.L, T, pairs, u)
    assert 0 < ref["naccepted"] < len(pairs)
    for prec in (H.HDMD_FP64, H.HDMD_MIXED):
        with H.System(d, s.L, s.sigma, s.x, precision=prec) as g:
            nacc, flags = g.swap(T, pairs=pairs, uniforms=u)
            sig = g.state(sigma=True)["sigma"]
        assert nacc == ref["naccepted"]
        assert (flags == ref["accepted"]).all()
        assert (sig == ref["sigma"]).all()


def test_seeded_swap_equals_oracle_draw(H):
    s = W.make_system(4, 500, phi=0.35, dist="bi", T=0.0, seed=6)
    T = 0.05
    sig = s.sigma.copy()
    total = 0
    for sweep in range(3):
        pairs, u = oracle.swap_draw(99, sweep, round(0.1 * s.N), s.N)
        r = oracle.swap(s.x, sig, s.L, T, pairs, u)
        sig = r["sigma"]
        total += r["naccepted"]
    with H.System(4, s.L, s.sigma, s.x, precision=H.HDMD_MIXED) as g:
        nacc, _ = g.swap(T, p=0.1, nsweeps=3, seed=99)
        gs = g.state(sigma=True)["sigma"]
    assert nacc == total
    assert (gs == sig).all()


def test_paper_rebuild_rule_matches_oracle(H):
    """The paper's rule (Sec. II.C) every n_bet = 5 steps: the same rebuild
    schedule as the oracle under that rule, hence the same (inexact) lists
    and the same trajectory; calls in pieces keep the step count."""
    s = W.make_system(3, 600, phi=0.5, dist="poly", T=0.05, seed=4)
    ref = oracle.md_steps(s.x, s.v, s.sigma, s.L, 100, 0.005, rule="paper", n_bet=5)
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(3, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            g.rebuild_rule("paper", 5)
            t1 = g.md_steps(37, 0.005)
            t2 = g.md_steps(63, 0.005)
            st = g.state()
        assert t1["rebuilds"] + t2["rebuilds"] + 1 == ref["builds"]
        dx = st["x"] - ref["x"]
        dx -= s.L * np.round(dx / s.L)
        assert np.abs(dx).max() < tol, (prec, np.abs(dx).max())
        assert t2["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))


@pytest.mark.parametrize("d,N,L", [(3, 1000, 11.78), (6, 1500, 4.4), (8, 600, 3.1)])
def test_global_list_radius_matches_oracle(H, d, N, L):
    """The paper's single list radius sigma_max + s (Sec. II.C): the lists
    equal the oracle's global-radius lists (ties within 1e-6 excepted) and
    the forces are unchanged."""
    rng = np.random.default_rng(d)
    x = W.uniform_positions(rng, N, d, L)
    sigma = W.polydisperse(rng, N)
    ref = oracle.neighbors_brute(x, sigma, L, 0.3, global_cut=True)
    rc = sigma.max() + 0.3
    for prec, tol in ((H.HDMD_FP64, 1e-12), (H.HDMD_MIXED, 1e-5)):
        with H.System(d, L, sigma, x, precision=prec) as g:
            F0, E0, _ = g.forces()
            g.list_radius(True)
            got = g.neighbors()
            F1, E1, _ = g.forces()
        gs, rs = oracle.lists_as_sets(*got), oracle.lists_as_sets(*ref)
        for i, (a, b) in enumerate(zip(gs, rs)):
            for j in a ^ b:
                dx = x[j] - x[i]
                dx -= L * np.round(dx / L)
                assert abs(np.sqrt(dx @ dx) - rc) <= TIE, (i, j)
        assert got[0].sum() > 0
        # the same pairs interact; only the summation order changes
        assert np.abs(F1 - F0).max() <= tol * max(np.abs(F0).max(), 1e-300)
