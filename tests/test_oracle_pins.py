"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics (closed forms, exact lattice counts, invariants, brute force),
never against the oracle's own formulas retyped.  CPU only."""
import math

import numpy as np
import pytest

from conftest import read_golden
from paper_2112_12271_gb300 import workloads as W


# ------------------------------------------------------------------ geometry
def test_sphere_volume_closed_forms(orc):
    # Eq. (2) against the textbook volumes of balls of radius r = sigma/2
    r = 0.65
    s = 2 * r
    assert orc.sphere_volume(2, s) == pytest.approx(math.pi * r ** 2, rel=1e-14)
    assert orc.sphere_volume(3, s) == pytest.approx(4.0 / 3.0 * math.pi * r ** 3, rel=1e-14)
    assert orc.sphere_volume(4, s) == pytest.approx(0.5 * math.pi ** 2 * r ** 4, rel=1e-14)
    assert orc.sphere_volume(6, s) == pytest.approx(math.pi ** 3 / 6 * r ** 6, rel=1e-14)
    # the input generator's copy agrees
    for d in range(2, 11):
        assert W.sphere_volume(d, s) == pytest.approx(orc.sphere_volume(d, s), rel=1e-14)


def test_benchmark_geometry_golden(orc):
    rows = read_golden("benchmark_geometry.txt")
    sysd3 = W.c0_bidisperse_d3()
    assert sysd3.L == pytest.approx(float(rows[0][4]), abs=1e-5)
    assert orc.n_cell(sysd3.L, 1.4 + 0.3) == int(rows[0][5])
    sysd6 = W.c1_poly_d6(N=4096)
    assert orc.n_cell(6.0, sysd6.sigma.max() + 0.3) == int(rows[1][5])
    # hand check of V_part for the bidisperse system
    vpart = 500 * math.pi / 6 * (1 + 1.4 ** 3)
    assert sysd3.L == pytest.approx((vpart / 0.6) ** (1 / 3), rel=1e-12)


def test_cell_index_hand_examples(orc):
    # Eq. (9), axis 1 most significant
    assert orc.cell_index(2, 3, [0, 0]) == 0
    assert orc.cell_index(2, 3, [0, 2]) == 2
    assert orc.cell_index(2, 3, [1, 0]) == 3
    assert orc.cell_index(2, 3, [2, 2]) == 8
    assert orc.cell_index(3, 4, [1, 2, 3]) == 27
    assert orc.n_cell(10.0, 2.5) == 4
    assert orc.n_cell(9.99, 2.5) == 3


def test_min_image(orc):
    assert orc.min_image(4.0, 10.0) == pytest.approx(4.0)
    assert orc.min_image(6.0, 10.0) == pytest.approx(-4.0)
    assert orc.min_image(-6.0, 10.0) == pytest.approx(4.0)


# ------------------------------------------------------------------ lists
@pytest.mark.parametrize("row", read_golden("lattice_neighbor_counts.txt"))
def test_lattice_counts(orc, row):
    d, n, rad, expect = int(row[0]), int(row[1]), float(row[2]), int(row[3])
    x, L = W.lattice(d, n)
    sigma = np.ones(len(x))
    skin = rad - 1.0
    for fn in (orc.neighbors_brute, orc.neighbors_cells):
        counts, idx = fn(x, sigma, L, skin)
        assert (counts == expect).all(), (fn.__name__, np.unique(counts))


def _random_system(d, N, L, seed):
    rng = np.random.default_rng(seed)
    return W.uniform_positions(rng, N, d, L), W.polydisperse(rng, N)


@pytest.mark.parametrize("d,N,L", [(2, 400, 14.0), (3, 500, 7.0), (3, 300, 4.6),
                                   (4, 600, 6.2), (5, 500, 4.6), (6, 700, 4.1),
                                   (7, 300, 3.2), (8, 300, 3.1), (9, 200, 3.05),
                                   (10, 200, 3.02)])
def test_cells_equal_brute(orc, d, N, L):
    x, sigma = _random_system(d, N, L, seed=d * 7 + N)
    for gc in (False, True):
        cb, ib = orc.neighbors_brute(x, sigma, L, 0.3, global_cut=gc)
        cc, ic = orc.neighbors_cells(x, sigma, L, 0.3, global_cut=gc)
        assert (cb == cc).all()
        assert (ib == ic).all()
        sets = orc.lists_as_sets(cb, ib)
        for i, s in enumerate(sets):   # j in VL(i) <=> i in VL(j)
            for j in s:
                assert i in sets[j]
    # explicit distance check of a few pairs against the plain definition,
    # per-pair radius sigma_ij + s and one global radius sigma_max + s
    sets = orc.lists_as_sets(*orc.neighbors_brute(x, sigma, L, 0.3))
    gsets = orc.lists_as_sets(*orc.neighbors_brute(x, sigma, L, 0.3, global_cut=True))
    for i in range(0, N, max(1, N // 7)):
        for j in range(N):
            if j == i:
                continue
            dx = x[j] - x[i]
            dx -= L * np.round(dx / L)
            inside = float(dx @ dx) < (0.5 * (sigma[i] + sigma[j]) + 0.3) ** 2
            assert inside == (j in sets[i])
            assert (float(dx @ dx) < (sigma.max() + 0.3) ** 2) == (j in gsets[i])


def test_cells_with_atoms_on_the_box_faces(orc):
    """Coordinates at -L/2 and at the last value below +L/2 lie in the first
    and the last subcell (Eq. (8)); the subcell search still equals brute
    force."""
    d, N, L = 3, 300, 7.0
    x, sigma = _random_system(d, N, L, seed=11)
    top = np.nextafter(0.5 * L, 0.0)
    x[:40, 0] = top
    x[40:80, 1] = -0.5 * L
    x[80:100, 2] = top
    x[100:110] = top
    for gc in (False, True):
        cb, ib = orc.neighbors_brute(x, sigma, L, 0.3, global_cut=gc)
        cc, ic = orc.neighbors_cells(x, sigma, L, 0.3, global_cut=gc)
        assert (cb == cc).all() and (ib == ic).all()


@pytest.mark.parametrize("row", read_golden("lattice_neighbor_counts.txt")[:6])
def test_single_atom_lists_on_lattices(orc, row):
    d, n, rad, expect = int(row[0]), int(row[1]), float(row[2]), int(row[3])
    x, L = W.lattice(d, n)
    sigma = np.ones(len(x))
    for i in (0, len(x) // 2, len(x) - 1):
        assert len(orc.neighbors_of(x, sigma, L, rad - 1.0, i)) == expect


@pytest.mark.parametrize("d,N,L", [(3, 300, 4.6), (6, 400, 4.1), (9, 150, 3.05)])
def test_single_atom_lists_and_forces_are_rows_of_all_pairs(orc, d, N, L):
    x, sigma = _random_system(d, N, L, seed=3 * d + N)
    cb, ib = orc.neighbors_brute(x, sigma, L, 0.3)
    off = np.concatenate([[0], np.cumsum(cb)])
    F, E, Wv = orc.forces(x, sigma, L)
    es = ws = 0.0
    for i in range(N):
        assert (orc.neighbors_of(x, sigma, L, 0.3, i) == ib[off[i]:off[i + 1]]).all()
        Fi, ei, wi = orc.force_on(x, sigma, L, i)
        assert np.abs(Fi - F[i]).max() <= 1e-13 * max(np.abs(F).max(), 1e-300)
        es += ei
        ws += wi
    assert es == pytest.approx(E, rel=1e-12)
    assert ws == pytest.approx(Wv, rel=1e-12)


def test_cells_need_two_subcells(orc):
    x, sigma = _random_system(3, 50, 2.5, 0)
    with pytest.raises(ValueError):
        orc.neighbors_cells(x, sigma, 2.5, 0.3)


# ------------------------------------------------------------------ forces
def test_two_body_closed_form(orc):
    L = 10.0
    for (xa, xb, sep) in [(-0.4, 0.4, 0.8), (-4.9, 4.7, 0.4)]:   # second pair wraps
        x = np.array([[xa, 0.0, 0.0], [xb, 0.0, 0.0]])
        sig = np.array([1.0, 1.0])
        F, E, Wv = orc.forces(x, sig, L)
        g = 1.0 - sep
        assert E == pytest.approx(0.5 * g * g, rel=1e-13)
        # |f| = (eps/sigma)(1 - r/sigma), repulsive; virial = r |f|
        direction = np.sign(orc.min_image(xa - xb, L))
        assert F[0, 0] == pytest.approx(direction * g, rel=1e-13)
        assert F[1, 0] == pytest.approx(-direction * g, rel=1e-13)
        assert Wv == pytest.approx(sep * g, rel=1e-13)
    # unequal diameters: sigma_ij = 1.2, eps = 2
    x = np.array([[0.0, 0.0], [0.6, 0.8]])
    F, E, Wv = orc.forces(x, np.array([1.0, 1.4]), 10.0, eps=2.0)
    g = 1.0 - 1.0 / 1.2
    assert E == pytest.approx(0.5 * 2.0 * g * g, rel=1e-13)
    assert np.linalg.norm(F[0]) == pytest.approx(2.0 / 1.2 * g, rel=1e-13)
    # touching or apart: nothing
    F, E, Wv = orc.forces(np.array([[0.0, 0.0], [1.2, 0.0]]), np.array([1.0, 1.4]), 10.0)
    assert E == 0.0 and not F.any()


def _dense(d, N, phi, seed):
    s = W.make_system(d, N, phi=phi, dist="poly", T=1e-3, seed=seed)
    return s.x, s.sigma, s.L


@pytest.mark.parametrize("d", [2, 3, 4, 6])
def test_force_is_minus_gradient(orc, d):
    x, sigma, L = _dense(d, 40, 0.5 if d < 5 else 0.25, seed=d)
    F, E, _ = orc.forces(x, sigma, L)
    h = 1e-6
    rng = np.random.default_rng(d)
    for i in rng.choice(len(x), 8, replace=False):
        for k in range(d):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd = -(orc.forces(xp, sigma, L)[1] - orc.forces(xm, sigma, L)[1]) / (2 * h)
            assert fd == pytest.approx(F[i, k], rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("d", [3, 5, 8])
def test_newton_third_law_and_list_equals_brute(orc, d):
    x, sigma, L = _dense(d, 300, 0.45 * W.jamming_estimate(d) / 0.7 + 0.1, seed=11 + d)
    Fb, Eb, Wb = orc.forces(x, sigma, L)
    lists = orc.neighbors_cells(x, sigma, L, 0.3) if orc.n_cell(L, sigma.max() + 0.3) >= 2 \
        else orc.neighbors_brute(x, sigma, L, 0.3)
    Fl, El, Wl = orc.forces(x, sigma, L, lists=lists)
    scale = np.abs(Fb).max()
    assert scale > 0
    assert np.abs(Fl.sum(axis=0)).max() < 1e-12 * scale * len(x)
    assert np.abs(Fl - Fb).max() < 1e-13 * scale
    assert El == pytest.approx(Eb, rel=1e-12)
    assert Wl == pytest.approx(Wb, rel=1e-12)


@pytest.mark.parametrize("d", [3, 6])
def test_virial_from_volume_scaling(orc, d):
    # W = sum_{i<j} r_ij . f_ij = -dE/dlambda under x -> lambda x, L -> lambda L
    x, sigma, L = _dense(d, 60, 0.55 if d == 3 else 0.2, seed=5)
    _, E0, Wv = orc.forces(x, sigma, L)
    h = 1e-6
    Ep = orc.forces(x * (1 + h), sigma, L * (1 + h))[1]
    Em = orc.forces(x * (1 - h), sigma, L * (1 - h))[1]
    assert Wv == pytest.approx(-(Ep - Em) / (2 * h), rel=1e-6)


def test_translation_invariance(orc):
    x, sigma, L = _dense(4, 80, 0.4, seed=3)
    F, E, Wv = orc.forces(x, sigma, L)
    y = x + np.array([0.37, -1.1, 2.9, 0.05])
    y = (y + 0.5 * L) % L - 0.5 * L
    F2, E2, W2 = orc.forces(y, sigma, L)
    assert E2 == pytest.approx(E, rel=1e-12)
    assert np.abs(F2 - F).max() < 1e-12 * np.abs(F).max()


# ------------------------------------------------------------------ velocity Verlet
def test_head_on_collision_closed_form(orc):
    # equal spheres (sigma = m = 1) approach at relative speed 1; in contact
    # the separation obeys r'' = 2 (1 - r): half a period pi/sqrt(2); then
    # the velocities are exchanged (elastic, equal masses).
    L = 10.0
    x = np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    v = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    sig = np.ones(2)
    dt = 0.001
    t_end = 5.0
    out = orc.md_steps(x, v, sig, L, int(round(t_end / dt)), dt, skin=0.3)
    t_exit = 1.0 + math.pi / math.sqrt(2.0)
    xa = -0.5 - 0.5 * (t_end - t_exit)
    assert out["x"][0, 0] == pytest.approx(xa, abs=2e-6)
    assert out["x"][1, 0] == pytest.approx(-xa, abs=2e-6)
    assert out["v"][0, 0] == pytest.approx(-0.5, abs=2e-6)   # O(dt^2)
    assert out["v"][1, 0] == pytest.approx(0.5, abs=2e-6)


def test_time_reversibility_and_momentum(orc):
    s = W.make_system(3, 200, phi=0.55, dist="bi", T=1e-2, seed=4)
    fwd = orc.md_steps(s.x, s.v, s.sigma, s.L, 200, 0.005)
    assert np.abs(fwd["v"].sum(axis=0)).max() < 1e-12
    back = orc.md_steps(fwd["x"], -fwd["v"], s.sigma, s.L, 200, 0.005, F=fwd["F"])
    dx = back["x"] - s.x
    dx -= s.L * np.round(dx / s.L)
    assert np.abs(dx).max() < 1e-9
    assert np.abs(back["v"] + s.v).max() < 1e-9
    assert fwd["builds"] >= 2      # the trigger fired on the way


def test_energy_error_scales_as_dt_squared(orc):
    s = W.make_system(3, 150, phi=0.60, dist="bi", T=1e-2, seed=8)
    errs = []
    for dt in (0.01, 0.005):
        n = int(round(2.0 / dt))
        F, E0, _ = orc.forces(s.x, s.sigma, s.L)
        H0 = E0 + orc.kinetic(s.v)
        dev, x, v = 0.0, s.x, s.v
        for _ in range(20):
            o = orc.md_steps(x, v, s.sigma, s.L, n // 20, dt, F=F)
            x, v, F = o["x"], o["v"], o["F"]
            dev = max(dev, abs(o["E"] + o["K"] - H0))
        errs.append(dev)
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.5, errs


# ------------------------------------------------------------------ FIRE
def test_fire_two_spheres_reach_contact(orc):
    x = np.array([[0.0, 0.0, 0.0], [0.7, 0.1, 0.0]])
    sig = np.array([1.0, 1.4])
    out = orc.fire(x, sig, 10.0)
    assert out["status"] == 0
    r = np.linalg.norm(out["x"][1] - out["x"][0])
    assert r >= 1.2 * (1 - 1e-9)
    assert out["E"] < 1e-19
    assert out["fmax"] < 1e-10


def test_fire_unjammed_packing_reaches_zero_energy(orc):
    s = W.make_system(3, 200, phi=0.35, dist="bi", T=0.0, seed=2)
    E0 = orc.forces(s.x, s.sigma, s.L)[1]
    out = orc.fire(s.x, s.sigma, s.L)
    assert out["status"] == 0 and out["fmax"] < 1e-10
    assert E0 > 1.0 and out["E"] < 1e-18


def test_fire_jammed_packing_converges_with_residual_energy(orc):
    s = W.make_system(3, 128, phi=0.90, dist="bi", T=0.0, seed=1)
    E0 = orc.forces(s.x, s.sigma, s.L)[1]
    out = orc.fire(s.x, s.sigma, s.L)
    assert out["status"] == 0 and out["fmax"] < 1e-10
    assert 0.0 < out["E"] < E0
    # independently: forces at the returned positions are below tolerance
    F, E, _ = orc.forces(out["x"], s.sigma, s.L)
    assert np.linalg.norm(F, axis=1).max() < 1e-10
    assert E == pytest.approx(out["E"], rel=1e-9)


def _fire_energies(orc, s, K):
    """E_pair after k = 0..K iterations, each from its own run capped at k
    iterations (the paper's stop criteria end a run; they never change its
    path)."""
    return np.array([orc.fire(s.x, s.sigma, s.L, max_iter=k)["E"] for k in range(K + 1)])


@pytest.mark.parametrize("th", [3e-3, 1e-3])
def test_fire_fractional_drop_stop_is_first_passage(orc, th):
    """Sec. II.B, Eq. (6): the run ends at the first iteration that closes ten
    consecutive fractional energy drops below F_thres."""
    s = W.make_system(3, 64, phi=0.75, dist="poly", T=0.0, seed=4)
    r = orc.fire(s.x, s.sigma, s.L, f_thres=th)
    E = _fire_energies(orc, s, r["iters"])
    below = np.abs(np.diff(E) / E[:-1]) < th          # drop into iteration k: index k-1
    first = next((k for k in range(10, len(E)) if below[k - 10:k].all()), None)
    assert first == r["iters"] and r["status"] == 0
    assert r["E"] == E[first]


@pytest.mark.parametrize("et", [1e-2, 5e-3])
def test_fire_energy_threshold_stop_is_first_passage(orc, et):
    """Sec. II.B: the run ends at the first iteration whose energy per atom
    is below E_thres."""
    s = W.make_system(3, 64, phi=0.75, dist="poly", T=0.0, seed=4)
    r = orc.fire(s.x, s.sigma, s.L, e_thres=et)
    per_atom = _fire_energies(orc, s, r["iters"]) / s.N
    assert per_atom[-1] < et and (per_atom[:-1] >= et).all()
    assert r["status"] == 0


def test_fire_displacement_cap_two_spheres(orc):
    """Two unit spheres 0.2 apart: each feels |f| = 1 - 0.2 = 0.8 and starts
    at rest, so the first FIRE iteration moves each by dt^2 f (here 2e-5)
    unless Delta_max (Table II) is smaller, when it moves Delta_max."""
    x = np.array([[0.0, 0.0, 0.0], [0.2, 0.0, 0.0]])
    sig = np.ones(2)
    dt = 0.005
    sep = lambda r: r["x"][1, 0] - r["x"][0, 0]
    assert sep(orc.fire(x, sig, 10.0, max_iter=1)) == pytest.approx(0.2 + 2 * dt * dt * 0.8, rel=1e-12)
    assert sep(orc.fire(x, sig, 10.0, max_iter=1, dx_max=1e-5)) == pytest.approx(0.2 + 2e-5, rel=1e-12)
    assert sep(orc.fire(x, sig, 10.0, max_iter=1, dx_max=1.0)) == pytest.approx(0.2 + 2 * dt * dt * 0.8, rel=1e-12)


def test_fire_displacement_cap_bounds_every_iteration(orc):
    """With Delta_max set no atom moves more than Delta_max per move: at most
    2 Delta_max per iteration (a back-off and a step), and the cap is reached."""
    s = W.make_system(3, 64, phi=0.75, dist="poly", T=0.0, seed=4)
    cap = 0.01

    def steps(**kw):
        prev, out = s.x, []
        for k in range(1, 80):
            xk = orc.fire(s.x, s.sigma, s.L, max_iter=k, **kw)["x"]
            dx = xk - prev
            dx -= s.L * np.round(dx / s.L)
            out.append(np.linalg.norm(dx, axis=1).max())
            prev = xk
        return np.array(out)

    free, capped = steps(), steps(dx_max=cap)
    assert free.max() > 2 * cap                       # the cap matters on this path
    assert capped.max() <= 2 * cap * (1 + 1e-12)
    assert (capped >= cap * (1 - 1e-12)).any()


def test_fire_displacement_cap_holds_for_the_back_off(orc):
    """A sphere pushed off its neighbour runs into a third one; there the
    power turns negative while it moves fast, and FIRE backs off by
    (dt/2) v.  That move too is capped at Delta_max, so no iteration moves an
    atom more than 2 Delta_max until the run converges."""
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.0], [1.6, 0.0, 0.0]])
    sig = np.ones(3)
    L, cap = 12.0, 0.002
    r = orc.fire(x, sig, L, dx_max=cap)
    assert r["status"] == 0
    prev, worst = x, 0.0
    for k in range(1, r["iters"] + 1):
        xk = orc.fire(x, sig, L, max_iter=k, dx_max=cap)["x"]
        dx = xk - prev
        dx -= L * np.round(dx / L)
        worst = max(worst, np.linalg.norm(dx, axis=1).max())
        prev = xk
    assert cap <= worst <= 2 * cap * (1 + 1e-12)


# ------------------------------------------------------------------ SWAP
def test_swap_delta_e_equals_total_energy_change(orc):
    s = W.make_system(3, 120, phi=0.6, dist="bi", T=0.0, seed=9)
    rng = np.random.default_rng(0)
    T = 0.05
    checked = 0
    for _ in range(40):
        i, j = rng.choice(s.N, 2, replace=False)
        if s.sigma[i] == s.sigma[j]:
            continue
        E0 = orc.forces(s.x, s.sigma, s.L)[1]
        sw = s.sigma.copy(); sw[i], sw[j] = sw[j], sw[i]
        E1 = orc.forces(s.x, sw, s.L)[1]
        thr = math.exp(-(E1 - E0) / T)
        if not (1e-6 < thr < 1 - 1e-6):
            continue
        for u, expect in ((thr * (1 - 1e-7), True), (thr * (1 + 1e-7), False)):
            out = orc.swap(s.x, s.sigma, s.L, T, [[i, j]], [u])
            assert bool(out["accepted"][0]) == expect
        checked += 1
    assert checked >= 5


def test_swap_equal_diameters_and_infinite_temperature(orc):
    s = W.make_system(4, 100, phi=0.4, dist="bi", T=0.0, seed=3)
    rng = np.random.default_rng(1)
    pairs, u = W.swap_pairs(rng, s.N, 50)
    out = orc.swap(s.x, np.ones(s.N), s.L, 1e-3, pairs, u)
    assert out["accepted"].all()
    out = orc.swap(s.x, s.sigma, s.L, 1e300, pairs, u)
    assert out["accepted"].all()
    # the exchanges compose as a product of transpositions
    sig = s.sigma.copy()
    for i, j in pairs:
        sig[i], sig[j] = sig[j], sig[i]
    assert (out["sigma"] == sig).all()


def test_swap_keeps_each_kinetic_energy(orc):
    s = W.make_system(3, 60, phi=0.5, dist="bi", T=1e-2, seed=5)
    mass = s.sigma ** 3
    pairs, u = W.swap_pairs(np.random.default_rng(2), s.N, 40)
    out = orc.swap(s.x, s.sigma, s.L, 1e300, pairs, u, mass=mass, v=s.v)
    k0 = 0.5 * mass * (s.v ** 2).sum(axis=1)
    k1 = 0.5 * out["mass"] * (out["v"] ** 2).sum(axis=1)
    assert np.allclose(k0, k1, rtol=1e-13)
    assert (out["mass"] == out["sigma"] ** 3).all()


def test_swap_detailed_balance_three_particles(orc):
    # fixed positions, diameters {a, a, b}: three states (who holds b); the
    # chain of SWAP passes must visit them with Boltzmann weights.
    x = np.array([[0.0, 0.0], [0.95, 0.0], [0.3, 0.9]])
    L = 8.0
    a, b = 1.0, 1.3
    T = 0.02
    E = []
    for k in range(3):
        sg = np.full(3, a); sg[k] = b
        E.append(orc.forces(x, sg, L)[1])
    E = np.array(E)
    w = np.exp(-(E - E.min()) / T)
    p = w / w.sum()
    assert p.min() > 0.05            # all states matter
    rng = np.random.default_rng(123)
    sg = np.array([b, a, a])
    visits = np.zeros(3)
    n = 60000
    pairs, u = W.swap_pairs(rng, 3, n)
    for blk in range(0, n, 2000):
        out = orc.swap(x, sg, L, T, pairs[blk:blk + 2000], u[blk:blk + 2000])
        # count the state after each attempt by replaying the accepted ones
        cur = sg.copy()
        for (i, j), acc in zip(pairs[blk:blk + 2000], out["accepted"]):
            if acc:
                cur[i], cur[j] = cur[j], cur[i]
            visits[int(np.argmax(cur))] += 1
        assert (cur == out["sigma"]).all()
        sg = out["sigma"]
    freq = visits / visits.sum()
    # loose chi-square-like bound for a correlated chain of 6e4 steps
    assert np.abs(freq - p).max() < 0.02, (freq, p)


# ------------------------------------------------------------------ Philox
@pytest.mark.parametrize("row", read_golden("philox4x32_10_kat.txt"))
def test_philox_known_answers(orc, row):
    ctr = [int(v, 16) for v in row[0:4]]
    key = [int(v, 16) for v in row[4:6]]
    out = [int(v, 16) for v in row[6:10]]
    assert orc.philox4x32_10(ctr, key).tolist() == out


def test_swap_draw_properties(orc):
    pairs, u = orc.swap_draw(12345, 3, 20000, 1000)
    assert (pairs[:, 0] != pairs[:, 1]).all()
    assert pairs.min() >= 0 and pairs.max() < 1000
    assert (u >= 0).all() and (u < 1).all()
    assert abs(u.mean() - 0.5) < 0.01
    hist = np.bincount(pairs.ravel(), minlength=1000)
    assert hist.min() > 10
    p2, u2 = orc.swap_draw(12345, 4, 20000, 1000)
    assert not (p2 == pairs).all()


# ------------------------------------------------------------------ Morse law (Eq. (1))
@pytest.mark.parametrize("row", read_golden("table3_phi_star.txt"))
def test_table3_effective_diameters(orc, row):
    """Eq. (12) with the Morse law of Eq. (1) reproduces Table III: the
    printed [sigma_eff(30, 0.25)]^d to 4 digits, and phi*_d = phi_d /
    sigma_eff^d to within 1e-4 (the printed d = 3 entry, 0.5980, exceeds the
    quotient 0.59794 by 0.6e-4)."""
    d, phi_d, seff_d, phi_star = int(row[0]), float(row[1]), float(row[2]), float(row[3])
    se = orc.sigma_eff(30.0, 0.25) ** d
    assert round(se, 4) == seff_d
    assert abs(phi_d / se - phi_star) <= 1e-4
    assert W.PHI_STAR[d] == phi_star


def test_morse_closed_forms(orc):
    a, s, eps = 30.0, 1.1, 0.7
    assert orc.morse(s, s, eps, a) == (0.0, 0.0)                    # truncated at r = s
    assert orc.morse(s + 0.1, s, eps, a) == (0.0, 0.0)
    r = s - math.log(2.0) / a                                         # exp(-a(r-s)) = 2
    u, fr = orc.morse(r, s, eps, a)
    assert u == pytest.approx(eps, rel=1e-14)                         # eps (4 - 4 + 1)
    assert fr * r == pytest.approx(4.0 * a * eps, rel=1e-14)          # eps (2a 4 - 2a 2)
    # just inside the cutoff U ~ eps a^2 (s - r)^2, the harmonic-like limit
    dr = 1e-5
    u, fr = orc.morse(s - dr, s, eps, a)
    assert u == pytest.approx(eps * a * a * dr * dr, rel=1e-3)
    assert fr * (s - dr) == pytest.approx(2 * eps * a * a * dr, rel=1e-3)


@pytest.mark.parametrize("d", [3, 5])
def test_volume_scaled_prefactors_two_bodies(orc, d):
    """eps_i = sigma_i^d mixed as sqrt(eps_i eps_j) (Sec. II.A): a pair's
    energy is (sigma_i sigma_j)^(d/2) times the unit-prefactor law."""
    L = 10.0
    x = np.zeros((2, d))
    x[1, 0] = 0.93
    sigma = np.array([0.9, 1.1])
    for kind, base in (("morse", lambda r, s: orc.morse(r, s, 1.0, 30.0)[0]),
                       ("harmonic", lambda r, s: orc.harmonic(r, s, 1.0)[0])):
        with orc.law(kind, 30.0, eps_scale=True):
            _, E, _ = orc.forces(x, sigma, L)
        assert E == pytest.approx((0.9 * 1.1) ** (0.5 * d) * base(0.93, 1.0), rel=1e-13)


@pytest.mark.parametrize("d", [3, 4, 6])
def test_morse_force_is_minus_gradient(orc, d):
    rng = np.random.default_rng(40 + d)
    s = W.paper_model(d, 40, phi=0.3 * W.PHI_STAR[d], seed=d)
    x, sigma, L = s.x, s.sigma, s.L
    with orc.law("morse", 30.0, eps_scale=True):
        F, E, _ = orc.forces(x, sigma, L)
        assert E > 0
        h = 1e-7
        for i in rng.choice(len(x), 6, replace=False):
            for k in range(d):
                xp = x.copy(); xp[i, k] += h
                xm = x.copy(); xm[i, k] -= h
                fd = -(orc.forces(xp, sigma, L)[1] - orc.forces(xm, sigma, L)[1]) / (2 * h)
                assert fd == pytest.approx(F[i, k], rel=1e-5, abs=1e-6 * np.abs(F).max())


@pytest.mark.parametrize("d,delta", [(3, 0.1056), (4, 0.0991), (5, 0.0910), (6, 0.0834)])
def test_power_law_diameters_polydispersity(d, delta):
    """Eq. (3) with R = d: the polydispersity index Delta from the
    distribution's closed-form moments (the paper prints 0.107, 0.099, 0.091,
    0.083), and the sampler's moments against them."""
    lo, hi = d ** (-0.5 / d), d ** (0.5 / d)

    def moment(k):   # integral of sigma^(k-d) over [lo, hi], normalised
        def prim(p, a, b):
            return math.log(b / a) if p == -1 else (b ** (p + 1) - a ** (p + 1)) / (p + 1)
        return prim(k - d, lo, hi) / prim(-d, lo, hi)

    m1, m2 = moment(1), moment(2)
    D = math.sqrt(m2 - m1 * m1) / m1
    assert round(D, 4) == delta
    sig = W.power_law_diameters(np.random.default_rng(d), 400000, d, float(d))
    assert sig.min() >= lo and sig.max() <= hi
    assert sig.mean() == pytest.approx(m1, rel=2e-3)
    assert (sig.std() / sig.mean()) == pytest.approx(D, rel=2e-2)


# ------------------------------------------------------------------ Berendsen thermostat
def _ideal_gas(d=3, N=400, seed=3):
    """Atoms too small to touch (sigma = 1e-3 in a box of side 6): no forces.
    Runs use a skin of 2 so that the box holds only 3 subcells per axis."""
    rng = np.random.default_rng(seed)
    L = 6.0
    x = W.uniform_positions(rng, N, d, L)
    sigma = np.full(N, 1e-3)
    v = W.thermal_velocities(rng, N, d, 0.7)
    return x, v, sigma, L


def test_berendsen_ideal_gas_relaxes_exponentially(orc):
    """Without forces T_{n+1} = lambda^2 T_n = T_n + (dt/tau)(T_t - T_n), so
    T_n - T_t = (T_0 - T_t)(1 - dt/tau)^n (Berendsen et al. 1984)."""
    x, v, sigma, L = _ideal_gas()
    N, d = x.shape
    T0 = 2 * orc.kinetic(v) / (d * (N - 1))
    assert T0 == pytest.approx(0.7, rel=1e-12)
    dt, tau, Tt = 0.005, 0.1, 0.25
    for n in (1, 7, 40):
        r = orc.md_steps(x, v, sigma, L, n, dt, skin=2.0, T_target=Tt, tau=tau)
        T = 2 * r["K"] / (d * (N - 1))
        assert T - Tt == pytest.approx((T0 - Tt) * (1 - dt / tau) ** n, rel=1e-10)


def test_berendsen_with_tau_equal_dt_hits_the_target_in_one_step(orc):
    x, v, sigma, L = _ideal_gas(d=4, N=300, seed=5)
    N, d = x.shape
    r = orc.md_steps(x, v, sigma, L, 1, 0.004, skin=2.0, T_target=0.3, tau=0.004)
    assert 2 * r["K"] / (d * (N - 1)) == pytest.approx(0.3, rel=1e-12)
    r0 = orc.md_steps(x, v, sigma, L, 1, 0.004, skin=2.0)       # NVE: unchanged
    assert r0["K"] == pytest.approx(orc.kinetic(v), rel=1e-14)


# ------------------------------------------------------------------ observables (Sec. II.E)
@pytest.mark.parametrize("d", [2, 3, 6])
def test_observables_of_a_uniform_translation(orc, d):
    """Every atom moved by the same vector c: msd = |c|^2, mqd = |c|^4,
    alpha2 = d/(d+2) - 1, f_ov = [|c| < a], G_s one bin holding 1/w."""
    rng = np.random.default_rng(d)
    N, L = 200, 9.0
    x0 = W.uniform_positions(rng, N, d, L)
    c = rng.normal(size=d)
    c *= 0.37 / np.linalg.norm(c)
    sigma = np.full(N, 0.01)
    for a, fov in ((0.5, 1.0), (0.3, 0.0)):
        r = orc.observables(x0 + c, x0, sigma, L, a, nbins=10, r_max=1.0)
        assert r["msd"] == pytest.approx(0.37 ** 2, rel=1e-13)
        assert r["mqd"] == pytest.approx(0.37 ** 4, rel=1e-13)
        assert r["alpha2"] == pytest.approx(d / (d + 2.0) - 1.0, abs=1e-12)
        assert r["f_ov"] == fov
        assert r["G_s"][3] == pytest.approx(1.0 / 0.1, rel=1e-12)
        assert r["G_s"].sum() * 0.1 == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("d", [3, 5])
def test_non_gaussian_parameter_vanishes_for_gaussian_displacements(orc, d):
    rng = np.random.default_rng(10 + d)
    N = 200000
    x0 = np.zeros((N, d))
    dx = rng.normal(scale=0.2, size=(N, d))
    r = orc.observables(dx, x0, None, 1e6, 0.1)
    assert abs(r["alpha2"]) < 0.02
    assert r["msd"] == pytest.approx(d * 0.04, rel=0.01)


@pytest.mark.parametrize("d,sig,expect", [(2, 1.05, 4), (3, 1.05, 6), (3, 1.45, 18), (4, 1.05, 8)])
def test_coordination_on_lattices(orc, d, sig, expect):
    x, L = W.lattice(d, 5)
    r = orc.observables(x, x, np.full(len(x), sig), L, 0.1)
    assert r["Z"] == expect


# ------------------------------------------------------------------ Mie law (Sec. II.A)
def test_mie_n6_is_the_wca_form(orc):
    """For n = 6 the truncated and shifted Mie law is WCA: 4 eps [(s'/r)^12 -
    (s'/r)^6] + eps for r < 2^(1/6) s' with s' = s 2^(-1/6)."""
    eps, s = 0.8, 1.1
    sp = s * 2.0 ** (-1.0 / 6.0)
    for r in (0.7, 0.95, 1.05, 1.0999):
        u, fr = orc.mie(r, s, eps, 6)
        lj = 4 * eps * ((sp / r) ** 12 - (sp / r) ** 6) + eps
        flj = 4 * eps * (12 * sp ** 12 / r ** 13 - 6 * sp ** 6 / r ** 7)
        assert u == pytest.approx(lj, rel=1e-12, abs=1e-15)
        assert fr * r == pytest.approx(flj, rel=1e-12, abs=1e-15)
    assert orc.mie(1.1, s, eps, 6) == (0.0, 0.0)


@pytest.mark.parametrize("n", [3, 8, 12])
def test_mie_closed_forms_and_gradient(orc, n):
    eps, s = 1.3, 0.9
    r = s * 2.0 ** (-1.0 / n)                   # (s/r)^n = 2
    u, fr = orc.mie(r, s, eps, n)
    assert u == pytest.approx(eps, rel=1e-13)   # eps (4 - 4 + 1)
    assert fr * r * r == pytest.approx(4 * n * eps, rel=1e-13)
    h = 1e-6
    for r in (0.6, 0.8, 0.89):
        fd = -(orc.mie(r + h, s, eps, n)[0] - orc.mie(r - h, s, eps, n)[0]) / (2 * h)
        assert fd == pytest.approx(orc.mie(r, s, eps, n)[1] * r, rel=1e-6)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_berendsen_barostat_ideal_gas_volume_relaxes_geometrically(orc, d):
    """No forces: P_n = N T / V_n with T fixed, and mu^d = 1 - c (P_t - P_n),
    c = beta n_baro dt / tau_P, so V_{n+1} - V* = (1 - c P_t)(V_n - V*) with
    V* = N T / P_t."""
    x, v, sigma, L = _ideal_gas(d=d, N=400, seed=7)
    N, d = x.shape
    T = 2 * orc.kinetic(v) / (d * (N - 1))
    Pt, tau_P, beta, nb, dt = 2.5, 0.5, 0.3, 10, 0.004
    c = beta * nb * dt / tau_P
    Vs = N * T * (N - 1) / N / Pt          # P = 2K/(dV) = (N - 1) T / V
    V0 = L ** d
    for cycles in (1, 3, 8):
        r = orc.md_npt(x, v, sigma, L, cycles * nb, dt, Pt, tau_P, beta, nb, skin=2.0)
        assert r["rescales"] == cycles
        assert r["L"] ** d - Vs == pytest.approx((1 - c * Pt) ** cycles * (V0 - Vs), rel=1e-9)


def test_paper_rebuild_rule_counts_and_misses(orc):
    """The paper's rule (Sec. II.C) rebuilds no more often than the exact
    one, only at multiples of n_bet, and can leave forces inexact; with the
    exact rule the forces equal brute force."""
    s = W.make_system(3, 600, phi=0.5, dist="poly", T=0.05, seed=4)
    ex = orc.md_steps(s.x, s.v, s.sigma, s.L, 300, 0.005, skin=0.3)
    pp = orc.md_steps(s.x, s.v, s.sigma, s.L, 300, 0.005, skin=0.3, rule="paper", n_bet=5)
    assert pp["step"] == 300
    assert 1 <= pp["builds"] <= ex["builds"]
    Fb, _, _ = orc.forces(ex["x"], s.sigma, s.L)
    assert np.abs(ex["F"] - Fb).max() < 1e-12 * np.abs(Fb).max()


@pytest.mark.parametrize("movers,period", [(1, 28), (2, 14)])
def test_paper_rule_thresholds(orc, movers, period):
    """Sec. II.C: rebuild when at least 0.1 % of the atoms have moved s/2 or
    more since the last build, or any atom s or more.  Of 2000 atoms at rest
    (too small to touch), `movers` fly 0.011 per step: one mover (0.05 %)
    triggers a build each time it has flown s = 0.3 (every 28 steps), two
    (0.1 %) each time they have flown s/2 (every 14 steps).  Checked every
    step (n_bet = 1), over 200 steps, plus the initial build."""
    d, N, L = 2, 2000, 60.0
    x, _ = W.lattice(d, 45, 60.0 / 45)
    x = x[:N].copy()
    v = np.zeros((N, d))
    v[:movers, 0] = 1.1
    x[:movers, 1] += 0.5              # off the lattice rows they fly along
    sigma = np.full(N, 1e-3)
    r = orc.md_steps(x, v, sigma, L, 200, 0.01, skin=0.3, rule="paper", n_bet=1)
    assert r["builds"] == 1 + 200 // period


def test_image_counts_unwrap_free_flight(orc):
    """Atoms that never touch fly straight: x + L img equals x0 + v t after
    several crossings of both faces of the box."""
    d, L = 3, 6.0
    x = np.array([[0.1, -2.9, 2.0], [-1.0, 1.0, -2.5], [2.5, 0.3, 0.0],
                  [-2.2, -1.4, 1.1], [1.3, 2.6, -0.7], [0.0, 0.0, 0.0]])
    v = np.array([[2.3, -1.7, 0.4], [-3.1, 0.2, 1.9], [0.7, 2.8, -2.6],
                  [1.5, -0.9, -3.3], [-0.6, 3.4, 0.8], [2.9, 2.1, -1.2]])
    sigma = np.full(len(x), 1e-3)
    r = orc.md_steps(x, v, sigma, L, 1000, 0.01, skin=2.0)
    assert np.abs(r["x"] + L * r["img"] - (x + 10.0 * v)).max() < 1e-9
    assert r["img"].max() >= 3 and r["img"].min() <= -3
    assert np.all(r["x"] >= -0.5 * L) and np.all(r["x"] < 0.5 * L)


def test_fire_mixing_and_schedule_seen_from_the_trajectory(orc):
    """FIRE 2.0 (Guenole et al. 2020) observed from outside, from the states
    after k and k + 1 iterations (capped runs).  An iteration with
    P = F.v > 0 moves x by dt v_{k+1} with v_{k+1} = (1 - alpha) v' +
    alpha |v'| F/|F|, v' = v_k + dt F_k (norms over all atoms); one with
    P <= 0 restarts from rest (v_{k+1} = dt F_k).  The dt so measured never
    exceeds dt_max and reaches it; a P <= 0 step past the initial delay
    multiplies dt by f_dec and sets alpha back to alpha0 (it had decayed).
    The scene: a sphere pushed off its neighbour runs into a third (the
    P <= 0 step), while a separate pair far away keeps F and v apart so that
    alpha is measurable."""
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.05, 0.0], [1.6, 0.0, 0.0],
                  [-4.0, 0.0, 0.0], [-4.0, 0.9, 0.0]])
    sig = np.ones(5)
    L, dt_max, f_dec, alpha0, n_delay = 12.0, 0.02, 0.5, 0.25, 20
    K = 110
    runs = [orc.fire(x, sig, L, max_iter=k, dt_max=dt_max) for k in range(K + 2)]
    dts, alphas, events = {}, {}, []
    for k in range(1, K + 1):
        a, b = runs[k], runs[k + 1]
        P = float((a["F"] * a["v"]).sum())
        v1 = b["v"]
        if P > 0:
            dx = b["x"] - a["x"]
            dx -= L * np.round(dx / L)
            dt = float((dx * v1).sum() / (v1 * v1).sum())
            assert np.abs(dx - dt * v1).max() <= 1e-12 * np.abs(v1).max() * dt + 1e-15
            vp = a["v"] + dt * a["F"]
            u = np.linalg.norm(vp) * a["F"] / np.linalg.norm(a["F"]) - vp
            if np.linalg.norm(u) > 1e-2 * np.linalg.norm(vp):     # alpha well defined
                al = float(((v1 - vp) * u).sum() / (u * u).sum())
                assert np.abs(v1 - (vp + al * u)).max() <= 1e-9 * np.abs(v1).max()
                alphas[k] = al
        else:
            dt = float(np.linalg.norm(v1) / np.linalg.norm(a["F"]))
            assert np.abs(v1 - dt * a["F"]).max() <= 1e-12 * np.abs(v1).max()
            events.append(k)
        dts[k] = dt
    assert max(dts.values()) <= dt_max * (1 + 1e-9)
    assert max(dts.values()) >= dt_max * (1 - 1e-9)
    # dt grows only after N_delay = 20 steps with P > 0 (iteration 0 starts
    # from rest, P = 0): dt0 through iteration 20, dt0 f_inc at 21
    assert all(dts[k] == pytest.approx(0.005, rel=1e-9) for k in range(1, n_delay + 1))
    assert dts[n_delay + 1] == pytest.approx(0.005 * 1.1, rel=1e-9)
    late = [k for k in events if k > n_delay]
    assert late, events
    j = late[0]
    assert dts[j] == pytest.approx(f_dec * dts[j - 1], rel=1e-9)
    assert alphas[j + 1] == pytest.approx(alpha0, rel=1e-6)
    assert alphas[j - 1] < 0.8 * alpha0


def _collision_scene():
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.05, 0.0], [1.6, 0.0, 0.0],
                  [-4.0, 0.0, 0.0], [-4.0, 0.9, 0.0]])
    return x, np.ones(5), 12.0


def _dt_of_step(a, b, L):
    """dt of the iteration from state a to state b, read off x_b - x_a =
    dt v_b (no displacement cap)."""
    dx = b["x"] - a["x"]
    dx -= L * np.round(dx / L)
    return float((dx * b["v"]).sum() / (b["v"] * b["v"]).sum())


@pytest.mark.parametrize("dt_min,halves", [(0.015, False), (1e-4, True)])
def test_fire_dt_back_off_only_above_dt_min(orc, dt_min, halves):
    """FIRE 2.0 (Guenole et al. 2020, Algorithm 2): on P <= 0 past the
    initial delay dt is multiplied by f_dec only when f_dec dt >= dt_min, and
    is left unchanged otherwise.  With dt_min = 0.015 above f_dec dt at the
    collision (dt <= dt_max = 0.02) the step after it runs with the dt of the
    step before (a floor at dt_min would give 0.015 instead, raising a dt
    below dt_min to it); with the default dt_min it runs with f_dec dt.  The
    velocity restarts from rest (v = dt F, unit masses)."""
    x, sig, L = _collision_scene()
    kw = dict(dt_max=0.02, dt_min=dt_min)
    runs = {}

    def run(k):
        if k not in runs:
            runs[k] = orc.fire(x, sig, L, max_iter=k, **kw)
        return runs[k]

    for k in range(22, 200):
        a = run(k)
        if float((a["F"] * a["v"]).sum()) <= 0:
            b = run(k + 1)
            dt = np.linalg.norm(b["v"]) / np.linalg.norm(a["F"])
            assert np.abs(b["v"] - dt * a["F"]).max() <= 1e-12 * np.abs(b["v"]).max()
            dt_before = _dt_of_step(run(k - 1), a, L)
            assert 0.005 <= dt_before <= 0.02 * (1 + 1e-9)
            if halves:
                assert dt == pytest.approx(0.5 * dt_before, rel=1e-9)
            else:
                assert 0.5 * dt_before < dt_min
                assert dt == pytest.approx(dt_before, rel=1e-9)
            return
    pytest.fail("no P <= 0 step")


def test_fire_mixing_in_every_step_with_masses(orc):
    """FIRE 2.0 mixes v = (1 - alpha) v + alpha |v| F/|F| in every MD
    integration step, after v += dt F/m.  With unequal masses m = sigma^d
    the first iteration (P = 0 from rest, a P <= 0 step inside the initial
    delay: dt = dt0, alpha = alpha0) therefore gives, in closed form,
    v_1 = (1 - alpha0) dt0 F/m + alpha0 dt0 |F/m| F/|F| (norms over all atoms)
    and x_1 = x_0 + dt0 v_1; mixing only on P > 0 would give v_1 = dt0 F/m.
    The same form holds at a later P <= 0 step past the delay, with
    alpha = alpha0 and dt = f_dec dt_before."""
    x, _, L = _collision_scene()
    x[2, 0] = 1.8
    sig = np.array([1.0, 1.0, 1.4, 1.2, 0.9])   # the pushed sphere meets a heavy one
    m = sig ** 3
    dt0, alpha0 = 0.005, 0.25
    F0, _, _ = orc.forces(x, sig, L)
    a1 = dt0 * F0 / m[:, None]
    v1 = (1 - alpha0) * a1 + alpha0 * np.linalg.norm(a1) * F0 / np.linalg.norm(F0)
    r1 = orc.fire(x, sig, L, mass=m, max_iter=1)
    assert np.abs(r1["v"] - v1).max() <= 1e-13 * np.abs(v1).max()
    dx = r1["x"] - x
    dx -= L * np.round(dx / L)
    # positions carry the rounding of coordinates up to |x| = 4
    assert np.abs(dx - dt0 * v1).max() <= 4 * np.finfo(float).eps * np.abs(x).max()
    # the mixing changes v_1 by much more than rounding
    assert np.abs(v1 - a1).max() > 1e-3 * np.abs(a1).max()
    kw = dict(dt_max=0.02)
    for k in range(22, 200):
        a = orc.fire(x, sig, L, mass=m, max_iter=k, **kw)
        if float((a["F"] * a["v"]).sum()) < 0:
            b = orc.fire(x, sig, L, mass=m, max_iter=k + 1, **kw)
            prev = orc.fire(x, sig, L, mass=m, max_iter=k - 1, **kw)
            dxp = a["x"] - prev["x"]
            dxp -= L * np.round(dxp / L)
            dt_before = float((dxp * a["v"]).sum() / (a["v"] * a["v"]).sum())
            dt = 0.5 * dt_before
            ak = dt * a["F"] / m[:, None]
            vk = (1 - alpha0) * ak + alpha0 * np.linalg.norm(ak) * a["F"] / np.linalg.norm(a["F"])
            assert np.abs(b["v"] - vk).max() <= 1e-9 * np.abs(vk).max()
            return
    pytest.fail("no P <= 0 step")


def test_fire_negative_step_counter_counts_consecutive_steps(orc):
    """N_neg,max bounds consecutive P <= 0 steps: the start from rest
    (P = 0) and the collision are separated by P > 0 steps, so even
    n_neg_max = 1 lets the run converge as with the default."""
    x, sig, L = _collision_scene()
    ref = orc.fire(x, sig, L)
    r = orc.fire(x, sig, L, n_neg_max=1)
    assert ref["status"] == 0 and r["status"] == 0 and r["iters"] == ref["iters"]


def test_barostat_count_carries_across_calls(orc):
    """The barostat acts every n_baro steps counted across calls: 15 + 15
    steps rescale at steps 10, 20 and 30 like one call of 30."""
    x, v, sigma, L = _ideal_gas(d=3, N=400, seed=7)
    args = (2.5, 0.5, 0.3, 10)
    one = orc.md_npt(x, v, sigma, L, 30, 0.004, *args, skin=2.0)
    a = orc.md_npt(x, v, sigma, L, 15, 0.004, *args, skin=2.0)
    b = orc.md_npt(a["x"], a["v"], sigma, a["L"], 15, 0.004, *args, skin=2.0, img=a["img"],
                   count=a["count"])
    assert one["rescales"] == 3 and a["rescales"] == 1 and b["rescales"] == 2
    assert a["count"] == 5 and b["count"] == 0
    assert b["L"] == pytest.approx(one["L"], rel=1e-12)


@pytest.mark.parametrize("nsteps,builds", [(15, 1), (16, 2)])
def test_paper_rule_checked_at_multiples_of_n_bet(orc, nsteps, builds):
    """With n_bet = 4 the paper's rule is evaluated after steps 4, 8, 12,
    16, ...: two movers pass s/2 during step 14, so the rebuild comes at step
    16, not before."""
    d, N, L = 2, 2000, 60.0
    x, _ = W.lattice(d, 45, 60.0 / 45)
    x = x[:N].copy()
    v = np.zeros((N, d))
    v[:2, 0] = 1.1
    x[:2, 1] += 0.5
    r = orc.md_steps(x, v, np.full(N, 1e-3), L, nsteps, 0.01, skin=0.3, rule="paper", n_bet=4)
    assert r["builds"] == builds


def test_swap_draw_is_a_scaled_uniform(orc):
    """Each candidate index is one uniform variate scaled to its range:
    i = floor(U N) and j' = floor(U' (N - 1)) with U, U' fixed by seed, pass
    and pair, so i(N)/N (and j'(N)/(N - 1)) agree across N to within 1/N."""
    big = 1 << 26
    Ns = [2, 3, 7, 10, 97, 1000, 4093, 65536]
    pairs_big, _ = orc.swap_draw(2024, 5, 16, big)
    for p in range(16):
        i_big = int(pairs_big[p, 0])
        U_lo, U_hi = i_big / big, (i_big + 1) / big
        for N in Ns:
            pr, _ = orc.swap_draw(2024, 5, 16, N)
            i, j = int(pr[p, 0]), int(pr[p, 1])
            assert math.floor(U_lo * N) <= i <= math.floor(U_hi * N - 1e-12)
            assert 0 <= j < N and j != i
    # j' = j - (j > i), over N - 1 values
    for p in range(16):
        i_b, j_b = (int(t) for t in pairs_big[p])
        jp_big = j_b - (j_b > i_b)
        V_lo, V_hi = jp_big / (big - 1), (jp_big + 1) / (big - 1)
        for N in Ns[1:]:
            pr, _ = orc.swap_draw(2024, 5, 16, N)
            i, j = int(pr[p, 0]), int(pr[p, 1])
            jp = j - (j > i)
            assert math.floor(V_lo * (N - 1)) <= jp <= math.floor(V_hi * (N - 1) - 1e-12)


def test_kinetic_energy_with_masses(orc):
    v = np.array([[1.0, 0.0], [0.0, 2.0], [3.0, -1.0]])
    m = np.array([2.0, 3.0, 0.5])
    assert orc.kinetic(v, m) == pytest.approx(0.5 * (2 * 1 + 3 * 4 + 0.5 * 10), rel=1e-15)
    assert orc.kinetic(v) == pytest.approx(0.5 * (1 + 4 + 10), rel=1e-15)


def test_thermo_describes_the_returned_state(orc):
    """E and W returned by a run describe the state it returns, also after
    zero steps and when the run ends on a barostat rescaling: the brute-force
    all-pairs forces at the returned positions and box give the same E, W."""
    s = W.make_system(3, 300, phi=0.5, dist="poly", T=0.05, seed=12)
    r0 = orc.md_steps(s.x, s.v, s.sigma, s.L, 0, 0.005)
    F, E, Wv = orc.forces(s.x, s.sigma, s.L)
    assert r0["E"] == pytest.approx(E, rel=1e-12) and r0["W"] == pytest.approx(Wv, rel=1e-12)
    assert np.abs(r0["F"] - F).max() <= 1e-12 * np.abs(F).max()
    r0f = orc.md_steps(s.x, s.v, s.sigma, s.L, 0, 0.005, F=F)      # forces handed in
    assert r0f["E"] == pytest.approx(E, rel=1e-12) and r0f["W"] == pytest.approx(Wv, rel=1e-12)
    r = orc.md_npt(s.x, s.v, s.sigma, s.L, 20, 0.005, 1.0, 0.5, 0.3, 10)
    assert r["rescales"] == 2 and r["count"] == 0
    _, E1, W1 = orc.forces(r["x"], s.sigma, r["L"])
    assert r["E"] == pytest.approx(E1, rel=1e-12) and r["W"] == pytest.approx(W1, rel=1e-12)
