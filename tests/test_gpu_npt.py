"""GPU parity of the Berendsen barostat (NPT): the ideal-gas volume
relaxation in closed form, trajectories and box sides over several
rescalings against the oracle (1e-9 FP64, 1e-5 mixed), and a box that grows
past its subcell grid (the grid and lists are set up again) checked by the
oracle's forces."""
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


def test_ideal_gas_volume_relaxes_in_closed_form(H):
    rng = np.random.default_rng(7)
    d, N, L = 3, 400, 6.0
    x = W.uniform_positions(rng, N, d, L)
    v = W.thermal_velocities(rng, N, d, 0.7)
    sigma = np.full(N, 1e-3)
    Pt, tau_P, beta, nb, dt = 2.5, 0.5, 0.3, 10, 0.004
    c = beta * nb * dt / tau_P
    Vs = (N - 1) * 0.7 / Pt
    for cycles in (1, 3, 8):
        with H.System(d, L, sigma, x, v, skin=2.0, precision=H.HDMD_MIXED) as g:
            g.barostat(Pt, tau_P, beta, nb)
            g.md_steps(cycles * nb, dt)
            Lg = g.box()
        assert Lg ** d - Vs == pytest.approx((1 - c * Pt) ** cycles * (L ** d - Vs), rel=1e-9)


@pytest.mark.parametrize("nvt", [False, True])
def test_npt_trajectory_matches_oracle(H, nvt):
    s = W.c0_bidisperse_d3()
    Pt, tau_P, beta, nb = 0.02, 0.2, 0.5, 25
    Tt, tau = (5e-3, 0.05) if nvt else (0.0, 0.0)
    ref = oracle.md_npt(s.x, s.v, s.sigma, s.L, 110, 0.005, Pt, tau_P, beta, nb,
                        T_target=Tt, tau=tau)
    assert ref["rescales"] == 4 and ref["L"] != s.L
    for prec, tol in ((H.HDMD_FP64, 1e-9), (H.HDMD_MIXED, 1e-5)):
        with H.System(s.d, s.L, s.sigma, s.x, s.v, precision=prec) as g:
            g.barostat(Pt, tau_P, beta, nb)
            if nvt:
                g.thermostat(Tt, tau)
            g.md_steps(60, 0.005)            # two calls: the piece count carries over
            t = g.md_steps(50, 0.005)
            st = g.state()
            Lg = g.box()
        assert Lg == pytest.approx(ref["L"], rel=tol)
        dx = st["x"] + Lg * st["img"] - (ref["x"] + ref["L"] * ref["img"])
        assert np.abs(dx).max() < 10 * tol, (prec, np.abs(dx).max())
        assert t["E_pair"] == pytest.approx(ref["E"], rel=max(tol, 1e-11))
        assert t["K"] == pytest.approx(ref["K"], rel=max(tol, 1e-11))


def test_growing_box_sets_up_a_larger_subcell_grid(H):
    s = W.make_system(3, 2000, phi=0.5, dist="poly", T=0.02, seed=4)
    with H.System(3, s.L, s.sigma, s.x, s.v, precision=H.HDMD_FP64) as g:
        n0 = g.info()["n_cell"]
        g.barostat(1e-4, 0.05, 2.0, 5)      # far below the pressure: the box expands
        g.md_steps(200, 0.005)
        n1 = g.info()["n_cell"]
        L1 = g.box()
        F, E, Wv = g.forces()
        xs = g.state()["x"]
    assert L1 > s.L and n1 > n0
    Fo, Eo, Wo = oracle.forces(xs, s.sigma, L1)
    assert np.abs(F - Fo).max() <= 1e-12 * max(np.abs(Fo).max(), 1e-300) + 1e-300
    assert E == pytest.approx(Eo, rel=1e-12, abs=1e-300)
